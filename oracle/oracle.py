"""Python wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark use it.  The CUDA library never imports or calls it.  It consumes the
workload descriptions of `paper_2406_19212_gb300.inputs` (names, qubits, angles) and
builds every matrix itself in oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

_KIND = {name: i for i, name in enumerate(
    ["X", "Y", "Z", "H", "S", "T", "SX", "SY", "SW", "RX", "RY", "RZ",
     "CNOT", "CZ", "SWAP", "ISWAP", "FSIM", "CONTROL", "DENSE1", "DENSE2",
     "DEPOL", "AMPDAMP", "PHASEDAMP", "KRAUS", "DEPOL2", "KRAUS2"])}


class OrcOp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nq", ctypes.c_int32), ("q", ctypes.c_int32 * 2),
                ("param", ctypes.c_int32), ("n_kraus", ctypes.c_int32), ("pmask", ctypes.c_int32),
                ("fixed", ctypes.c_double * 5), ("data", ctypes.c_double * 32),
                ("kraus", ctypes.c_void_p)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP on the outer amplitude loops)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        op_p = ctypes.POINTER(OrcOp)
        L.orc_gate_matrix.argtypes = [op_p, dp, dp]
        L.orc_kraus.argtypes = [op_p, dp, ctypes.POINTER(ctypes.c_int)]
        L.orc_apply_matrix.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp]
        L.orc_apply_circuit.argtypes = [dp, ctypes.c_int, op_p, ctypes.c_int, dp]
        L.orc_apply_hamiltonian.argtypes = [dp, dp, ctypes.c_int, dp, ctypes.c_char_p, ctypes.c_int]
        L.orc_expect.argtypes = [dp, ctypes.c_int, dp, ctypes.c_char_p, ctypes.c_int, dp]
        L.orc_adjoint_grad.argtypes = [ctypes.c_int, op_p, ctypes.c_int, dp, ctypes.c_int, dp,
                                       ctypes.c_char_p, ctypes.c_int, dp, dp]
        L.orc_rho_apply_circuit.argtypes = [dp, ctypes.c_int, op_p, ctypes.c_int, dp]
        L.orc_rho_expect.argtypes = [dp, ctypes.c_int, dp, ctypes.c_char_p, ctypes.c_int, dp]
        L.orc_noisy_adjoint_grad.argtypes = [ctypes.c_int, op_p, ctypes.c_int, dp, ctypes.c_int,
                                             dp, ctypes.c_char_p, ctypes.c_int, dp, dp]
        L.orc_vec_apply_circuit.argtypes = [dp, ctypes.c_int, op_p, ctypes.c_int, dp]
        L.orc_measure.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_int), dp]
        L.orc_sample.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int64)]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ops(ops) -> ctypes.Array:
    arr = (OrcOp * max(1, len(ops)))()
    arr._keep = []  # KRAUS2 operator buffers referenced by pointer
    for i, op in enumerate(ops):
        o = arr[i]
        o.kind = _KIND[op.name]
        o.nq = len(op.qubits)
        for t, q in enumerate(op.qubits):
            o.q[t] = q
        o.param = op.param
        o.pmask = getattr(op, "pmask", 0)
        for t, v in enumerate(op.fixed):
            o.fixed[t] = v
        if op.name == "KRAUS2":
            ks = [np.asarray(k, dtype=np.complex128).reshape(4, 4) for k in op.data]
            o.n_kraus = len(ks)
            buf = np.ascontiguousarray(np.concatenate([k.reshape(-1) for k in ks])).view(np.float64)
            arr._keep.append(buf)
            o.kraus = buf.ctypes.data
        elif op.data is not None:
            if op.name == "KRAUS":
                ks = [np.asarray(k, dtype=np.complex128) for k in op.data]
                o.n_kraus = len(ks)
                flat = np.concatenate([k.reshape(-1) for k in ks])
            else:
                flat = np.asarray(op.data, dtype=np.complex128).reshape(-1)
            for t, v in enumerate(flat):
                o.data[2 * t] = v.real
                o.data[2 * t + 1] = v.imag
    return arr


def _theta(theta) -> np.ndarray:
    t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    return t if t.size else np.zeros(1)


def _paulis(terms, n: int) -> Tuple[np.ndarray, bytes]:
    coeff = np.array([float(c) for c, _ in terms], dtype=np.float64)
    s = bytearray(b"I" * (n * len(terms)))
    for t, (_, factors) in enumerate(terms):
        for q, p in factors:
            s[t * n + q] = ord(p)
    return coeff, bytes(s)


def gate_matrix(op, theta=()) -> np.ndarray:
    out = np.zeros(32)
    k = lib().orc_gate_matrix(_ops([op]), _dp(_theta(theta)), _dp(out))
    if k < 0:
        raise ValueError(op.name)
    d = 1 << k
    return (out[0:2 * d * d:2] + 1j * out[1:2 * d * d:2]).reshape(d, d)


def kraus(op) -> List[np.ndarray]:
    out = np.zeros(512)
    k = ctypes.c_int()
    m = lib().orc_kraus(_ops([op]), _dp(out), ctypes.byref(k))
    if m < 0:
        raise ValueError(op.name)
    d = 1 << k.value
    c = out[0::2] + 1j * out[1::2]
    return [c[d * d * s:d * d * (s + 1)].reshape(d, d) for s in range(m)]


def apply_matrix(psi: np.ndarray, n: int, qubits: Sequence[int], mat: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    m = np.ascontiguousarray(np.asarray(mat, dtype=np.complex128))
    qs = np.array(qubits, dtype=np.int32)
    rc = lib().orc_apply_matrix(_dp(psi.view(np.float64)), n, len(qubits),
                                qs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                _dp(m.view(np.float64)))
    assert rc == 0
    return psi


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_circuit(circuit, theta, psi=None) -> np.ndarray:
    n = circuit.n_qubits
    psi = zero_state(n) if psi is None else np.ascontiguousarray(psi, dtype=np.complex128).copy()
    rc = lib().orc_apply_circuit(_dp(psi.view(np.float64)), n, _ops(circuit.ops),
                                 len(circuit.ops), _dp(_theta(theta)))
    if rc != 0:
        raise ValueError(f"oracle apply_circuit failed ({rc})")
    return psi


def apply_hamiltonian(terms, psi: np.ndarray, n: int) -> np.ndarray:
    coeff, s = _paulis(terms, n)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros_like(psi)
    lib().orc_apply_hamiltonian(_dp(out.view(np.float64)), _dp(psi.view(np.float64)), n,
                                _dp(coeff), s, len(terms))
    return out


def expect(terms, psi: np.ndarray, n: int, return_imag: bool = False):
    coeff, s = _paulis(terms, n)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(2)
    lib().orc_expect(_dp(psi.view(np.float64)), n, _dp(coeff), s, len(terms), _dp(out))
    return (out[0], out[1]) if return_imag else out[0]


def adjoint_grad(circuit, theta, terms) -> Tuple[float, np.ndarray]:
    """Energy and gradient by Algorithm 2 (pure state)."""
    n = circuit.n_qubits
    coeff, s = _paulis(terms, n)
    e = np.zeros(1)
    g = np.zeros(max(1, circuit.n_params))
    rc = lib().orc_adjoint_grad(n, _ops(circuit.ops), len(circuit.ops), _dp(_theta(theta)),
                                circuit.n_params, _dp(coeff), s, len(terms), _dp(e), _dp(g))
    if rc != 0:
        raise ValueError(f"oracle adjoint_grad failed ({rc})")
    return float(e[0]), g[:circuit.n_params].copy()


def zero_density(n: int) -> np.ndarray:
    rho = np.zeros(1 << (2 * n), dtype=np.complex128)
    rho[0] = 1.0
    return rho


def rho_apply_circuit(circuit, theta, rho=None) -> np.ndarray:
    """Kraus-sum evolution of the 2^n x 2^n density matrix (vectorised a + 2^n b)."""
    n = circuit.n_qubits
    rho = zero_density(n) if rho is None else np.ascontiguousarray(rho, dtype=np.complex128).copy()
    rc = lib().orc_rho_apply_circuit(_dp(rho.view(np.float64)), n, _ops(circuit.ops),
                                     len(circuit.ops), _dp(_theta(theta)))
    if rc != 0:
        raise ValueError(f"oracle rho_apply_circuit failed ({rc})")
    return rho


def vec_apply_circuit(circuit, theta, rho=None) -> np.ndarray:
    """Superoperator evolution of |rho>> on 2n qubits (Eq. channel2)."""
    n = circuit.n_qubits
    rho = zero_density(n) if rho is None else np.ascontiguousarray(rho, dtype=np.complex128).copy()
    rc = lib().orc_vec_apply_circuit(_dp(rho.view(np.float64)), n, _ops(circuit.ops),
                                     len(circuit.ops), _dp(_theta(theta)))
    if rc != 0:
        raise ValueError(f"oracle vec_apply_circuit failed ({rc})")
    return rho


def rho_expect(terms, rho: np.ndarray, n: int, return_imag: bool = False):
    coeff, s = _paulis(terms, n)
    rho = np.ascontiguousarray(rho, dtype=np.complex128)
    out = np.zeros(2)
    lib().orc_rho_expect(_dp(rho.view(np.float64)), n, _dp(coeff), s, len(terms), _dp(out))
    return (out[0], out[1]) if return_imag else out[0]


def noisy_adjoint_grad(circuit, theta, terms) -> Tuple[float, np.ndarray]:
    """Energy tr(H rho) and gradient by the noisy Algorithm 2 (Sec. III.E)."""
    n = circuit.n_qubits
    coeff, s = _paulis(terms, n)
    e = np.zeros(1)
    g = np.zeros(max(1, circuit.n_params))
    rc = lib().orc_noisy_adjoint_grad(n, _ops(circuit.ops), len(circuit.ops),
                                      _dp(_theta(theta)), circuit.n_params, _dp(coeff), s,
                                      len(terms), _dp(e), _dp(g))
    if rc != 0:
        raise ValueError(f"oracle noisy_adjoint_grad failed ({rc})")
    return float(e[0]), g[:circuit.n_params].copy()


def energy(circuit, theta, terms) -> float:
    """Loss of Eq. (loss_pure) or Eq. (loss_mixed) by plain forward evolution."""
    if circuit.density:
        return rho_expect(terms, rho_apply_circuit(circuit, theta), circuit.n_qubits)
    return expect(terms, apply_circuit(circuit, theta), circuit.n_qubits)


def parameter_shift_grad(circuit, theta, terms, indices=None) -> np.ndarray:
    """g_j = [L(theta_j + pi/2) - L(theta_j - pi/2)] / 2, exact for parameters that each
    drive Pauli rotations exp(-i theta P / 2) (the loss is a trigonometric polynomial of
    degree one in each such angle when the angle appears once)."""
    theta = np.asarray(theta, dtype=np.float64)
    idx = range(len(theta)) if indices is None else indices
    out = []
    for j in idx:
        tp = theta.copy(); tp[j] += np.pi / 2
        tm = theta.copy(); tm[j] -= np.pi / 2
        out.append(0.5 * (energy(circuit, tp, terms) - energy(circuit, tm, terms)))
    return np.array(out)


def finite_difference_grad(circuit, theta, terms, indices, h: float = 1e-5) -> np.ndarray:
    theta = np.asarray(theta, dtype=np.float64)
    out = []
    for j in indices:
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        out.append((energy(circuit, tp, terms) - energy(circuit, tm, terms)) / (2 * h))
    return np.array(out)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def measure(state: np.ndarray, n: int, qubit: int, u: float, density: bool = False):
    """measure!(state, qubit) of Sec. II.D with the uniform draw u: returns
    (outcome, probability, collapsed state); the input is not modified."""
    st = np.ascontiguousarray(np.array(state, dtype=np.complex128).reshape(-1))
    outcome = ctypes.c_int()
    prob = ctypes.c_double()
    r = lib().orc_measure(_dp(st.view(np.float64)), n, int(bool(density)), qubit, float(u),
                          ctypes.byref(outcome), ctypes.byref(prob))
    if r != 0:
        raise ValueError("orc_measure failed")
    return outcome.value, prob.value, st


def sample(state: np.ndarray, n: int, u, density: bool = False) -> np.ndarray:
    """Basis indices sampled from |psi_a|^2 (or rho_aa) with the uniform draws u."""
    st = np.ascontiguousarray(np.array(state, dtype=np.complex128).reshape(-1))
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
    out = np.zeros(max(1, uu.size), dtype=np.int64)
    r = lib().orc_sample(_dp(st.view(np.float64)), n, int(bool(density)), _dp(uu), uu.size,
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if r != 0:
        raise ValueError("orc_sample failed")
    return out[:uu.size]
