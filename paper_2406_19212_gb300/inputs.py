"""Seeded synthetic workloads: circuits, parameter vectors and Pauli-sum observables.

This module only *describes* inputs (gate names, qubit lists, angles, Pauli strings).
It holds none of the simulation arithmetic: no gate matrices, no amplitudes, no
expectation values.  Both the CUDA library binding and the CPU oracle consume the
same descriptions, each turning names into matrices with its own code.

Conventions (paper Sec. II.A, II.B): qubits are 0-based and qubit q is bit q of the
amplitude index (the paper's "qubit 1 varies fastest", column-major).  For a gate on
the ordered qubits (q_0, ..., q_{k-1}) the first listed qubit is the least significant
bit of the gate-matrix index; CNOT/CONTROL list (control, target).  A density matrix
of n qubits is a 2n-qubit vector with ket bits low and bra bits high (Sec. III.D).

Random numbers come from numpy's PCG64 generator with the seed given.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Gate and channel names understood by both consumers (paper Sec. II.B).
ONE_QUBIT_FIXED = ("X", "Y", "Z", "H", "S", "T", "SX", "SY", "SW")
ROTATIONS = ("RX", "RY", "RZ")
TWO_QUBIT_FIXED = ("CNOT", "CZ", "SWAP", "ISWAP")
CHANNELS = ("DEPOL", "AMPDAMP", "PHASEDAMP", "KRAUS")
CHANNELS2 = ("DEPOL2", "KRAUS2")  # two-qubit QuantumMap: depolarising, general Kraus list
ALL_NAMES = ONE_QUBIT_FIXED + ROTATIONS + TWO_QUBIT_FIXED + (
    "FSIM", "CONTROL", "DENSE1", "DENSE2") + CHANNELS + CHANNELS2


@dataclass(frozen=True)
class Op:
    """One circuit element.

    name   : a name from ALL_NAMES.
    qubits : logical qubits; first listed = least significant bit of the matrix index.
    param  : index into the parameter vector theta for a variational rotation, -1 if fixed;
             for a variational FSIM the index of its first variational parameter.
    fixed  : fixed parameters: the angle of a fixed RX/RY/RZ, (theta, phi, d_plus,
             d_minus, d_minus_off) of FSIM (missing trailing entries are 0), the strength
             p or gamma of a channel.
    pmask  : FSIM with param >= 0: bit k set = parameter k of (theta, phi, d_plus,
             d_minus, d_minus_off) is variational (the paper's `isparas` array); the
             variational ones read theta[param], theta[param + 1], ... in increasing k.
    data   : complex matrix for DENSE1 (2x2), DENSE2 (4x4), CONTROL (2x2 target block),
             a list of 2x2 Kraus operators for KRAUS or of 4x4 ones for KRAUS2;
             row-major [row][col].
    """
    name: str
    qubits: Tuple[int, ...]
    param: int = -1
    fixed: Tuple[float, ...] = ()
    data: Optional[object] = None
    pmask: int = 0


@dataclass
class Circuit:
    n_qubits: int                 # logical qubits (density circuits act on 2n physical)
    ops: List[Op]
    n_params: int
    density: bool = False


# A Pauli term: (coefficient, ((qubit, 'X'|'Y'|'Z'), ...)); identity factors omitted.
PauliTerm = Tuple[float, Tuple[Tuple[int, str], ...]]


@dataclass
class Workload:
    name: str
    circuit: Circuit
    theta: np.ndarray
    observable: List[PauliTerm]
    extra: dict = field(default_factory=dict)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ising_chain(n: int, field_coeffs: Sequence[float]) -> List[PauliTerm]:
    """H = sum_{i<n-1} Z_i Z_{i+1} + sum_i h_i X_i (open boundary)."""
    terms: List[PauliTerm] = []
    for i in range(n - 1):
        terms.append((1.0, ((i, "Z"), (i + 1, "Z"))))
    for i in range(n):
        terms.append((float(field_coeffs[i]), ((i, "X"),)))
    return terms


def heisenberg_1d(n: int, hz: float = 1.0, J: float = 1.0) -> List[PauliTerm]:
    """Listing 5 of the paper: hz*sum Z_i + J*sum (X_iX_{i+1} + Y_iY_{i+1} + Z_iZ_{i+1})."""
    terms: List[PauliTerm] = [(hz, ((i, "Z"),)) for i in range(n)]
    for i in range(n - 1):
        for p in "XYZ":
            terms.append((J, ((i, p), (i + 1, p))))
    return terms


def hea_rx_rz_rx(n: int, layers: int, seed: int, field: float = 0.5,
                 name: str = "hea_rxrzrx") -> Workload:
    """Hardware-efficient ansatz: per layer Rx.Rz.Rx on every qubit, then CNOT(i,i+1).

    Parameter index = layer*(3n) + q*3 + k; angles uniform in [0, 2pi).
    Observable: sum Z_iZ_{i+1} + field * sum X_i, open boundary.
    """
    rng = _rng(seed)
    ops: List[Op] = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            for g in ("RX", "RZ", "RX"):
                ops.append(Op(g, (q,), param=p))
                p += 1
        for i in range(n - 1):
            ops.append(Op("CNOT", (i, i + 1)))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=p)
    return Workload(name, Circuit(n, ops, p), theta, ising_chain(n, [field] * n))


def plain_10q(seed: int = 0) -> Workload:
    """10 qubits, 4 layers of Rx.Rz.Rx + CNOT ladder, 120 angles, H = ZZ + 0.5 X."""
    return hea_rx_rz_rx(10, 4, seed, 0.5, name="plain_10q_hea4")


def _couplers(rows: int, cols: int, kind: int) -> List[Tuple[int, int]]:
    """Coupler pattern kind of a rows x cols grid (qubit = cols*r + c):
    A (0): (r,c)-(r,c+1), c even; B (1): c odd; C (2): (r,c)-(r+1,c), r even; D (3): r odd."""
    pairs = []
    for r in range(rows):
        for c in range(cols):
            q = cols * r + c
            if kind < 2 and c + 1 < cols and c % 2 == kind:
                pairs.append((q, q + 1))
            if kind >= 2 and r + 1 < rows and r % 2 == kind - 2:
                pairs.append((q, q + cols))
    return pairs


def grid_rqc(rows: int, cols: int, cycles: int, seed: int) -> Workload:
    """Random circuit on a rows x cols grid (qubit = cols*r + c).

    Each cycle: one of sqrt(X), sqrt(Y), sqrt(W) per qubit, never the same gate twice in
    a row on a qubit; then FSIM(theta = pi/2 + N(0,0.05), phi = pi/6 + N(0,0.05)) on every
    coupler of pattern [A, B, C, D][cycle mod 4]:
    A: (r,c)-(r,c+1), c even; B: c odd; C: (r,c)-(r+1,c), r even; D: r odd.
    Every gate is fixed (no variational parameters).
    """
    rng = _rng(seed)
    n = rows * cols
    ops: List[Op] = []
    last = [-1] * n
    names = ("SX", "SY", "SW")
    patterns = [_couplers(rows, cols, kind) for kind in range(4)]
    for t in range(cycles):
        for q in range(n):
            choices = [i for i in range(3) if i != last[q]]
            pick = choices[int(rng.integers(0, len(choices)))]
            last[q] = pick
            ops.append(Op(names[pick], (q,)))
        for (a, b) in patterns[t % 4]:
            th = math.pi / 2 + rng.normal(0.0, 0.05)
            ph = math.pi / 6 + rng.normal(0.0, 0.05)
            ops.append(Op("FSIM", (a, b), fixed=(th, ph)))
    return Workload(f"rqc_{rows}x{cols}_c{cycles}", Circuit(n, ops, 0), np.zeros(0),
                    [(1.0, ((0, "Z"),))])


def precision_28q(seed: int = 1) -> Workload:
    return grid_rqc(4, 7, 20, seed)


def precision_24q(seed: int = 1) -> Workload:
    return grid_rqc(4, 6, 20, seed)


def hea_ry_rz_cz(n: int, layers: int, seed: int, field: float = 1.0,
                 name: str = "hea_ryrz_cz") -> Workload:
    """Per layer Ry.Rz on every qubit then a CZ brick: even layers (0,1),(2,3)...,
    odd layers (1,2),(3,4)...  Parameter index = layer*2n + 2q + k, uniform [0, 2pi).
    Observable: sum Z_iZ_{i+1} + field * sum X_i."""
    rng = _rng(seed)
    ops: List[Op] = []
    p = 0
    for layer in range(layers):
        for q in range(n):
            ops.append(Op("RY", (q,), param=p))
            ops.append(Op("RZ", (q,), param=p + 1))
            p += 2
        for i in range(layer % 2, n - 1, 2):
            ops.append(Op("CZ", (i, i + 1)))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=p)
    fd = [int(round(x)) for x in np.linspace(0, p - 1, 10)]
    return Workload(name, Circuit(n, ops, p), theta, ising_chain(n, [field] * n),
                    extra={"fd_indices": fd})


def diff_20q(seed: int = 2) -> Workload:
    """20 qubits, 20 layers Ry.Rz + CZ brick, 800 angles, H = ZZ + 1.0 X (39 terms)."""
    return hea_ry_rz_cz(20, 20, seed, 1.0, name="vqe_20q_hea20")


def random_rotation_heisenberg(n: int, layers: int, seed: int, hz: float = 1.0, J: float = 1.0,
                               name: str = "heisenberg_rand") -> Workload:
    """Random variational circuit with the Heisenberg observable of the paper's operator
    example: per layer a rotation drawn from {Rx, Ry, Rz} on every qubit (each with its
    own angle), then CNOTs on alternating pairs (even layers (0,1),(2,3)..., odd layers
    (1,2),(3,4)...); H = hz sum Z_i + J sum (X_iX_i+1 + Y_iY_i+1 + Z_iZ_i+1).  The random
    circuit of the paper's gradient benchmark is not given in its text; this stands in."""
    rng = _rng(seed)
    ops: List[Op] = []
    p = 0
    for layer in range(layers):
        for q in range(n):
            ops.append(Op(ROTATIONS[int(rng.integers(0, 3))], (q,), param=p))
            p += 1
        for i in range(layer % 2, n - 1, 2):
            ops.append(Op("CNOT", (i, i + 1)))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=p)
    return Workload(name, Circuit(n, ops, p), theta, heisenberg_1d(n, hz, J))


def heisenberg_20q(seed: int = 6) -> Workload:
    """20 qubits, 10 layers of random rotations + CNOT brick, 200 angles, Heisenberg H
    (20 Z terms + 57 XX/YY/ZZ terms)."""
    return random_rotation_heisenberg(20, 10, seed, name="heisenberg_20q_rand10")


def fsim_grid_vqe(rows: int, cols: int, cycles: int, seed: int, pmask: int = 0b00011,
                  name: str = "fsim_vqe") -> Workload:
    """Grid circuit of the random-circuit construction (sqrt(X/Y/W) per qubit, never the
    same twice in a row, then FSIM on the cycle's coupler pattern) whose FSIM parameters
    selected by pmask are variational (initial values: theta ~ pi/2 + N(0, .05),
    phi ~ pi/6 + N(0, .05), the Delta's ~ N(0, .1)); H = sum Z_iZ_i+1 + 0.5 sum X_i over
    the qubit index chain."""
    rng = _rng(seed)
    n = rows * cols
    names = ("SX", "SY", "SW")
    last = [-1] * n
    ops: List[Op] = []
    theta: List[float] = []
    p = 0
    for t in range(cycles):
        for q in range(n):
            choices = [i for i in range(3) if i != last[q]]
            g = choices[int(rng.integers(0, len(choices)))]
            last[q] = g
            ops.append(Op(names[g], (q,)))
        for (a, b) in _couplers(rows, cols, t % 4):
            vals = [math.pi / 2 + rng.normal(0, 0.05), math.pi / 6 + rng.normal(0, 0.05),
                    rng.normal(0, 0.1), rng.normal(0, 0.1), rng.normal(0, 0.1)]
            if pmask:
                ops.append(Op("FSIM", (a, b), param=p, fixed=tuple(vals), pmask=pmask))
                for k in range(5):
                    if (pmask >> k) & 1:
                        theta.append(vals[k])
                        p += 1
            else:
                ops.append(Op("FSIM", (a, b), fixed=tuple(vals)))
    return Workload(name, Circuit(n, ops, p), np.array(theta), ising_chain(n, [0.5] * n))


def ry_rz_cnot_instance(n: int, depth: int, rng: np.random.Generator) -> Workload:
    """One batched-VQE instance: per layer Ry.Rz on every qubit then CNOT(i,i+1);
    H = sum Z_iZ_{i+1} + sum h_i X_i with h_i ~ U[-1, 1]."""
    ops: List[Op] = []
    p = 0
    for _ in range(depth):
        for q in range(n):
            ops.append(Op("RY", (q,), param=p))
            ops.append(Op("RZ", (q,), param=p + 1))
            p += 2
        for i in range(n - 1):
            ops.append(Op("CNOT", (i, i + 1)))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=p)
    h = rng.uniform(-1.0, 1.0, size=n)
    return Workload(f"vqe_{n}q_d{depth}", Circuit(n, ops, p), theta, ising_chain(n, h))


def batch_512(seed: int = 3, count: int = 512, n_lo: int = 12, n_hi: int = 20,
              d_lo: int = 4, d_hi: int = 16) -> List[Workload]:
    """Independent VQE instances with qubit counts U{n_lo..n_hi}, depths U{d_lo..d_hi}."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(rng.integers(d_lo, d_hi + 1))
        out.append(ry_rz_cnot_instance(n, d, rng))
    return out


def noisy_hea(n: int, layers: int, seed: int, p1: float = 1e-3, p2: float = 1e-2,
              gamma: float = 1e-3, name: str = "noisy_hea") -> Workload:
    """Rx.Rz.Rx + CNOT ladder on a density matrix, with single-qubit depolarising p1
    after every one-qubit gate, depolarising p2 on both qubits after every CNOT and
    amplitude damping gamma on every qubit at the end of every layer.
    Observable: sum Z_iZ_{i+1} + 0.5 sum X_i."""
    rng = _rng(seed)
    ops: List[Op] = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            for g in ("RX", "RZ", "RX"):
                ops.append(Op(g, (q,), param=p))
                ops.append(Op("DEPOL", (q,), fixed=(p1,)))
                p += 1
        for i in range(n - 1):
            ops.append(Op("CNOT", (i, i + 1)))
            ops.append(Op("DEPOL", (i,), fixed=(p2,)))
            ops.append(Op("DEPOL", (i + 1,), fixed=(p2,)))
        for q in range(n):
            ops.append(Op("AMPDAMP", (q,), fixed=(gamma,)))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=p)
    return Workload(name, Circuit(n, ops, p, density=True), theta,
                    ising_chain(n, [0.5] * n))


def noisy_13q(seed: int = 4) -> Workload:
    """13 qubits (26 vectorised), 8 layers, 312 angles."""
    return noisy_hea(13, 8, seed, name="noisy_13q_hea8")


def random_unitary(k: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-ish random 2^k x 2^k unitary (QR of a complex Gaussian matrix)."""
    d = 1 << k
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def random_kraus2(rng: np.random.Generator, count: int = 3, weight: Optional[float] = None) -> List[np.ndarray]:
    """A random two-qubit channel: count 4x4 Kraus operators cut from a random isometry
    (orthonormal columns of a 4 count x 4 matrix), so sum K^dag K = I.  With weight w the
    channel is mixed with the identity: sqrt(1-w) I followed by sqrt(w) K_s (weak noise,
    whose superoperator inverse stays well conditioned)."""
    A = rng.normal(size=(4 * count, 4)) + 1j * rng.normal(size=(4 * count, 4))
    Q, _ = np.linalg.qr(A)
    ks = [Q[4 * s:4 * s + 4, :] for s in range(count)]
    if weight is None:
        return ks
    return [math.sqrt(1.0 - weight) * np.eye(4, dtype=complex)] + [math.sqrt(weight) * k for k in ks]


def random_kraus(rng: np.random.Generator, count: int = 3) -> List[np.ndarray]:
    """A random single-qubit channel: Kraus operators from a random isometry."""
    d = 2 * count
    z = rng.normal(size=(d, 2)) + 1j * rng.normal(size=(d, 2))
    q, _ = np.linalg.qr(z)           # d x 2 isometry: sum K^dag K = I
    return [q[2 * s:2 * s + 2, :] for s in range(count)]


def random_circuit(n: int, n_ops: int, seed: int, density: bool = False,
                   with_channels: bool = False, param_share: bool = False) -> Workload:
    """Mixed circuit over every gate kind (and channels if asked), random qubits.

    Covers q = 0, q = n-1, adjacent and far pairs; about half the rotations are
    variational.  With param_share, some parameters drive several gates."""
    rng = _rng(seed)
    ops: List[Op] = []
    p = 0
    kinds1 = ONE_QUBIT_FIXED + ROTATIONS + ("DENSE1",)
    kinds2 = TWO_QUBIT_FIXED + ("FSIM", "CONTROL", "DENSE2")
    for i in range(n_ops):
        r = rng.random()
        if with_channels and r < 0.2:
            q = int(rng.integers(0, n))
            kind = ("DEPOL", "AMPDAMP", "PHASEDAMP", "KRAUS")[int(rng.integers(0, 4))]
            if kind == "KRAUS":
                ops.append(Op(kind, (q,), data=random_kraus(rng, int(rng.integers(1, 4)))))
            else:
                ops.append(Op(kind, (q,), fixed=(float(rng.uniform(0.01, 0.3)),)))
        elif n >= 2 and r < 0.55:
            a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
            kind = kinds2[int(rng.integers(0, len(kinds2)))]
            if kind == "FSIM":
                ops.append(Op(kind, (a, b), fixed=tuple(float(x) for x in
                                                        rng.uniform(-math.pi, math.pi, 5))))
            elif kind == "CONTROL":
                ops.append(Op(kind, (a, b), data=random_unitary(1, rng)))
            elif kind == "DENSE2":
                ops.append(Op(kind, (a, b), data=random_unitary(2, rng)))
            else:
                ops.append(Op(kind, (a, b)))
        else:
            q = int(rng.integers(0, n))
            kind = kinds1[int(rng.integers(0, len(kinds1)))]
            if kind in ROTATIONS:
                if rng.random() < 0.6:
                    if param_share and p > 0 and rng.random() < 0.3:
                        ops.append(Op(kind, (q,), param=int(rng.integers(0, p))))
                    else:
                        ops.append(Op(kind, (q,), param=p))
                        p += 1
                else:
                    ops.append(Op(kind, (q,), fixed=(float(rng.uniform(0, 2 * math.pi)),)))
            elif kind == "DENSE1":
                ops.append(Op(kind, (q,), data=random_unitary(1, rng)))
            else:
                ops.append(Op(kind, (q,)))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=p)
    terms: List[PauliTerm] = []
    for _ in range(max(3, n)):
        k = int(rng.integers(1, min(n, 3) + 1))
        qs = rng.choice(n, size=k, replace=False)
        terms.append((float(rng.normal()), tuple((int(q), "XYZ"[int(rng.integers(0, 3))])
                                                 for q in sorted(qs))))
    return Workload(f"random_{n}q_{n_ops}", Circuit(n, ops, p, density=density), theta, terms)


def random_state(n_qubits: int, seed: int) -> np.ndarray:
    """Normalised random complex128 vector of 2^n amplitudes."""
    rng = _rng(seed)
    v = rng.normal(size=1 << n_qubits) + 1j * rng.normal(size=1 << n_qubits)
    return v / np.linalg.norm(v)


def random_density(n_qubits: int, seed: int, rank: int = 3) -> np.ndarray:
    """Random density matrix as the vectorised 2^(2n) array, rho[a + 2^n b] = rho_ab."""
    rng = _rng(seed)
    d = 1 << n_qubits
    a = rng.normal(size=(d, rank)) + 1j * rng.normal(size=(d, rank))
    rho = a @ a.conj().T
    rho /= np.trace(rho).real
    return rho.reshape(-1, order="F").copy()   # column b holds rho[:, b] -> index a + d*b
