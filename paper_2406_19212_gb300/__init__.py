"""GB300-native variational quantum circuit simulator core (JuliVQC, arXiv 2406.19212).

Python face of libgbvqc.so.  The functions keep the names of the C entry points
(sv_alloc, circuit_create, apply_circuit, apply_channel, obs_create, expect, grad,
grad_batch) and only marshal arguments; every step runs in the library's CUDA kernels.
There is no CPU fallback: calls fail if the library is missing.

    import paper_2406_19212_gb300 as gb
    from paper_2406_19212_gb300 import inputs
    w = inputs.diff_20q()
    circ = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, w.circuit.n_qubits)
    energy, g = gb.grad(circ, w.theta, obs, dtype=gb.C64, mode=gb.FUSED)
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence, Tuple

import numpy as np

from . import _abi
from ._abi import C64, C128, FUSED, JIT, PLAIN, GbvqcError

__all__ = ["C64", "C128", "PLAIN", "FUSED", "JIT", "GbvqcError", "StateVector", "CircuitHandle",
           "Observable", "sv_alloc", "sv_wrap", "sv_set", "sv_get", "sv_reset",
           "circuit_create", "apply_circuit", "apply_channel", "obs_create", "expect", "grad",
           "grad_profile", "grad_batch", "batch_create", "BatchHandle", "expect_noalloc", "mem_info", "measure", "sample", "shard_plan", "ShardedState",
           "sharded_alloc",
           "gate_shape",
           "VQEEnergy",
           "load"]


def load():
    """Load the CUDA library (raises if it is not built)."""
    return _abi.lib()


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class StateVector:
    """A state owned (sv_alloc) or wrapped (sv_wrap) by the library."""

    def __init__(self, handle: int, n_qubits: int, dtype: int, density: bool, keep=None):
        self.handle = handle
        self.n_qubits = n_qubits
        self.dtype = dtype
        self.density = density
        self._keep = keep

    @property
    def n_amps(self) -> int:
        return 1 << (2 * self.n_qubits if self.density else self.n_qubits)

    def free(self):
        if self.handle:
            _abi.lib().sv_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sv_alloc(n_qubits: int, dtype: int = C64, is_density: bool = False, stream=None) -> StateVector:
    h = ctypes.c_void_p()
    _abi.check(_abi.lib().sv_alloc(n_qubits, dtype, int(is_density), _stream_ptr(stream),
                                   ctypes.byref(h)))
    return StateVector(h.value, n_qubits, dtype, bool(is_density))


def _check_cuda_amplitudes(tensor, n_amps: int, what: str):
    """A contiguous CUDA complex64/complex128 tensor of exactly n_amps elements (the kernels
    index 2^n amplitudes from its data pointer: a shorter or strided tensor would be read
    out of bounds)."""
    import torch
    if not (isinstance(tensor, torch.Tensor) and tensor.is_cuda):
        raise GbvqcError(_abi.ERR_ARG, f"{what} must be a CUDA tensor")
    if tensor.dtype not in (torch.complex64, torch.complex128):
        raise GbvqcError(_abi.ERR_ARG, f"{what} must be complex64 or complex128, not {tensor.dtype}")
    if not tensor.is_contiguous():
        raise GbvqcError(_abi.ERR_ARG, f"{what} must be contiguous")
    if tensor.numel() != n_amps:
        raise GbvqcError(_abi.ERR_ARG, f"{what} holds {tensor.numel()} amplitudes, expected {n_amps}")
    return C64 if tensor.dtype == torch.complex64 else C128


def sv_wrap(tensor, n_qubits: int, is_density: bool = False, stream=None) -> StateVector:
    """Wrap a contiguous CUDA torch.complex64/complex128 tensor of 2^n (density: 2^(2n))
    amplitudes (the library never frees it)."""
    if not 1 <= n_qubits <= 34:
        raise GbvqcError(_abi.ERR_ARG, f"qubit count {n_qubits}")
    dtype = _check_cuda_amplitudes(tensor, 1 << (2 * n_qubits if is_density else n_qubits), "state tensor")
    h = ctypes.c_void_p()
    _abi.check(_abi.lib().sv_wrap(tensor.data_ptr(), n_qubits, dtype, int(is_density),
                                  _stream_ptr(stream), ctypes.byref(h)))
    return StateVector(h.value, n_qubits, dtype, bool(is_density), keep=tensor)


def mem_info() -> Tuple[int, int]:
    """(bytes of device memory the library holds now, device allocations it has made)."""
    live, count = ctypes.c_int64(), ctypes.c_int64()
    _abi.check(_abi.lib().gbvqc_mem_info(ctypes.byref(live), ctypes.byref(count)))
    return live.value, count.value


def _np_dtype(dtype: int):
    return np.complex64 if dtype == C64 else np.complex128


def sv_set(sv: StateVector, amps) -> None:
    if _is_cuda_tensor(amps):
        _abi.check(_abi.lib().sv_set(sv.handle, amps.data_ptr(), amps.numel(), 0))
        return
    a = np.ascontiguousarray(np.asarray(amps), dtype=_np_dtype(sv.dtype))
    _abi.check(_abi.lib().sv_set(sv.handle, a.ctypes.data, a.size, 1))


def sv_get(sv: StateVector) -> np.ndarray:
    out = np.empty(sv.n_amps, dtype=_np_dtype(sv.dtype))
    _abi.check(_abi.lib().sv_get(sv.handle, out.ctypes.data, out.size, 1))
    return out


def sv_reset(sv: StateVector) -> None:
    _abi.check(_abi.lib().sv_reset(sv.handle))


class CircuitHandle:
    def __init__(self, handle: int, circuit):
        self.handle = handle
        self.n_qubits = circuit.n_qubits
        self.n_params = circuit.n_params
        self.density = circuit.density
        self.n_ops = len(circuit.ops)

    def set_tiling(self, tile_qubits: int = 0, low_qubits: int = 0) -> None:
        _abi.check(_abi.lib().circuit_set_tiling(self.handle, tile_qubits, low_qubits))

    def plan_info(self) -> Tuple[int, int, int]:
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _abi.check(_abi.lib().circuit_plan_info(self.handle, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c)))
        return a.value, b.value, c.value

    def autotune(self, theta, obs, dtype: int = C64, stream=None):
        """Pick the fastest tiling for `grad` on this circuit (cached on disk, see
        GBVQC_TUNE_CACHE); returns (tile_qubits, low_qubits, ms per evaluation)."""
        t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
        bt, bl, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _abi.check(_abi.lib().circuit_autotune(self.handle, t.ctypes.data if t.size else None, t.size,
                                               obs.handle, dtype, _stream_ptr(stream), ctypes.byref(bt),
                                               ctypes.byref(bl), ctypes.byref(ms)))
        return bt.value, bl.value, ms.value

    STAT_NAMES = ("tile_qubits", "passes", "fwd_subruns", "fwd_gates", "fwd_phase_blocks",
                  "rev_subruns", "grad_slots", "fwd_smem_max", "rev_smem_max", "phys_gates")

    def specialize(self, dtype: int = C64, for_grad: bool = True) -> dict:
        """Compile the plan's specialised tile passes (mode JIT) into the on-disk cache
        (host only); returns the number of kernels, how many were cached, and seconds."""
        nk, nc, sec = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _abi.check(_abi.lib().circuit_specialize(self.handle, dtype, int(for_grad), ctypes.byref(nk),
                                                 ctypes.byref(nc), ctypes.byref(sec)))
        return {"kernels": nk.value, "cached": nc.value, "seconds": sec.value}

    def plan_stats(self, dtype: int = C64, for_grad: bool = False) -> dict:
        """Host-only statistics of the fused schedule (no GPU needed)."""
        arr = (ctypes.c_int64 * 10)()
        _abi.check(_abi.lib().circuit_plan_stats(self.handle, dtype, int(for_grad), arr, 10))
        return dict(zip(self.STAT_NAMES, list(arr)))

    def free(self):
        if self.handle:
            _abi.lib().circuit_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def circuit_create(circuit) -> CircuitHandle:
    """Build a circuit from an `inputs.Circuit` description."""
    arr = _abi.ops_array(circuit.ops)
    h = ctypes.c_void_p()
    _abi.check(_abi.lib().circuit_create(arr, len(circuit.ops), circuit.n_qubits, circuit.n_params,
                                         int(circuit.density), ctypes.byref(h)))
    return CircuitHandle(h.value, circuit)


def _theta_args(theta, n: int):
    if _is_cuda_tensor(theta):
        import torch
        t = theta.detach().to(torch.float64).contiguous()
        return t, t.data_ptr(), _abi.PTR_DEVICE
    t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
    return t, (t.ctypes.data if t.size else None), _abi.PTR_HOST


def _len(t) -> int:
    return int(t.numel()) if hasattr(t, "numel") else int(t.size)


def apply_circuit(sv: StateVector, circ: CircuitHandle, theta=(), mode: int = FUSED) -> None:
    """In-place psi <- C(theta) psi on the state's stream (apply!)."""
    keep, ptr, loc = _theta_args(theta, circ.n_params)
    _abi.check(_abi.lib().apply_circuit(sv.handle, circ.handle, ptr, _len(keep), loc, mode))
    del keep


CHANNELS = {"DEPOL": 20, "AMPDAMP": 21, "PHASEDAMP": 22, "KRAUS": 23}


def apply_channel(sv: StateVector, name: str, qubit: int, strength: float = 0.0, kraus=None) -> None:
    buf = None
    n = 0
    if kraus is not None:
        mats = [np.asarray(k, dtype=np.complex128).reshape(4) for k in kraus]
        n = len(mats)
        buf = np.ascontiguousarray(np.concatenate(mats).view(np.float64))
    _abi.check(_abi.lib().apply_channel(
        sv.handle, CHANNELS[name], qubit, float(strength),
        buf.ctypes.data_as(_abi.dp) if buf is not None else None, n))


class Observable:
    def __init__(self, handle: int, n_qubits: int, terms):
        self.handle = handle
        self.n_qubits = n_qubits
        self.terms = list(terms)

    def free(self):
        if self.handle:
            _abi.lib().obs_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def obs_create(terms, n_qubits: int) -> Observable:
    arr = _abi.pauli_array(terms)
    h = ctypes.c_void_p()
    _abi.check(_abi.lib().obs_create(arr, len(terms), n_qubits, ctypes.byref(h)))
    return Observable(h.value, n_qubits, terms)


def expect(sv: StateVector, obs: Observable) -> float:
    out = ctypes.c_double()
    _abi.check(_abi.lib().expect(sv.handle, obs.handle, ctypes.byref(out)))
    return out.value


SHAPE_NAMES = {0: "DENSE1", 1: "DIAG1", 2: "ANTI1", 3: "REAL1", 4: "DENSE2", 5: "DIAG2", 6: "PERM2",
               7: "CTRL2", 8: "BLOCK2", 9: "IMAG1", 11: "PAR2", 12: "RPAR2", 13: "CX", 14: "CZ"}


def gate_shape(matrix) -> str:
    """Name of the kernel structure the library picks for a 2x2 or 4x4 matrix (host only)."""
    m = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128))
    if m.ndim != 2 or m.shape[0] != m.shape[1]:
        raise ValueError("a square matrix is required")
    flat = np.ascontiguousarray(m.reshape(-1).view(np.float64))
    out = ctypes.c_int()
    _abi.check(_abi.lib().gate_shape(flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m.shape[0],
                                     ctypes.byref(out)))
    return SHAPE_NAMES[out.value]


def measure(sv: StateVector, qubit: int, u: float) -> Tuple[int, float]:
    """measure!(state, qubit) of Sec. II.D: collapses the state in place and returns
    (outcome, probability); u in [0, 1) is the caller's uniform draw (outcome 0 if
    u < P(0))."""
    k = ctypes.c_int()
    p = ctypes.c_double()
    _abi.check(_abi.lib().measure(sv.handle, int(qubit), float(u), ctypes.byref(k), ctypes.byref(p)))
    return k.value, p.value


def sample(sv: StateVector, u) -> np.ndarray:
    """Basis indices of len(u) shots (every qubit measured on fresh copies of the state,
    which is left unchanged); u are the caller's uniform draws in [0, 1)."""
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
    out = np.zeros(max(1, uu.size), dtype=np.int64)
    _abi.check(_abi.lib().sample(sv.handle, uu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), uu.size,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out[:uu.size]


def expect_noalloc(psi, n_qubits: int, terms, out, stream=None) -> None:
    """<psi|H|psi> of a CUDA complex64/complex128 tensor without any device allocation.

    For callers that cannot allocate device memory themselves or through the library
    (a framework that owns the whole device memory budget through its own pool, a loop
    that cannot take the device-wide synchronisation of cudaMalloc / cudaFree): `psi` is
    a contiguous CUDA tensor of 2^n_qubits amplitudes, `out` a caller-provided CUDA
    float64 tensor (one element is written) on the same device, written asynchronously
    on `stream` (default: torch's current stream of psi's device).  At most 64 terms.
    Calls share one fixed scratch array in the library, so calls that overlap on the GPU
    race; keep them on one stream."""
    import torch
    if not 1 <= n_qubits <= 34:
        raise GbvqcError(_abi.ERR_ARG, f"qubit count {n_qubits}")
    dtype = _check_cuda_amplitudes(psi, 1 << n_qubits, "psi")
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
        raise GbvqcError(_abi.ERR_ARG, "out must be a CUDA float64 tensor with at least one element")
    if out.device != psi.device:
        raise GbvqcError(_abi.ERR_ARG, f"out is on {out.device}, psi on {psi.device}")
    arr = _abi.pauli_array(terms)
    with torch.cuda.device(psi.device):
        s = _stream_ptr(stream if stream is not None else torch.cuda.current_stream(psi.device))
        _abi.check(_abi.lib().expect_noalloc(psi.data_ptr(), n_qubits, dtype, arr, len(terms), s,
                                             out.data_ptr()))


def grad(circ: CircuitHandle, theta, obs: Observable, dtype: int = C64, mode: int = FUSED,
         stream=None, out=None):
    """Energy and exact gradient by the reverse sweep (Algorithm 2).

    Host theta (numpy / sequence): returns (float, numpy array) and synchronises; `out`
    = (float64 array of shape (1,), float64 array of shape (n_params,)) receives the
    results in caller memory (e.g. numpy views of pinned host buffers) if given.
    CUDA theta (torch float64): results stay on the device, written into `out`
    = (energy tensor of shape (1,), grad tensor of shape (n_params,)) if given, or into
    new tensors; the call is asynchronous on `stream` (default: torch's current stream).
    """
    if _is_cuda_tensor(theta):
        import torch
        keep, ptr, loc = _theta_args(theta, circ.n_params)
        if out is None:
            e = torch.empty(1, dtype=torch.float64, device=theta.device)
            g = torch.empty(circ.n_params, dtype=torch.float64, device=theta.device)
        else:
            e, g = out
        s = _stream_ptr(stream if stream is not None else torch.cuda.current_stream(theta.device))
        _abi.check(_abi.lib().grad(circ.handle, ptr, _len(keep), obs.handle, dtype, mode, loc,
                                   s, e.data_ptr(), g.data_ptr() if circ.n_params else None))
        del keep
        return e, g
    keep, ptr, loc = _theta_args(theta, circ.n_params)
    if out is not None:
        e_arr, g = out
        for a, size in ((e_arr, 1), (g, circ.n_params)):
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size < size:
                raise ValueError("out arrays must be contiguous float64 of sizes (1, n_params)")
        _abi.check(_abi.lib().grad(circ.handle, ptr, _len(keep), obs.handle, dtype, mode, loc,
                                   _stream_ptr(stream), e_arr.ctypes.data,
                                   g.ctypes.data if circ.n_params else None))
        del keep
        return float(e_arr[0]), g[:circ.n_params]
    e = ctypes.c_double()
    g = np.zeros(max(1, circ.n_params))
    _abi.check(_abi.lib().grad(circ.handle, ptr, _len(keep), obs.handle, dtype, mode, loc,
                               _stream_ptr(stream), ctypes.byref(e), g.ctypes.data))
    del keep
    return e.value, g[:circ.n_params]


def grad_profile(circ: CircuitHandle, theta, obs: Observable, dtype: int = C64,
                 mode: int = FUSED, stream=None):
    """Per-kernel CUDA-event timing of one gradient evaluation:
    {name: (launches, ms, alg_flops, alg_bytes)}."""
    keep, ptr, loc = _theta_args(theta, circ.n_params)
    stats = (_abi.KernelStat * 64)()
    n = ctypes.c_int()
    _abi.check(_abi.lib().grad_profile(circ.handle, ptr, _len(keep), obs.handle, dtype, mode,
                                       _stream_ptr(stream), stats, 64, ctypes.byref(n)))
    del keep
    return {stats[i].name.decode(): (stats[i].launches, stats[i].ms, stats[i].alg_flops,
                                     stats[i].alg_bytes) for i in range(n.value)}


def shard_plan(circ: CircuitHandle, n_global: int):
    """Exchange schedule for n_global global qubits: [("ops", begin, end) | ("swap", j, l)]."""
    cap = 2 * circ.n_ops + 16
    buf = (ctypes.c_int32 * (3 * cap))()
    n, sw = ctypes.c_int(), ctypes.c_int()
    _abi.check(_abi.lib().shard_plan(circ.handle, n_global, buf, cap, ctypes.byref(n), ctypes.byref(sw)))
    return [("ops" if buf[3 * i] == 0 else "swap", buf[3 * i + 1], buf[3 * i + 2]) for i in range(n.value)]


class ShardedState:
    """A pure state split into 2^n_global shards by its global qubits (sharded_alloc)."""

    def __init__(self, n_qubits: int, n_global: int, dtype: int = C64):
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().sharded_alloc(n_qubits, n_global, dtype, ctypes.byref(h)))
        self.handle, self.n_qubits, self.n_global, self.dtype = h.value, n_qubits, n_global, dtype

    def set(self, amps) -> None:
        a = np.ascontiguousarray(np.asarray(amps), dtype=_np_dtype(self.dtype))
        assert a.size == 1 << self.n_qubits
        _abi.check(_abi.lib().sharded_set(self.handle, a.ctypes.data))

    def get(self) -> np.ndarray:
        out = np.empty(1 << self.n_qubits, dtype=_np_dtype(self.dtype))
        _abi.check(_abi.lib().sharded_get(self.handle, out.ctypes.data))
        return out

    def apply(self, circ: CircuitHandle, theta=()) -> None:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
        _abi.check(_abi.lib().sharded_apply(self.handle, circ.handle,
                                            th.ctypes.data_as(_abi.dp) if th.size else None, th.size))

    def info(self):
        pos = (ctypes.c_int32 * self.n_qubits)()
        ex, by = ctypes.c_int64(), ctypes.c_int64()
        _abi.check(_abi.lib().sharded_info(self.handle, pos, ctypes.byref(ex), ctypes.byref(by)))
        return list(pos), ex.value, by.value

    def free(self):
        if self.handle:
            _abi.lib().sharded_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sharded_alloc(n_qubits: int, n_global: int, dtype: int = C64) -> ShardedState:
    return ShardedState(n_qubits, n_global, dtype)


class BatchHandle:
    """Many independent circuits evaluated together (batch_create / batch_grad)."""

    def __init__(self, circs: Sequence[CircuitHandle], obss: Sequence[Observable], dtype: int = C64):
        n = len(circs)
        ch = (ctypes.c_void_p * n)(*[c.handle for c in circs])
        oh = (ctypes.c_void_p * n)(*[o.handle for o in obss])
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().batch_create(ch, oh, n, dtype, ctypes.byref(h)))
        self.handle = h.value
        self._keep = (list(circs), list(obss))   # the batch points at these handles
        self.n_params = [c.n_params for c in circs]
        self.total = sum(self.n_params)

    def grad(self, thetas, stream=None, out=None):
        """Energies and gradients.  Host input (list of arrays or one concatenated array)
        returns (numpy energies, list of numpy gradients); a CUDA float64 tensor of all
        parameters returns device tensors (energies, concatenated gradients)."""
        n = len(self.n_params)
        if _is_cuda_tensor(thetas):
            import torch
            t = thetas.detach().to(torch.float64).contiguous()
            if out is None:
                e = torch.empty(n, dtype=torch.float64, device=t.device)
                g = torch.empty(max(1, self.total), dtype=torch.float64, device=t.device)
            else:
                e, g = out
            s = _stream_ptr(stream if stream is not None else torch.cuda.current_stream(t.device))
            _abi.check(_abi.lib().batch_grad(self.handle, t.data_ptr(), t.numel(), _abi.PTR_DEVICE, s,
                                             e.data_ptr(), g.data_ptr()))
            return e, g
        if isinstance(thetas, np.ndarray) and thetas.ndim == 1:
            th = np.ascontiguousarray(thetas, dtype=np.float64)
        else:
            th = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).reshape(-1)
                                                      for t in thetas]) if n else np.zeros(0))
        e = np.zeros(n)
        g = np.zeros(max(1, self.total))
        _abi.check(_abi.lib().batch_grad(self.handle, th.ctypes.data if th.size else None, th.size,
                                         _abi.PTR_HOST, _stream_ptr(stream), e.ctypes.data, g.ctypes.data))
        out_g, off = [], 0
        for k in self.n_params:
            out_g.append(g[off:off + k].copy())
            off += k
        return e, out_g

    def autotune(self, thetas, stream=None):
        """Batch autotuner (batch_autotune): returns (tile size of every member, ms per
        batch_grad of the chosen assignment)."""
        if isinstance(thetas, np.ndarray) and thetas.ndim == 1:
            th = np.ascontiguousarray(thetas, dtype=np.float64)
        else:
            th = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).reshape(-1)
                                                      for t in thetas]))
        n = len(self.n_params)
        tiles = (ctypes.c_int * max(1, n))()
        ms = ctypes.c_double()
        _abi.check(_abi.lib().batch_autotune(self.handle, th.ctypes.data_as(_abi.dp) if th.size else None,
                                             th.size, _stream_ptr(stream), tiles, ctypes.byref(ms)))
        return [tiles[i] for i in range(n)], ms.value

    def free(self):
        if self.handle:
            _abi.lib().batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def batch_create(circs, obss, dtype: int = C64) -> BatchHandle:
    return BatchHandle(circs, obss, dtype)


def grad_batch(circs: Sequence[CircuitHandle], obss: Sequence[Observable], thetas, stream=None):
    """One-shot batched energies and gradients (complex64); see BatchHandle for reuse."""
    n = len(circs)
    ch = (ctypes.c_void_p * n)(*[c.handle for c in circs])
    oh = (ctypes.c_void_p * n)(*[o.handle for o in obss])
    th = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).reshape(-1)
                                              for t in thetas]) if n else np.zeros(1))
    total = sum(c.n_params for c in circs)
    e = np.zeros(max(1, n))
    g = np.zeros(max(1, total))
    _abi.check(_abi.lib().grad_batch(ch, oh, n, th.ctypes.data_as(_abi.dp), _stream_ptr(stream),
                                     e.ctypes.data_as(_abi.dp), g.ctypes.data_as(_abi.dp)))
    out, off = [], 0
    for c in circs:
        out.append(g[off:off + c.n_params].copy())
        off += c.n_params
    return e[:n], out


def _autograd_class():
    import torch

    class VQEEnergy(torch.autograd.Function):
        """L(theta) = <H> after the circuit; backward scales the adjoint gradient.

        forward(theta, circ, obs, dtype, mode) runs `grad` once (energy and gradient),
        saves the gradient and returns the energy as a 0-d tensor on theta's device."""

        @staticmethod
        def forward(ctx, theta, circ, obs, dtype=C64, mode=FUSED):
            if theta.is_cuda:
                e, g = grad(circ, theta.detach().to(torch.float64), obs, dtype, mode)
                ctx.save_for_backward(g)
                return e.reshape(()).to(theta.dtype)
            e, g = grad(circ, theta.detach().cpu().numpy(), obs, dtype, mode)
            ctx.save_for_backward(torch.from_numpy(g))
            return torch.tensor(e, dtype=theta.dtype)

        @staticmethod
        def backward(ctx, dE):
            (g,) = ctx.saved_tensors
            return (dE.to(g.dtype) * g).to(dE.dtype), None, None, None, None

    return VQEEnergy


class _LazyAutograd:
    _cls = None

    def __getattr__(self, name):
        if _LazyAutograd._cls is None:
            _LazyAutograd._cls = _autograd_class()
        return getattr(_LazyAutograd._cls, name)


VQEEnergy = _LazyAutograd()
