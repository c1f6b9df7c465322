"""ctypes binding of libgbvqc.so (include/gbvqc.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python circuit
descriptions to the C structs and raises GbvqcError on a non-zero status.  Importing
it does not load the library; the first call does, and fails loudly if the library has
not been built or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbvqc.so")

C64, C128 = 0, 1
PLAIN, FUSED, JIT = 0, 1, 2
PTR_HOST, PTR_DEVICE = 0, 1
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT = 1, 2, 3, 4

KIND = {name: i for i, name in enumerate(
    ["X", "Y", "Z", "H", "S", "T", "SX", "SY", "SW", "RX", "RY", "RZ", "CNOT", "CZ", "SWAP",
     "ISWAP", "FSIM", "CONTROL", "DENSE1", "DENSE2", "DEPOL", "AMPDAMP", "PHASEDAMP", "KRAUS",
     "DEPOL2", "KRAUS2"])}

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT",
          5: "ERR_NOT_DENSITY", 6: "ERR_UNSUPPORTED"}


class GbvqcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("qubits", ctypes.c_int32 * 2),
                ("param_index", ctypes.c_int32), ("n_kraus", ctypes.c_int32),
                ("param_mask", ctypes.c_int32), ("params", ctypes.c_double * 5),
                ("data", ctypes.c_double * 32), ("kraus", ctypes.c_void_p)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("ms", ctypes.c_double),
                ("alg_flops", ctypes.c_double), ("alg_bytes", ctypes.c_double)]


class Pauli(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("x_mask", ctypes.c_uint64),
                ("z_mask", ctypes.c_uint64)]


_lib = None
vp = ctypes.c_void_p
dp = ctypes.POINTER(ctypes.c_double)


def lib() -> ctypes.CDLL:
    """Load libgbvqc.so; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgbvqc.so not built ({LIB_PATH}); run "
                           "`python -m paper_2406_19212_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    L.gbvqc_last_error.restype = ctypes.c_char_p
    L.gbvqc_version.restype = ctypes.c_int
    sig = {
        "sv_alloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)],
        "sv_wrap": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)],
        "sv_free": [vp],
        "sv_reset": [vp],
        "sv_set": [vp, vp, ctypes.c_size_t, ctypes.c_int],
        "sv_get": [vp, vp, ctypes.c_size_t, ctypes.c_int],
        "sv_info": [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp)],
        "circuit_create": [ctypes.POINTER(Op), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, ctypes.POINTER(vp)],
        "circuit_free": [vp],
        "circuit_set_tiling": [vp, ctypes.c_int, ctypes.c_int],
        "circuit_plan_info": [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_int)],
        "circuit_autotune": [vp, vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
        "circuit_plan_stats": [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int],
        "circuit_specialize": [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_double)],
        "gate_shape": [dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "apply_circuit": [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "apply_channel": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, ctypes.c_int],
        "obs_create": [ctypes.POINTER(Pauli), ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
        "obs_free": [vp],
        "expect": [vp, vp, dp],
        "measure": [vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int), dp],
        "sample": [vp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
        "grad": [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp],
        "grad_profile": [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp,
                         ctypes.POINTER(KernelStat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "expect_noalloc": [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Pauli), ctypes.c_int, vp, vp],
        "grad_batch": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, dp, vp, dp, dp],
        "batch_create": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
        "batch_free": [vp],
        "batch_grad": [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp],
        "batch_autotune": [vp, dp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
        "gbvqc_mem_info": [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
        "shard_plan": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_int)],
        "sharded_alloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
        "sharded_free": [vp],
        "sharded_set": [vp, vp],
        "sharded_get": [vp, vp],
        "sharded_apply": [vp, vp, dp, ctypes.c_int],
        "sharded_info": [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_int64)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    _lib = L
    return L


def check(status: int) -> None:
    if status != 0:
        raise GbvqcError(status, lib().gbvqc_last_error().decode())


def exported_symbols() -> List[str]:
    return ["gbvqc_last_error", "gbvqc_version", "sv_alloc", "sv_wrap", "sv_free", "sv_reset",
            "sv_set", "sv_get", "sv_info", "circuit_create", "circuit_free", "circuit_set_tiling",
            "circuit_plan_info", "circuit_plan_stats", "circuit_autotune", "apply_circuit", "apply_channel", "obs_create", "obs_free",
            "expect", "grad", "grad_profile", "grad_batch", "batch_create", "batch_free",
            "batch_grad", "expect_noalloc", "measure", "sample", "gate_shape", "gbvqc_mem_info", "circuit_specialize", "batch_autotune", "shard_plan", "sharded_alloc",
            "sharded_free", "sharded_set", "sharded_get", "sharded_apply", "sharded_info"]


# ------------------------------------------------------------------ marshalling

def ops_array(ops) -> ctypes.Array:
    """inputs.Op list -> gbvqc_op array."""
    arr = (Op * max(1, len(ops)))()
    arr._keep = []  # KRAUS2 operator buffers referenced by pointer (copied by circuit_create)
    for i, op in enumerate(ops):
        o = arr[i]
        o.kind = KIND[op.name]
        for t, q in enumerate(op.qubits):
            o.qubits[t] = int(q)
        o.param_index = int(op.param)
        o.param_mask = int(getattr(op, "pmask", 0))
        for t, v in enumerate(op.fixed):
            o.params[t] = float(v)
        if op.name == "KRAUS2":
            mats = [np.asarray(k, dtype=np.complex128).reshape(4, 4) for k in op.data]
            o.n_kraus = len(mats)
            buf = np.ascontiguousarray(np.concatenate([m.reshape(-1) for m in mats])).view(np.float64)
            arr._keep.append(buf)
            o.kraus = buf.ctypes.data
        elif op.data is not None:
            if op.name == "KRAUS":
                mats = [np.asarray(k, dtype=np.complex128) for k in op.data]
                o.n_kraus = len(mats)
                flat = (np.concatenate([m.reshape(-1) for m in mats]) if mats
                        else np.zeros(0, dtype=np.complex128))
            else:
                flat = np.asarray(op.data, dtype=np.complex128).reshape(-1)
            for t, v in enumerate(flat):
                o.data[2 * t] = float(v.real)
                o.data[2 * t + 1] = float(v.imag)
    return arr


def pauli_array(terms) -> ctypes.Array:
    """[(coeff, ((q, 'X'|'Y'|'Z'), ...)), ...] -> gbvqc_pauli array (Y sets both masks)."""
    arr = (Pauli * max(1, len(terms)))()
    for i, (coeff, factors) in enumerate(terms):
        x = z = 0
        for q, p in factors:
            if p in "XY":
                x |= 1 << q
            if p in "ZY":
                z |= 1 << q
        arr[i].coeff = float(coeff)
        arr[i].x_mask = x
        arr[i].z_mask = z
    return arr
