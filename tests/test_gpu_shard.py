"""Sharded states on one GPU: the library's exchange schedule, per-shard tile passes and
shard-pair swap kernel against the FP64 oracle.  Shards are separate device buffers (one
per would-be device); the result is read back through the qubit positions the schedule
leaves, so a second apply starts from a permuted layout."""
import numpy as np
import pytest

import paper_2406_19212_gb300 as gb
from oracle import oracle as O
from paper_2406_19212_gb300 import inputs as I
from tests.test_gpu_parity import DTYPES, check_amps

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,g,seed", [(8, 1, 0), (10, 2, 1), (14, 3, 2)])
def test_sharded_random_circuit_matches_oracle(n, g, seed, dtype):
    w = I.random_circuit(n, 160, seed)
    c = gb.circuit_create(w.circuit)
    st = gb.sharded_alloc(n, g, dtype)
    st.apply(c, w.theta)
    ref = O.apply_circuit(w.circuit, w.theta)
    check_amps(st.get().astype(np.complex128), ref, dtype)
    # again, from the permuted layout the first apply left
    st.apply(c, w.theta)
    check_amps(st.get().astype(np.complex128), O.apply_circuit(w.circuit, w.theta, ref), dtype)
    pos, exchanges, nbytes = st.info()
    assert sorted(pos) == list(range(n))
    swaps = sum(1 for s in gb.shard_plan(c, g) if s[0] == "swap")
    assert exchanges >= swaps * (1 << (g - 1))
    st.free()


def test_sharded_set_get_round_trip():
    n, g = 9, 2
    psi = I.random_state(n, 4)
    st = gb.sharded_alloc(n, g, gb.C128)
    st.set(psi)
    assert np.abs(st.get() - psi).max() == 0
    st.free()


def test_sharded_vqe20_and_rqc24():
    """The 20-qubit VQE circuit (CZ brick: diagonal gates on global qubits need no
    exchange) with 2 global qubits in complex128, and the 24-qubit grid random circuit with
    3 global qubits in complex64, against the oracle."""
    w = I.diff_20q()
    c = gb.circuit_create(w.circuit)
    st = gb.sharded_alloc(20, 2, gb.C128)
    st.apply(c, w.theta)
    check_amps(st.get(), O.apply_circuit(w.circuit, w.theta), gb.C128)
    st.free()
    w = I.precision_24q()
    c = gb.circuit_create(w.circuit)
    st = gb.sharded_alloc(24, 3, gb.C64)
    st.apply(c, w.theta)
    check_amps(st.get().astype(np.complex128), O.apply_circuit(w.circuit, w.theta), gb.C64)
    st.free()
