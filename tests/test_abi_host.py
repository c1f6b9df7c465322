"""Host-side checks of the C ABI that need no GPU: the library builds and loads, it
exports every entry point include/gbvqc.h declares, and argument validation returns
the documented status codes before any CUDA call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2406_19212_gb300 as gb
from paper_2406_19212_gb300 import _abi
from paper_2406_19212_gb300 import build as gbuild
from paper_2406_19212_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gb.load()


def declared_functions():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            if m.group(1) not in ("if", "for", "while", "sizeof"):
                names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    declared = declared_functions()
    assert {"sv_alloc", "apply_circuit", "apply_channel", "expect", "grad"} <= declared
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(_abi.exported_symbols()) <= declared


def test_version(lib):
    assert lib.gbvqc_version() >= 100


def expect_status(status, fn, *args):
    with pytest.raises(gb.GbvqcError) as ei:
        fn(*args)
    assert ei.value.status == status, str(ei.value)


def test_circuit_validation(lib):
    ARG, NOT_DENSITY = 1, 5
    expect_status(ARG, gb.circuit_create, I.Circuit(2, [I.Op("RX", (2,), param=0)], 1))
    expect_status(ARG, gb.circuit_create, I.Circuit(2, [I.Op("RX", (0,), param=3)], 1))
    expect_status(ARG, gb.circuit_create, I.Circuit(2, [I.Op("CNOT", (1, 1))], 0))
    expect_status(ARG, gb.circuit_create, I.Circuit(2, [I.Op("CZ", (0, 1), param=0)], 1))
    expect_status(ARG, gb.circuit_create, I.Circuit(0, [], 0))
    expect_status(ARG, gb.circuit_create, I.Circuit(18, [], 0, True))
    expect_status(NOT_DENSITY, gb.circuit_create, I.Circuit(2, [I.Op("DEPOL", (0,), fixed=(0.1,))], 0))
    expect_status(ARG, gb.circuit_create, I.Circuit(2, [I.Op("DEPOL", (0,), fixed=(1.5,))], 0, True))
    expect_status(ARG, gb.circuit_create, I.Circuit(2, [I.Op("KRAUS", (0,), data=[])], 0, True))
    # a channel whose superoperator has no inverse cannot be uncomputed (Algorithm 2)
    expect_status(ARG, gb.circuit_create, I.Circuit(2, [I.Op("AMPDAMP", (0,), fixed=(1.0,))], 0, True))


def test_observable_and_state_validation(lib):
    ARG = 1
    expect_status(ARG, gb.obs_create, [(1.0, ((3, "X"),))], 3)
    expect_status(ARG, gb.obs_create, [(1.0, ())], 0)
    expect_status(ARG, gb.sv_alloc, 4, 5)
    expect_status(ARG, gb.sv_alloc, 0, gb.C64)
    expect_status(ARG, gb.sv_alloc, 18, gb.C64, True)


def test_null_handles(lib):
    L = lib
    out = ctypes.c_double()
    assert L.expect(None, None, ctypes.byref(out)) == 1
    assert L.apply_circuit(None, None, None, 0, 0, 0) == 1
    assert L.grad(None, None, 0, None, 0, 0, 0, None, None, None) == 1
    assert b"NULL" in L.gbvqc_last_error()
    assert L.sv_free(None) == 0 and L.circuit_free(None) == 0 and L.obs_free(None) == 0


def test_pauli_marshalling():
    arr = _abi.pauli_array([(0.5, ((0, "X"), (2, "Y"), (3, "Z")))])
    assert arr[0].x_mask == 0b0101 and arr[0].z_mask == 0b1100 and arr[0].coeff == 0.5


def test_op_marshalling():
    u = I.random_unitary(2, np.random.default_rng(0))
    arr = _abi.ops_array([I.Op("DENSE2", (3, 1), data=u), I.Op("FSIM", (0, 2), fixed=(0.1, 0.2))])
    assert arr[0].kind == _abi.KIND["DENSE2"] and list(arr[0].qubits) == [3, 1]
    assert arr[0].data[2 * 6] == u.reshape(-1)[6].real and arr[0].data[2 * 6 + 1] == u.reshape(-1)[6].imag
    assert arr[1].params[0] == 0.1 and arr[1].params[1] == 0.2 and arr[1].param_index == -1


@pytest.mark.parametrize("dtype", [gb.C64, gb.C128])
def test_planner_invariants_host(lib, dtype):
    # host-only schedule statistics: every variational gate gets a gradient slot (two
    # per rotation on a density matrix: ket and bra), tiles respect the thread cap, and
    # every pass fits the shared-memory opt-in
    cases = [(I.diff_20q(), 800), (I.plain_10q(), 120), (I.noisy_hea(6, 2, 1), 2 * 36),
             (I.precision_24q(), 0), (I.random_circuit(14, 300, 3, param_share=True), None)]
    for w, slots in cases:
        c = gb.circuit_create(w.circuit)
        st = c.plan_stats(dtype, for_grad=True)
        n_phys = (2 if w.circuit.density else 1) * w.circuit.n_qubits
        nr_min = 4 if dtype == gb.C64 else 3
        assert st["tile_qubits"] <= min(n_phys, nr_min + 8)
        assert st["passes"] >= 1 and st["fwd_subruns"] >= st["passes"]
        assert st["fwd_smem_max"] <= 200 * 1024 and st["rev_smem_max"] <= 200 * 1024
        n_var = sum(1 for o in w.circuit.ops if o.param >= 0)
        assert st["grad_slots"] == (2 * n_var if w.circuit.density else n_var)
        if slots is not None:
            assert st["grad_slots"] == slots
        assert st["fwd_gates"] <= st["phys_gates"]


def test_passes_leave_two_ctas_per_sm_host(lib):
    # single-circuit plans take passes as large as 110 KiB of reverse-pass shared memory
    # allows (two CTAs per SM); the 20-qubit step then needs 5 passes at tile 12
    cases = [I.diff_20q(), I.noisy_hea(6, 2, 1), I.precision_24q(), I.heisenberg_20q(),
             I.random_circuit(14, 300, 3, param_share=True)]
    for w in cases:
        c = gb.circuit_create(w.circuit)
        for dtype in (gb.C64, gb.C128):
            for t, lo in ((10, 2), (11, 3), (12, 4)):
                try:
                    c.set_tiling(t, lo)
                    st = c.plan_stats(dtype, for_grad=True)
                except gb.GbvqcError:
                    continue  # tile above the precision's thread cap
                assert st["rev_smem_max"] <= 110 * 1024
    c = gb.circuit_create(I.diff_20q().circuit)
    c.set_tiling(12, 4)
    assert c.plan_stats(gb.C64, for_grad=True)["passes"] == 5


def test_tiling_options_host(lib):
    w = I.random_circuit(14, 200, 5)
    c = gb.circuit_create(w.circuit)
    last = None
    for t in (6, 8, 10, 12):
        c.set_tiling(t, 2)
        st = c.plan_stats(gb.C64)
        assert st["tile_qubits"] == t
        if last is not None:
            assert st["passes"] <= last   # larger tiles never need more passes here
        last = st["passes"]
    with pytest.raises(gb.GbvqcError):
        c.set_tiling(20, 2)


def test_batch_validation_host(lib):
    pure = gb.circuit_create(I.plain_10q().circuit)
    dens = gb.circuit_create(I.noisy_hea(4, 1, 0).circuit)
    tiny = gb.circuit_create(I.hea_ry_rz_cz(3, 1, 0).circuit)
    o10, o4, o3 = gb.obs_create([(1.0, ((0, "Z"),))], 10), gb.obs_create([(1.0, ((0, "Z"),))], 4), \
        gb.obs_create([(1.0, ((0, "Z"),))], 3)
    expect_status(1, gb.batch_create, [dens], [o4])        # density circuits are not batched
    expect_status(1, gb.batch_create, [pure], [o4])        # observable / circuit qubit mismatch
    expect_status(6, gb.batch_create, [tiny], [o3])        # fewer than 6 qubits: no tiles
    expect_status(1, gb.batch_create, [], [])


def test_gradient_layout_cuts_passes_of_a_ladder(lib):
    """A CNOT ladder across more qubits than a tile: the gradient plan moves the physical
    low qubits into the overlap of neighbouring tiles and needs fewer passes than the
    identity layout of apply_circuit (host planner only)."""
    rng = np.random.default_rng(0)
    w = I.ry_rz_cnot_instance(20, 16, rng)
    c = gb.circuit_create(w.circuit)
    c.set_tiling(12, 4)
    grad_passes = c.plan_stats(gb.C64, for_grad=True)["passes"]
    apply_passes = c.plan_stats(gb.C64, for_grad=False)["passes"]
    assert grad_passes < apply_passes
    assert grad_passes <= 20


def test_variational_fsim_validation(lib):
    ok = I.Circuit(2, [I.Op("FSIM", (0, 1), param=0, fixed=(1.0, 0.5), pmask=0b11)], 2)
    gb.circuit_create(ok)
    bad_mask = I.Circuit(2, [I.Op("FSIM", (0, 1), param=0, fixed=(1.0, 0.5), pmask=0)], 2)
    too_few = I.Circuit(2, [I.Op("FSIM", (0, 1), param=0, fixed=(1.0, 0.5), pmask=0b111)], 2)
    density = I.Circuit(2, [I.Op("FSIM", (0, 1), param=0, fixed=(1.0, 0.5), pmask=0b11)], 2, density=True)
    gb.circuit_create(density)  # density circuits take variational FSIM too
    for circ, status in ((bad_mask, 1), (too_few, 1)):
        with pytest.raises(gb.GbvqcError) as ex:
            gb.circuit_create(circ)
        assert ex.value.status == status
    # the gradient plan of a variational FSIM circuit carries one slot per parameter
    w = I.fsim_grid_vqe(3, 3, 3, 5, pmask=0b11111)
    c = gb.circuit_create(w.circuit)
    st = c.plan_stats(gb.C64, for_grad=True)
    assert st["grad_slots"] == w.circuit.n_params


def test_two_qubit_channel_validation_and_barrier_passes(lib):
    pure = I.Circuit(3, [I.Op("DEPOL2", (0, 1), fixed=(0.1,))], 0)
    with pytest.raises(gb.GbvqcError) as ex:
        gb.circuit_create(pure)
    assert ex.value.status == 5  # ERR_NOT_DENSITY
    bad_p = I.Circuit(3, [I.Op("DEPOL2", (0, 1), fixed=(1.5,))], 0, density=True)
    with pytest.raises(gb.GbvqcError):
        gb.circuit_create(bad_p)
    singular = I.Circuit(3, [I.Op("KRAUS2", (0, 2), data=[np.zeros((4, 4))])], 0, density=True)
    with pytest.raises(gb.GbvqcError):
        gb.circuit_create(singular)
    rng = np.random.default_rng(2)
    ops = [I.Op("RY", (0,), param=0), I.Op("KRAUS2", (0, 2), data=I.random_kraus2(rng, 3)),
           I.Op("RX", (1,), param=1), I.Op("DEPOL2", (1, 2), fixed=(0.05,)), I.Op("RZ", (2,), param=2)]
    c = gb.circuit_create(I.Circuit(4, ops, 3, density=True))
    c.set_tiling(6, 2)
    st = c.plan_stats(gb.C64, for_grad=True)
    assert st["passes"] >= 3  # the two channels are passes of their own between tile passes


def _superop(kraus):
    """sum_s K_s (ket, matrix bit 0) x conj(K_s) (bra, matrix bit 1), Eq. channel2."""
    return sum(np.kron(np.conj(k), k) for k in kraus)


def test_gate_shape_classification_host(lib):
    # the sweep a matrix takes: exact structure decides (textbook gates and channels)
    s2, c, s = np.sqrt(0.5), np.cos(0.15), np.sin(0.15)
    cases = {
        "DIAG1": np.diag([1, 1j]),
        "ANTI1": np.array([[0, 1], [1, 0]]),
        "REAL1": s2 * np.array([[1, 1], [1, -1]]),
        "IMAG1": np.array([[c, -1j * s], [-1j * s, c]]),
        "DENSE1": 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]]),  # sqrt(X)
        "CX": np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]]),  # control = first qubit
        "CZ": np.diag([1, 1, 1, -1]),
        "DIAG2": np.diag([1, 1, 1, np.exp(0.3j)]),
        "PERM2": np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]]),  # SWAP
        "CTRL2": np.array([[1, 0, 0, 0], [0, c, 0, -1j * s], [0, 0, 1, 0], [0, -1j * s, 0, c]]),
        "BLOCK2": np.array([[1, 0, 0, 0], [0, c, -1j * s, 0], [0, -1j * s, c, 0], [0, 0, 0, np.exp(-0.2j)]]),
        "DENSE2": np.eye(4) + 0.1 * np.arange(16).reshape(4, 4),
    }
    for name, m in cases.items():
        assert gb.gate_shape(m) == name, name
    # CNOT with the second qubit as control is a permutation; a CZ off by one rounding
    # step is a general diagonal
    assert gb.gate_shape(np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]])) == "PERM2"
    assert gb.gate_shape(np.diag([1, 1, 1, -1 + 2.0 ** -52])) == "DIAG2"
    # one-qubit channel superoperators (Sec. II.B channels, completeness-corrected)
    p, g = 0.1, 0.2
    paulis = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]
    depol = [np.sqrt(1 - 3 * p / 4) * paulis[0]] + [np.sqrt(p / 4) * q for q in paulis[1:]]
    ampdamp = [np.array([[1, 0], [0, np.sqrt(1 - g)]]), np.array([[0, np.sqrt(g)], [0, 0]])]
    phasedamp = [np.array([[1, 0], [0, np.sqrt(1 - g)]]), np.array([[0, 0], [0, np.sqrt(g)]])]
    phased = [np.sqrt(0.9) * np.diag([1, np.exp(0.4j)]), np.sqrt(0.1) * np.array([[0, np.exp(0.3j)], [np.exp(-1.1j), 0]])]
    assert gb.gate_shape(_superop(depol)) == "RPAR2"
    assert gb.gate_shape(_superop(ampdamp)) == "RPAR2"
    assert gb.gate_shape(_superop(phasedamp)) == "DIAG2"
    assert gb.gate_shape(_superop(phased)) == "PAR2"
    rng = np.random.default_rng(1)
    assert gb.gate_shape(_superop(I.random_kraus(rng, 3))) == "DENSE2"
    with pytest.raises(ValueError):
        gb.gate_shape(np.zeros((2, 3)))
    with pytest.raises(gb.GbvqcError):
        gb.gate_shape(np.eye(8))


# ------------------------------------------------- status codes and fault injection

def _run_child(code, env_extra):
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=300)


def test_allocation_cap_returns_oom(lib):
    """GBVQC_DEVICE_ALLOC_LIMIT caps the library's device memory: with a cap of 0 bytes
    every allocation fails with ERR_OOM before any CUDA call (so this runs without a
    GPU), and the message names the cap."""
    code = ("import paper_2406_19212_gb300 as gb\n"
            "from paper_2406_19212_gb300 import inputs as I\n"
            "try:\n    gb.sv_alloc(4)\nexcept gb.GbvqcError as e:\n    print('sv_alloc', e.status, e)\n"
            "w = I.plain_10q()\n"
            "c = gb.circuit_create(w.circuit)\n"
            "o = gb.obs_create(w.observable, 10)\n"
            "try:\n    gb.grad(c, w.theta, o)\nexcept gb.GbvqcError as e:\n    print('grad', e.status)\n"
            "print('mem', gb.mem_info())\n")
    res = _run_child(code, {"GBVQC_DEVICE_ALLOC_LIMIT": "0"})
    assert res.returncode == 0, res.stderr
    lines = res.stdout.splitlines()
    assert lines[0].startswith("sv_alloc 2 ") and "GBVQC_DEVICE_ALLOC_LIMIT" in lines[0], res.stdout
    assert "grad 2" in lines, res.stdout
    assert "mem (0, 0)" in lines, res.stdout


def test_no_device_returns_cuda_error(lib):
    """Without a usable GPU the first device allocation fails inside CUDA: ERR_CUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    expect_status(3, gb.sv_alloc, 4)


def test_wrappers_reject_host_tensors(lib):
    """sv_wrap and expect_noalloc take CUDA tensors only: a host tensor, or anything
    else, is refused before the library sees a pointer."""
    import torch
    psi = torch.zeros(16, dtype=torch.complex64)
    out = torch.zeros(1, dtype=torch.float64)
    expect_status(1, gb.sv_wrap, psi, 4)
    expect_status(1, gb.sv_wrap, np.zeros(16, np.complex64), 4)
    expect_status(1, gb.expect_noalloc, psi, 4, [(1.0, ((0, "Z"),))], out)
    expect_status(1, gb.sv_wrap, psi, 0)


def test_specialised_sources_compile_host(lib, tmp_path, monkeypatch):
    """The generated CUDA of every record kind compiles with NVRTC for sm_103a without a
    GPU (one-qubit layers and gates, table and factor-pair phase blocks, two-qubit gates,
    FSIM probes, density circuits with barrier passes), and a second call finds every
    kernel in the cache."""
    from tests.test_gpu_parity import _noisy_two_qubit_channels
    monkeypatch.setenv("GBVQC_JIT_CACHE", str(tmp_path))
    circs = [I.random_circuit(9, 120, 4).circuit, I.fsim_grid_vqe(3, 3, 2, 7, pmask=0b11111).circuit,
             _noisy_two_qubit_channels(5, 3)[0]]
    for circ in circs:
        c = gb.circuit_create(circ)
        c.set_tiling(7, 2)
        for dtype in (gb.C64, gb.C128):
            for for_grad in (True, False):
                info = c.specialize(dtype, for_grad)
                assert info["kernels"] >= 1
                assert c.specialize(dtype, for_grad)["cached"] == info["kernels"]
