"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Tolerances: complex128 amplitudes 1e-12; complex64 fidelity >= 1 - 1e-6 and
amplitudes 2e-5; energies 1e-5 relative (complex64) / 1e-10 (complex128); gradients
1e-4 * max|g| (complex64) / 1e-10 * max(1, max|g|) (complex128).
"""
import math

import numpy as np
import pytest

import paper_2406_19212_gb300 as gb
from oracle import oracle as O
from paper_2406_19212_gb300 import inputs as I

pytestmark = pytest.mark.gpu

AMP_TOL = {gb.C64: 2e-5, gb.C128: 1e-12}
MODES = [gb.PLAIN, gb.FUSED]


def amp_tol(dtype, c64_factor=1):
    """Amplitude tolerance; c64_factor widens the complex64 bound only, for density
    matrices after a measurement and for 16x16 two-qubit superoperators, where one
    output element sums up to 4x as many FP32-rounded products as a one-qubit gate's.
    The complex128 bound stays 1e-12."""
    return AMP_TOL[dtype] * (c64_factor if dtype == gb.C64 else 1)
DTYPES = [gb.C64, gb.C128]


def fidelity(a, b):
    return abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def run_apply(circuit, theta, dtype, mode, start=None, tiling=None):
    c = gb.circuit_create(circuit)
    if tiling:
        c.set_tiling(*tiling)
    sv = gb.sv_alloc(circuit.n_qubits, dtype, circuit.density)
    if start is not None:
        gb.sv_set(sv, start)
    gb.apply_circuit(sv, c, theta, mode)
    return gb.sv_get(sv).astype(np.complex128)


def check_amps(got, ref, dtype):
    np.testing.assert_allclose(got, ref, atol=AMP_TOL[dtype], rtol=0)
    if dtype == gb.C64:
        assert fidelity(got, ref) >= 1 - 1e-6


def check_grad(g, ref, dtype):
    scale = max(1.0, float(np.abs(ref).max())) if ref.size else 1.0
    tol = 1e-4 * max(float(np.abs(ref).max()), 1e-12) if dtype == gb.C64 else 1e-10 * scale
    np.testing.assert_allclose(g, ref, atol=tol, rtol=0)


def check_energy(e, ref, dtype):
    if dtype == gb.C64:
        assert abs(e - ref) <= 1e-5 * max(1.0, abs(ref))
    else:
        assert abs(e - ref) <= 1e-10 * max(1.0, abs(ref))


# ----------------------------------------------------------------- state evolution

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,ops,seed", [(1, 20, 0), (2, 30, 1), (5, 60, 2), (6, 80, 3),
                                        (9, 120, 4), (13, 200, 5), (15, 150, 6)])
def test_apply_matches_oracle(n, ops, seed, dtype, mode):
    w = I.random_circuit(n, ops, seed)
    ref = O.apply_circuit(w.circuit, w.theta)
    check_amps(run_apply(w.circuit, w.theta, dtype, mode), ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_apply_from_custom_state(dtype):
    w = I.random_circuit(11, 150, 7)
    start = I.random_state(11, 8)
    ref = O.apply_circuit(w.circuit, w.theta, start)
    for mode in MODES:
        check_amps(run_apply(w.circuit, w.theta, dtype, mode, start=start), ref, dtype)


@pytest.mark.parametrize("tiling", [(6, 1), (7, 2), (8, 3), (10, 4), (12, 6), (13, 4), (13, 1)])
def test_fused_tilings(tiling):
    w = I.random_circuit(14, 250, 9)
    ref = O.apply_circuit(w.circuit, w.theta)
    for dtype in DTYPES:
        t = tiling if not (dtype == gb.C128 and tiling[0] > 12) else (12, tiling[1])
        check_amps(run_apply(w.circuit, w.theta, dtype, gb.FUSED, tiling=t), ref, dtype)


def test_ghz_and_qft_closed_forms():
    n = 16
    ops = [I.Op("H", (0,))] + [I.Op("CNOT", (i, i + 1)) for i in range(n - 1)]
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    for dtype in DTYPES:
        for mode in MODES:
            check_amps(run_apply(I.Circuit(n, ops, 0), [], dtype, mode), ref, dtype)
    from tests.test_oracle import qft_ops
    n, x = 12, 1234
    psi0 = np.zeros(1 << n, dtype=complex)
    psi0[x] = 1
    y = np.arange(1 << n)
    ref = np.exp(2j * np.pi * x * y / 2 ** n) / 2 ** (n / 2)
    for dtype in DTYPES:
        for mode in MODES:
            check_amps(run_apply(I.Circuit(n, qft_ops(n), 0), [], dtype, mode, start=psi0), ref, dtype)


def test_empty_circuit_and_reset():
    for dtype in DTYPES:
        for mode in MODES:
            got = run_apply(I.Circuit(7, [], 0), [], dtype, mode)
            assert got[0] == 1 and np.count_nonzero(got) == 1


# ------------------------------------------------------------------- expectation

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,seed", [(1, 0), (4, 1), (10, 2), (16, 3)])
def test_expect_matches_oracle(n, seed, dtype):
    psi = I.random_state(n, seed)
    terms = I.random_circuit(n, 1, seed).observable
    if n > 1:
        terms = terms + I.heisenberg_1d(n, 0.7, -1.3) + [(0.25, tuple((q, "Y") for q in range(n)))]
    sv = gb.sv_alloc(n, dtype)
    gb.sv_set(sv, psi)
    e = gb.expect(sv, gb.obs_create(terms, n))
    check_energy(e, O.expect(terms, psi, n), dtype)


def rich_observable(n, seed, count=16):
    """Pauli strings on random qubits (the highest ones included), each with two companions
    on the same X mask: its X and Y factors exchanged, and an extra Z factor.  Groups of
    equal X mask then hold several terms whose Z masks and Y counts differ, so a group's
    coefficient is complex and depends on the amplitude index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    terms = []
    for _ in range(count):
        k = int(rng.integers(1, 5))
        qs = [int(q) for q in sorted(rng.choice(n, size=k, replace=False))]
        ps = ["XYZ"[int(rng.integers(0, 3))] for _ in qs]
        if all(p == "Z" for p in ps):
            ps[0] = "X"
        c = float(rng.normal())
        terms.append((c, tuple(zip(qs, ps))))
        swapped = ["Y" if p == "X" else "X" if p == "Y" else p for p in ps]
        terms.append((0.5 * c, tuple(zip(qs, swapped))))
        free = [q for q in range(n) if q not in qs]
        z = int(rng.choice(free))
        terms.append((-0.25 * c, tuple(sorted(list(zip(qs, ps)) + [(z, "Z")]))))
    return terms


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,seed", [(10, 21), (11, 22), (15, 23)])
def test_expect_rich_observable(n, seed, dtype):
    """Groups flipping qubits inside and outside a 2^10-amplitude chunk, complex group
    coefficients, Z masks on every qubit."""
    psi = I.random_state(n, seed)
    terms = rich_observable(n, seed)
    sv = gb.sv_alloc(n, dtype)
    gb.sv_set(sv, psi)
    check_energy(gb.expect(sv, gb.obs_create(terms, n)), O.expect(terms, psi, n), dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES + [gb.JIT])
@pytest.mark.parametrize("n,seed", [(12, 31), (14, 32)])
def test_grad_rich_observable(n, seed, dtype, mode):
    """The adjoint seed lambda = H Phi of an observable with complex, index-dependent group
    coefficients and flips of high qubits: every gradient entry is a linear functional of
    lambda, compared with the oracle's."""
    w = I.random_circuit(n, 90, seed)
    terms = rich_observable(n, seed)
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, terms)
    e, g = gb.grad(gb.circuit_create(w.circuit), w.theta, gb.obs_create(terms, n), dtype, mode)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


# --------------------------------------------------------------------- gradients

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,ops,seed,share", [(2, 30, 11, False), (6, 80, 12, True),
                                              (9, 150, 13, False), (13, 160, 14, True)])
def test_grad_matches_oracle(n, ops, seed, share, dtype, mode):
    w = I.random_circuit(n, ops, seed, param_share=share)
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    c = gb.circuit_create(w.circuit)
    e, g = gb.grad(c, w.theta, gb.obs_create(w.observable, n), dtype, mode)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)
    # second call replays the captured graph with new angles
    th2 = w.theta + 0.37
    e_ref2, g_ref2 = O.adjoint_grad(w.circuit, th2, w.observable)
    e2, g2 = gb.grad(c, th2, gb.obs_create(w.observable, n), dtype, mode)
    check_energy(e2, e_ref2, dtype)
    check_grad(g2, g_ref2, dtype)


def test_plain10_config_and_finite_differences():
    w = I.plain_10q()
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 10)
    for dtype in DTYPES:
        for mode in MODES:
            e, g = gb.grad(c, w.theta, obs, dtype, mode)
            check_energy(e, e_ref, dtype)
            check_grad(g, g_ref, dtype)
    # central differences of the GPU complex128 energy, h = 1e-5
    e, g = gb.grad(c, w.theta, obs, gb.C128, gb.PLAIN)
    for j in (0, 41, 119):
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[j] += 1e-5
        tm[j] -= 1e-5
        fd = (gb.grad(c, tp, obs, gb.C128, gb.PLAIN)[0] - gb.grad(c, tm, obs, gb.C128, gb.PLAIN)[0]) / 2e-5
        assert abs(fd - g[j]) < 1e-8


def test_grad_device_pointers_and_autograd():
    import torch
    w = I.plain_10q(seed=5)
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 10)
    th = torch.tensor(w.theta, device="cuda", dtype=torch.float64)
    e, g = gb.grad(c, th, obs, gb.C64, gb.FUSED)
    torch.cuda.synchronize()
    check_energy(float(e.item()), e_ref, gb.C64)
    check_grad(g.cpu().numpy(), g_ref, gb.C64)
    th.requires_grad_(True)
    loss = gb.VQEEnergy.apply(th, c, obs, gb.C128, gb.FUSED)
    loss.backward()
    check_energy(float(loss.item()), e_ref, gb.C128)
    check_grad(th.grad.cpu().numpy(), g_ref, gb.C128)


def test_zero_parameter_grad():
    w = I.random_circuit(8, 40, 21)
    ops = [o for o in w.circuit.ops if o.param < 0]
    circ = I.Circuit(8, ops, 0)
    c = gb.circuit_create(circ)
    for dtype in DTYPES:
        e, g = gb.grad(c, np.zeros(0), gb.obs_create(w.observable, 8), dtype, gb.FUSED)
        check_energy(e, O.energy(circ, [], w.observable), dtype)
        assert g.size == 0


# ------------------------------------------------------------------------ density

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,ops,seed", [(1, 10, 0), (3, 40, 1), (4, 60, 2), (6, 80, 3)])
def test_density_apply_matches_oracle(n, ops, seed, dtype, mode):
    w = I.random_circuit(n, ops, seed, density=True, with_channels=True)
    start = I.random_density(n, seed + 50)
    ref = O.rho_apply_circuit(w.circuit, w.theta, start)
    check_amps(run_apply(w.circuit, w.theta, dtype, mode, start=start), ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_apply_channel_matches_oracle(dtype):
    n = 5
    rho = I.random_density(n, 3)
    rng = np.random.default_rng(4)
    sv = gb.sv_alloc(n, dtype, True)
    gb.sv_set(sv, rho)
    ops = []
    for name, q, p in (("DEPOL", 0, 0.2), ("AMPDAMP", 4, 0.3), ("PHASEDAMP", 2, 0.5)):
        gb.apply_channel(sv, name, q, p)
        ops.append(I.Op(name, (q,), fixed=(p,)))
    ks = I.random_kraus(rng, 3)
    gb.apply_channel(sv, "KRAUS", 3, kraus=ks)
    ops.append(I.Op("KRAUS", (3,), data=ks))
    ref = O.rho_apply_circuit(I.Circuit(n, ops, 0, True), [], rho)
    check_amps(gb.sv_get(sv).astype(np.complex128), ref, dtype)
    with pytest.raises(gb.GbvqcError):
        gb.apply_channel(gb.sv_alloc(3, dtype), "DEPOL", 0, 0.1)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,ops,seed", [(2, 30, 31), (3, 50, 32), (5, 70, 33)])
def test_noisy_grad_matches_oracle(n, ops, seed, dtype, mode):
    w = I.random_circuit(n, ops, seed, density=True, with_channels=True, param_share=True)
    e_ref, g_ref = O.noisy_adjoint_grad(w.circuit, w.theta, w.observable)
    c = gb.circuit_create(w.circuit)
    e, g = gb.grad(c, w.theta, gb.obs_create(w.observable, n), dtype, mode)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_noisy_hea_small_matches_oracle(dtype):
    w = I.noisy_hea(6, 3, 9)
    e_ref, g_ref = O.noisy_adjoint_grad(w.circuit, w.theta, w.observable)
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 6)
    for mode in MODES:
        e, g = gb.grad(c, w.theta, obs, dtype, mode)
        check_energy(e, e_ref, dtype)
        check_grad(g, g_ref, dtype)


def test_density_trace_and_expect():
    w = I.noisy_hea(5, 2, 3)
    ref = O.rho_apply_circuit(w.circuit, w.theta)
    for dtype in DTYPES:
        sv = gb.sv_alloc(5, dtype, True)
        gb.apply_circuit(sv, gb.circuit_create(w.circuit), w.theta, gb.FUSED)
        tr = gb.expect(sv, gb.obs_create([(1.0, ())], 5))
        # each FP32-rounded superoperator preserves the trace to ~2 eps (eps = 6e-8)
        n_ch = sum(1 for o in w.circuit.ops if o.name in I.CHANNELS)
        assert abs(tr - 1.0) < (4 * n_ch * 6e-8 if dtype == gb.C64 else 1e-13)
        check_energy(gb.expect(sv, gb.obs_create(w.observable, 5)),
                     O.rho_expect(w.observable, ref, 5), dtype)


# ------------------------------------------------------------------------- errors

def test_argument_errors():
    w = I.random_circuit(4, 10, 1)
    c = gb.circuit_create(w.circuit)
    with pytest.raises(gb.GbvqcError):
        gb.apply_circuit(gb.sv_alloc(5, gb.C64), c, w.theta)
    with pytest.raises(gb.GbvqcError):
        gb.grad(c, np.zeros(w.circuit.n_params + 1), gb.obs_create(w.observable, 4))
    with pytest.raises(gb.GbvqcError):
        gb.grad(c, w.theta, gb.obs_create(w.observable + [(1.0, ((5, "Z"),))], 6))


# ------------------------------------------- phase-normalised one-qubit gates (fused)

def _sqrt_layers(n, extra, seed):
    """sqrt(X/Y/W) layers plus `extra` gates: exercises the fused engine's global-phase
    bookkeeping (normalised gates, and the gate that takes the phase back)."""
    rng = np.random.default_rng(seed)
    ops, n_par = [], 0
    for layer in range(4):
        for q in range(n):
            ops.append(I.Op(("SX", "SY", "SW")[int(rng.integers(0, 3))], (q,)))
        for q in range(layer % 2, n - 1, 2):
            if extra == "cz":
                ops.append(I.Op("CZ", (q, q + 1)))
            elif extra == "t":
                ops.append(I.Op("T", (q,)))
            elif extra == "ry":
                ops.append(I.Op("RY", (q,), param=n_par))
                n_par += 1
    return I.Circuit(n, ops, n_par), rng.uniform(0, 2 * math.pi, n_par)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("extra", ["none", "cz", "t", "ry"])
def test_fused_sqrt_gates_exact_state(dtype, extra):
    circ, theta = _sqrt_layers(9, extra, 11)
    ref = O.apply_circuit(circ, theta)
    got = run_apply(circ, theta, dtype, gb.FUSED, tiling=(7, 2))
    check_amps(got, ref, dtype)
    # gradient and energy do not depend on global phases either way
    if circ.n_params:
        obs = I.ising_chain(9, [0.7] * 9)
        e_ref, g_ref = O.adjoint_grad(circ, theta, obs)
        c = gb.circuit_create(circ)
        o = gb.obs_create(obs, 9)
        e, g = gb.grad(c, theta, o, dtype, gb.FUSED)
        check_energy(e, e_ref, dtype)
        check_grad(g, g_ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_fused_grad_permuted_layout_heisenberg(dtype):
    """Gradient plan in a permuted qubit layout (CNOT ladder wider than the tile) with an
    observable holding X, Y and Z factors: the masks are permuted on the host."""
    rng = np.random.default_rng(5)
    w = I.ry_rz_cnot_instance(14, 6, rng)
    obs = I.heisenberg_1d(14, hz=0.3, J=0.8)
    c = gb.circuit_create(w.circuit)
    c.set_tiling(9, 2)
    assert c.plan_stats(dtype, for_grad=True)["passes"] <= c.plan_stats(dtype, for_grad=False)["passes"]
    o = gb.obs_create(obs, 14)
    e, g = gb.grad(c, w.theta, o, dtype, gb.FUSED)
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, obs)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
def test_heisenberg_random_circuit_gradient(dtype, mode):
    """Random rotations + CNOT brick with the Heisenberg observable (XX and YY groups)."""
    w = I.random_rotation_heisenberg(11, 6, 21)
    c = gb.circuit_create(w.circuit)
    o = gb.obs_create(w.observable, 11)
    e, g = gb.grad(c, w.theta, o, dtype, mode)
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


# ----------------------------------------------------------------- measurement

@pytest.mark.parametrize("dtype", DTYPES)
def test_measure_listing4_on_gpu(dtype):
    """Listing 4 end to end: apply the circuit, measure qubit 2 (0-based 1); the outcome
    probabilities are the hand-derived ones of tests/golden/listing4.txt."""
    c = I.Circuit(2, [I.Op("H", (0,)), I.Op("RY", (0,), fixed=(math.pi / 4,)),
                      I.Op("CNOT", (0, 1))], 0)
    for u, k_ref, p_ref, idx in ((0.1, 0, (2 - math.sqrt(2)) / 4, 0), (0.9, 1, (2 + math.sqrt(2)) / 4, 3)):
        sv = gb.sv_alloc(2, dtype)
        gb.apply_circuit(sv, gb.circuit_create(c), [], gb.PLAIN)
        k, p = gb.measure(sv, 1, u)
        assert k == k_ref
        assert p == pytest.approx(p_ref, abs=1e-7 if dtype == gb.C64 else 1e-14)
        ref = np.zeros(4, complex)
        ref[idx] = 1
        check_amps(gb.sv_get(sv).astype(np.complex128), ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("density", [False, True])
def test_measure_sequence_matches_oracle(dtype, density):
    """Three measurements in a row on a random (pure: 11 qubits; density: 5) state:
    outcome, probability and collapsed state against the oracle after each one."""
    n = 5 if density else 11
    if density:
        rho = I.random_density(n, 8)
        state = rho.T.reshape(-1).astype(np.complex128)
    else:
        state = I.random_state(n, 8)
    sv = gb.sv_alloc(n, dtype, density)
    gb.sv_set(sv, state)
    ref = state
    for q, u in ((0, 0.37), (n - 1, 0.81), (2, 0.05)):
        k, p = gb.measure(sv, q, u)
        k_ref, p_ref, ref = O.measure(ref, n, q, u, density=density)
        assert k == k_ref
        assert p == pytest.approx(p_ref, abs=1e-6 if dtype == gb.C64 else 1e-12)
        got = gb.sv_get(sv).astype(np.complex128)
        np.testing.assert_allclose(got, ref, atol=amp_tol(dtype, 4 if density else 1), rtol=0)


def test_measure_rejects_bad_arguments():
    sv = gb.sv_alloc(3, gb.C64)
    for q, u in ((3, 0.5), (-1, 0.5), (0, 1.0), (0, -0.1), (0, float("nan"))):
        with pytest.raises(gb.GbvqcError):
            gb.measure(sv, q, u)


# ----------------------------------------------------------------- variational FSIM

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("pmask", [0b00011, 0b11111, 0b10100])
def test_fsim_parameter_gradients(dtype, mode, pmask):
    """Grid circuit whose FSIM couplers carry variational parameters (the paper's isparas
    mask over theta, phi and the three Delta's): energy and every gradient vs the oracle."""
    w = I.fsim_grid_vqe(3, 4, 6, 17, pmask=pmask)
    c = gb.circuit_create(w.circuit)
    if mode == gb.FUSED:
        c.set_tiling(8, 2)
    o = gb.obs_create(w.observable, 12)
    e, g = gb.grad(c, w.theta, o, dtype, mode)
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


def test_fsim_parameter_gradients_batched():
    ws = [I.fsim_grid_vqe(3, 3 + i, 4 + i, 30 + i, pmask=(0b00011, 0b11111, 0b01001)[i]) for i in range(3)]
    circs = [gb.circuit_create(w.circuit) for w in ws]
    obss = [gb.obs_create(w.observable, w.circuit.n_qubits) for w in ws]
    energies, grads = gb.batch_create(circs, obss, gb.C128).grad([w.theta for w in ws])
    for w, e, g in zip(ws, energies, grads):
        e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
        check_energy(e, e_ref, gb.C128)
        check_grad(g, g_ref, gb.C128)


# ----------------------------------------------------------------- two-qubit channels

def _noisy_two_qubit_channels(n, seed):
    """Rx.Rz layers with CNOTs followed by two-qubit depolarising, plus random two-qubit
    Kraus channels (QuantumMap on two positions) of weak strength: the reverse sweep
    uncomputes with the superoperator inverse, whose norm grows with the noise, so strong
    random channels amplify complex64 rounding beyond the gradient tolerance."""
    rng = np.random.default_rng(seed)
    ops, p = [], 0
    for layer in range(3):
        for q in range(n):
            ops += [I.Op("RX", (q,), param=p), I.Op("RZ", (q,), param=p + 1)]
            p += 2
        for q in range(layer % 2, n - 1, 2):
            ops += [I.Op("CNOT", (q, q + 1)), I.Op("DEPOL2", (q, q + 1), fixed=(0.02,))]
        a, b = rng.choice(n, 2, replace=False)
        ops.append(I.Op("KRAUS2", (int(a), int(b)), data=I.random_kraus2(rng, 2 + layer, weight=0.05)))
    theta = rng.uniform(0, 2 * math.pi, p)
    obs = I.ising_chain(n, [0.5] * n) + [(0.3, ((0, "Y"), (n - 1, "X")))]
    return I.Circuit(n, ops, p, density=True), theta, obs


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
def test_two_qubit_channels_apply_and_grad(dtype, mode):
    n = 5
    circ, theta, obs = _noisy_two_qubit_channels(n, 3)
    ref = O.rho_apply_circuit(circ, theta)
    got = run_apply(circ, theta, dtype, mode, tiling=(7, 2) if mode == gb.FUSED else None)
    np.testing.assert_allclose(got, ref, atol=amp_tol(dtype, 4), rtol=0)
    c = gb.circuit_create(circ)
    if mode == gb.FUSED:
        c.set_tiling(7, 2)
    o = gb.obs_create(obs, n)
    e, g = gb.grad(c, theta, o, dtype, mode)
    e_ref, g_ref = O.noisy_adjoint_grad(circ, theta, obs)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


def test_two_qubit_channels_rejected_by_batches():
    """Batches take pure-state circuits only (a density circuit is refused before its
    plan, so a two-qubit channel never reaches the batched kernels)."""
    circ, theta, obs = _noisy_two_qubit_channels(4, 9)
    c = gb.circuit_create(circ)
    o = gb.obs_create(obs, 4)
    with pytest.raises(gb.GbvqcError) as ex:
        gb.batch_create([c], [o], gb.C64)
    assert ex.value.status == 1


# ----------------------------------------------------------------- sampling

def _check_samples(got, weights, u):
    """Equal to the oracle's sequential-CDF answer, except that within rounding of a CDF
    boundary either neighbouring index is valid."""
    cdf = np.cumsum(weights)
    total = cdf[-1]
    for g, uu in zip(got, u):
        t = uu * total
        lo = cdf[g - 1] if g > 0 else 0.0
        assert weights[g] > 0
        assert lo - 1e-12 * total <= t <= cdf[g] + 1e-12 * total


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("density", [False, True])
def test_sample_matches_oracle(dtype, density):
    n = 5 if density else 13
    if density:
        state = I.random_density(n, 12)
    else:
        state = I.random_state(n, 12)
    sv = gb.sv_alloc(n, dtype, density)
    gb.sv_set(sv, state)
    stored = gb.sv_get(sv).astype(np.complex128)  # the amplitudes the GPU sampled from
    u = np.random.default_rng(3).uniform(0, 1, 3000)
    got = gb.sample(sv, u)
    ref = O.sample(stored, n, u, density=density)
    d = 1 << n
    w = (stored[np.arange(d) * (d + 1)].real if density else np.abs(stored) ** 2)
    _check_samples(got, w, u)
    assert np.mean(got == ref) > 0.999
    np.testing.assert_array_equal(gb.sv_get(sv), stored.astype(gb.sv_get(sv).dtype))  # unchanged


def test_sample_small_register_and_ghz():
    n = 3  # smaller than one warp's scan step
    c = I.Circuit(n, [I.Op("H", (0,)), I.Op("CNOT", (0, 1)), I.Op("CNOT", (1, 2))], 0)
    sv = gb.sv_alloc(n, gb.C128)
    gb.apply_circuit(sv, gb.circuit_create(c), [], gb.PLAIN)
    assert gb.sample(sv, [0.0, 0.2, 0.49, 0.51, 0.999]).tolist() == [0, 0, 0, 7, 7]
    with pytest.raises(gb.GbvqcError):
        gb.sample(sv, [1.0])


@pytest.mark.parametrize("dtype", DTYPES)
def test_sample_largest_draw_with_zero_tail(dtype):
    """u = nextafter(1, 0) on a state whose weight ends before the last chunks (13 qubits:
    chunks of 32 amplitudes, most of them empty) returns the last index of non-zero
    weight, as the oracle does."""
    n = 13
    rng = np.random.default_rng(21)
    for last in (40, 1000, 4095):
        psi = np.zeros(1 << n, complex)
        psi[: last + 1] = rng.normal(size=last + 1) + 1j * rng.normal(size=last + 1)
        sv = gb.sv_alloc(n, dtype)
        gb.sv_set(sv, psi)
        u = [np.nextafter(1.0, 0.0), 0.0]
        assert gb.sample(sv, u).tolist() == [last, 0]
        assert O.sample(gb.sv_get(sv).astype(np.complex128), n, u).tolist() == [last, 0]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
def test_fsim_parameter_gradients_density(dtype, mode):
    """Variational FSIM couplers inside a noisy density circuit (the ket gate U and the bra
    gate conj(U) each contribute Re <<Psi| dS |Phi>>) against the noisy oracle."""
    n = 4
    ops = [I.Op("RX", (q,), param=q) for q in range(n)]
    p = n
    for (a, b), mask in (((0, 1), 0b11111), ((2, 3), 0b00011), ((1, 2), 0b10101)):
        vals = (1.0 + 0.1 * a, 0.5, 0.2, -0.1, 0.3)
        ops.append(I.Op("FSIM", (a, b), param=p, fixed=vals, pmask=mask))
        p += bin(mask).count("1")
        ops += [I.Op("DEPOL", (a,), fixed=(0.02,)), I.Op("AMPDAMP", (b,), fixed=(0.03,))]
    circ = I.Circuit(n, ops, p, density=True)
    theta = np.random.default_rng(5).uniform(-1, 1, p)
    obs = I.ising_chain(n, [0.6] * n) + [(0.4, ((1, "Y"), (3, "X")))]
    c = gb.circuit_create(circ)
    if mode == gb.FUSED:
        c.set_tiling(7, 2)
    o = gb.obs_create(obs, n)
    e, g = gb.grad(c, theta, o, dtype, mode)
    e_ref, g_ref = O.noisy_adjoint_grad(circ, theta, obs)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


def _phase_covariant_kraus(p, angles):
    """Kraus operators that are each diagonal or anti-diagonal: the superoperator couples
    |00> only with |11> and |01> only with |10> (Eq. channel; complex entries)."""
    a, b, c = angles
    k0 = np.sqrt(1 - p) * np.diag([1.0, np.exp(1j * a)])
    k1 = np.sqrt(p) * np.array([[0, np.exp(1j * b)], [np.exp(1j * c), 0]])
    return [k0, k1]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
def test_parity_preserving_channels(dtype, mode):
    """Channels whose superoperators keep (ket xor bra) of a qubit: the real ones
    (depolarising, amplitude and phase damping, a bit flip) and complex ones (phased
    Kraus operators), inside a variational density circuit, state and gradient."""
    n = 4
    rng = np.random.default_rng(11)
    ops, p = [], 0
    for layer in range(2):
        for q in range(n):
            ops.append(I.Op("RY", (q,), param=p)); p += 1
            ops.append(I.Op("RZ", (q,), param=p)); p += 1
        for q in range(layer % 2, n - 1, 2):
            ops.append(I.Op("CNOT", (q, q + 1)))
        ops += [I.Op("DEPOL", (0,), fixed=(0.05,)), I.Op("AMPDAMP", (1,), fixed=(0.1,)),
                I.Op("PHASEDAMP", (2,), fixed=(0.2,)),
                I.Op("KRAUS", (3,), data=_phase_covariant_kraus(0.1, rng.uniform(-3, 3, 3))),
                I.Op("KRAUS", (layer,), data=_phase_covariant_kraus(0.05, (0.0, 0.0, 0.0))),
                I.Op("KRAUS", (2,), data=[np.sqrt(0.9) * np.eye(2), np.sqrt(0.1) * np.array([[0, 1], [1, 0]])])]
    circ = I.Circuit(n, ops, p, density=True)
    theta = rng.uniform(0, 2 * np.pi, p)
    obs = I.ising_chain(n, [0.7] * n) + [(0.3, ((0, "Y"), (2, "Y")))]
    start = I.random_density(n, 12)
    tiling = (6, 2) if mode == gb.FUSED else None
    check_amps(run_apply(circ, theta, dtype, mode, start=start, tiling=tiling),
               O.rho_apply_circuit(circ, theta, start), dtype)
    c = gb.circuit_create(circ)
    if mode == gb.FUSED:
        c.set_tiling(6, 2)
    o = gb.obs_create(obs, n)
    e, g = gb.grad(c, theta, o, dtype, mode)
    e_ref, g_ref = O.noisy_adjoint_grad(circ, theta, obs)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)
