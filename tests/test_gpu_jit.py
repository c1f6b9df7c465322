"""Parity of the specialised tile passes (GBVQC_MODE_JIT) with the FP64 oracle.

Each circuit's passes are generated from its fused plan and compiled at run time; the
circuits below exercise every record the generator emits: one-qubit layers and single
gates of every shape, phase blocks in table and factor-pair form, two-qubit gates of
every shape (the two-qubit kernel flavour), variational FSIM probes, density circuits
with separate Phi / Psi phases and two-qubit channel barrier passes, both precisions.
Tolerances are those of the other parity tests.
"""
import os
import tempfile

import numpy as np
import pytest

import paper_2406_19212_gb300 as gb
from oracle import oracle as O
from paper_2406_19212_gb300 import inputs as I
from tests.test_gpu_parity import (DTYPES, _noisy_two_qubit_channels, amp_tol, check_amps, check_energy,
                                   check_grad)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def jit_cache():
    """A private compilation cache for this module (the first compile of each plan is
    real, repeats hit the cache)."""
    old = os.environ.get("GBVQC_JIT_CACHE")
    with tempfile.TemporaryDirectory() as d:
        os.environ["GBVQC_JIT_CACHE"] = d
        yield d
    if old is None:
        os.environ.pop("GBVQC_JIT_CACHE", None)
    else:
        os.environ["GBVQC_JIT_CACHE"] = old


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,ops,seed", [(6, 80, 3), (9, 120, 4), (13, 200, 5)])
def test_jit_apply_and_grad_random(n, ops, seed, dtype):
    w = I.random_circuit(n, ops, seed)
    c = gb.circuit_create(w.circuit)
    sv = gb.sv_alloc(n, dtype)
    gb.apply_circuit(sv, c, w.theta, gb.JIT)
    check_amps(gb.sv_get(sv).astype(np.complex128), O.apply_circuit(w.circuit, w.theta), dtype)
    obs = gb.obs_create(w.observable, n)
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    for k in range(2):  # the second call replays the captured graph with new angles
        th = w.theta + 0.37 * k
        e_ref, g_ref = O.adjoint_grad(w.circuit, th, w.observable)
        e, g = gb.grad(c, th, obs, dtype, gb.JIT)
        check_energy(e, e_ref, dtype)
        check_grad(g, g_ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_jit_small_tiles_and_density(dtype):
    """Density circuit with two-qubit channels (barrier passes, separate Psi phases) on
    7-qubit tiles, so one state spans many tiles."""
    circ, theta, obs = _noisy_two_qubit_channels(5, 3)
    c = gb.circuit_create(circ)
    c.set_tiling(7, 2)
    sv = gb.sv_alloc(5, dtype, True)
    gb.apply_circuit(sv, c, theta, gb.JIT)
    np.testing.assert_allclose(gb.sv_get(sv).astype(np.complex128), O.rho_apply_circuit(circ, theta),
                               atol=amp_tol(dtype, 4), rtol=0)
    e, g = gb.grad(c, theta, gb.obs_create(obs, 5), dtype, gb.JIT)
    e_ref, g_ref = O.noisy_adjoint_grad(circ, theta, obs)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_jit_variational_fsim(dtype):
    w = I.fsim_grid_vqe(3, 3, 4, 7, pmask=0b11111)
    c = gb.circuit_create(w.circuit)
    e, g = gb.grad(c, w.theta, gb.obs_create(w.observable, w.circuit.n_qubits), dtype, gb.JIT)
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)


def test_jit_vqe20_full_gradient():
    """The benchmark's 20-qubit gradient in the benchmark's launch configuration (the
    autotuned tiling of the benchmark: 12 tile qubits, 4 low), both precisions."""
    w = I.diff_20q()
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    c = gb.circuit_create(w.circuit)
    c.set_tiling(12, 4)
    obs = gb.obs_create(w.observable, 20)
    info = c.specialize(gb.C64, True)
    assert info["kernels"] == c.plan_stats(gb.C64, True)["passes"] * 2
    gmax = np.abs(g_ref).max()
    for dtype in DTYPES:
        for k in range(2):
            e, g = gb.grad(c, w.theta, obs, dtype, gb.JIT)
            if dtype == gb.C64:
                assert abs(e - e_ref) <= 1e-5 * max(1.0, abs(e_ref))
                assert np.abs(g - g_ref).max() <= 1e-4 * gmax
            else:
                assert abs(e - e_ref) <= 1e-10
                assert np.abs(g - g_ref).max() <= 1e-10
    assert c.specialize(gb.C64, True)["cached"] == info["kernels"]  # now all in the cache


def test_jit_rqc24_matches_oracle():
    w = I.precision_24q()
    ref = O.apply_circuit(w.circuit, w.theta)
    c = gb.circuit_create(w.circuit)
    for dtype in DTYPES:
        sv = gb.sv_alloc(24, dtype)
        gb.apply_circuit(sv, c, (), gb.JIT)
        got = gb.sv_get(sv).astype(np.complex128)
        sv.free()
        check_amps(got, ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", [gb.FUSED, gb.JIT])
def test_grad_rotation_angles_at_the_shear_branches(dtype, mode):
    """Gradient plans apply Ry as three shears, with the shears of -R where cos(theta/2) < 0
    (a global sign that Phi and Psi share).  Angles on and around the branch point
    (theta = pi), near 0 and 2 pi, and beyond [0, 2 pi): energy and gradient against the
    oracle, which applies the rotation matrices directly."""
    n = 11
    angles = [0.0, np.pi, np.pi - 1e-7, np.pi + 1e-7, 2 * np.pi - 1e-9, 3 * np.pi, -np.pi / 2, 0.5, 2.5, 4.0, 5.9]
    ops, p = [], 0
    for layer in range(3):
        for q in range(n):
            ops.append(I.Op("RY", (q,), param=p))
            p += 1
        for q in range(layer % 2, n - 1, 2):
            ops.append(I.Op("CZ", (q, q + 1)))
        ops.append(I.Op("RY", ((layer * 5) % n,), fixed=(angles[layer * 3 % len(angles)],)))
    theta = np.array([angles[i % len(angles)] for i in range(p)])
    circuit = I.Circuit(n, ops, p)
    obs = [(0.7, ((q, "X"),)) for q in range(n)] + [(1.0, ((q, "Z"), (q + 1, "Z"))) for q in range(n - 1)]
    e_ref, g_ref = O.adjoint_grad(circuit, theta, obs)
    e, g = gb.grad(gb.circuit_create(circuit), theta, gb.obs_create(obs, n), dtype, mode)
    check_energy(e, e_ref, dtype)
    check_grad(g, g_ref, dtype)
