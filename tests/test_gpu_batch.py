"""Batched gradients (batch_create / batch_grad): every member of a batch must give the
same energy and gradient as its own `grad` call and as the oracle."""
import numpy as np
import pytest

import paper_2406_19212_gb300 as gb
from oracle import oracle as O
from paper_2406_19212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def small_batch(seed=7, count=12, n_lo=6, n_hi=13, d_lo=2, d_hi=6):
    return I.batch_512(seed=seed, count=count, n_lo=n_lo, n_hi=n_hi, d_lo=d_lo, d_hi=d_hi)


@pytest.mark.parametrize("dtype", [gb.C64, gb.C128])
def test_batch_matches_individual_and_oracle(dtype):
    ws = small_batch()
    circs = [gb.circuit_create(w.circuit) for w in ws]
    obss = [gb.obs_create(w.observable, w.circuit.n_qubits) for w in ws]
    b = gb.batch_create(circs, obss, dtype)
    for rep in range(2):  # second call replays the captured graph with new angles
        thetas = [w.theta + 0.21 * rep for w in ws]
        e, gs = b.grad(thetas)
        for i, w in enumerate(ws):
            e1, g1 = gb.grad(circs[i], thetas[i], obss[i], dtype, gb.FUSED)
            tol_e = 1e-5 if dtype == gb.C64 else 1e-10
            assert abs(e[i] - e1) <= tol_e * max(1.0, abs(e1))
            scale = max(np.abs(g1).max(), 1e-12)
            assert np.abs(gs[i] - g1).max() <= (1e-4 * scale if dtype == gb.C64 else 1e-10 * max(1.0, scale))
        for i in (0, len(ws) - 1):
            e_ref, g_ref = O.adjoint_grad(ws[i].circuit, thetas[i], ws[i].observable)
            assert abs(e[i] - e_ref) <= (1e-5 if dtype == gb.C64 else 1e-10) * max(1.0, abs(e_ref))
            tol = 1e-4 * np.abs(g_ref).max() if dtype == gb.C64 else 1e-10 * max(1.0, np.abs(g_ref).max())
            assert np.abs(gs[i] - g_ref).max() <= tol
    b.free()


def test_batch_device_pointers_and_one_shot():
    import torch
    ws = small_batch(seed=9, count=5)
    circs = [gb.circuit_create(w.circuit) for w in ws]
    obss = [gb.obs_create(w.observable, w.circuit.n_qubits) for w in ws]
    b = gb.batch_create(circs, obss)
    th = torch.tensor(np.concatenate([w.theta for w in ws]), device="cuda", dtype=torch.float64)
    e, g = b.grad(th)
    torch.cuda.synchronize()
    e2, gs2 = gb.grad_batch(circs, obss, [w.theta for w in ws])
    np.testing.assert_allclose(e.cpu().numpy(), e2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g.cpu().numpy()[:sum(w.circuit.n_params for w in ws)], np.concatenate(gs2),
                               rtol=0, atol=1e-12)
    b.free()


def test_batch512_full_sample():
    # the full 512-instance batch (12..20 qubits, depths 4..16): a sample of members
    # against their own grad calls, and every energy against its grad call
    ws = I.batch_512()
    circs = [gb.circuit_create(w.circuit) for w in ws]
    obss = [gb.obs_create(w.observable, w.circuit.n_qubits) for w in ws]
    b = gb.batch_create(circs, obss)
    e, gs = b.grad([w.theta for w in ws])
    rng = np.random.default_rng(0)
    for i in rng.choice(len(ws), size=12, replace=False):
        e1, g1 = gb.grad(circs[i], ws[i].theta, obss[i], gb.C64, gb.FUSED)
        assert abs(e[i] - e1) <= 1e-5 * max(1.0, abs(e1))
        assert np.abs(gs[i] - g1).max() <= 1e-4 * np.abs(g1).max()
    assert np.all(np.isfinite(e)) and np.all(np.abs(e) <= [sum(abs(c) for c, _ in w.observable) for w in ws])
    # full-size members against the oracle directly: the largest 20-qubit member, the
    # deepest member and a 12-qubit one
    n20 = [i for i, w in enumerate(ws) if w.circuit.n_qubits == 20]
    big = max(n20, key=lambda i: ws[i].circuit.n_params)
    deep = max(range(len(ws)), key=lambda i: len(ws[i].circuit.ops))
    small = min(range(len(ws)), key=lambda i: ws[i].circuit.n_qubits)
    for i in sorted({big, deep, small}):
        e_ref, g_ref = O.adjoint_grad(ws[i].circuit, ws[i].theta, ws[i].observable)
        assert abs(e[i] - e_ref) <= 1e-5 * max(1.0, abs(e_ref))
        assert np.abs(gs[i] - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    b.free()


def test_batch_autotune_keeps_results():
    """batch_autotune picks member tile sizes in [8, 12] (within each member's qubits)
    and the rebuilt batch still matches the oracle."""
    ws = small_batch(seed=11, count=10, n_lo=8, n_hi=14)
    circs = [gb.circuit_create(w.circuit) for w in ws]
    obss = [gb.obs_create(w.observable, w.circuit.n_qubits) for w in ws]
    b = gb.batch_create(circs, obss)
    thetas = [w.theta for w in ws]
    tiles, ms = b.autotune(thetas)
    assert ms > 0 and len(tiles) == len(ws)
    for t, w in zip(tiles, ws):
        assert min(8, w.circuit.n_qubits) <= t <= min(12, w.circuit.n_qubits)
    for i, c in enumerate(circs):
        assert c.plan_stats(gb.C64, True)["tile_qubits"] == tiles[i]
    e, gs = b.grad(thetas)
    for i in (0, 3, len(ws) - 1):
        e_ref, g_ref = O.adjoint_grad(ws[i].circuit, thetas[i], ws[i].observable)
        assert abs(e[i] - e_ref) <= 1e-5 * max(1.0, abs(e_ref))
        assert np.abs(gs[i] - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    b.free()


def test_autotune_picks_valid_tiling_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("GBVQC_TUNE_CACHE", str(tmp_path / "tune.txt"))
    w = I.random_circuit(14, 200, 17, param_share=True)
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 14)
    t, lo, ms = c.autotune(w.theta, obs)
    assert 8 <= t <= 12 and 2 <= lo <= 4 and ms > 0
    assert c.plan_stats(gb.C64, True)["tile_qubits"] == t
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    e, g = gb.grad(c, w.theta, obs, gb.C64, gb.FUSED)
    assert abs(e - e_ref) <= 1e-5 * max(1.0, abs(e_ref))
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    c2 = gb.circuit_create(w.circuit)          # same structure: served from the cache
    assert c2.autotune(w.theta, obs) == (t, lo, ms)
    assert (tmp_path / "tune.txt").read_text().count("\n") == 1
