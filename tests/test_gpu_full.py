"""Full-size parity at the benchmark configurations, in the launch configuration the
benchmark uses (fused tile passes, CUDA-graph replay).

- 20-qubit VQE (800 parameters): energy and gradient vs the oracle's Algorithm 2,
  plus central finite differences (h = 1e-5) of the complex128 energy.
- 24-qubit grid random circuit: amplitudes vs the oracle.
- 28-qubit grid random circuit: complex64 vs complex128 fidelity >= 1 - 1e-6,
  complex128 fused vs per-gate agreement, Porter-Thomas second moment.
- 13-qubit noisy density matrix (26 vectorised qubits): complex64 vs complex128,
  trace = 1, parameter-shift spot checks (exact for the noisy loss).
- 32-qubit GHZ state (2^32 amplitudes, 32 GiB): closed form at the largest size.
"""
import math

import numpy as np
import pytest

import paper_2406_19212_gb300 as gb
from oracle import oracle as O
from paper_2406_19212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_vqe20_full_gradient():
    w = I.diff_20q()
    e_ref, g_ref = O.adjoint_grad(w.circuit, w.theta, w.observable)
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 20)
    gmax = np.abs(g_ref).max()
    for dtype, mode in ((gb.C64, gb.FUSED), (gb.C64, gb.PLAIN), (gb.C128, gb.FUSED), (gb.C128, gb.PLAIN)):
        for _ in range(2):  # second call replays the captured graph
            e, g = gb.grad(c, w.theta, obs, dtype, mode)
            if dtype == gb.C64:
                assert abs(e - e_ref) <= 1e-5 * max(1.0, abs(e_ref))
                assert np.abs(g - g_ref).max() <= 1e-4 * gmax
            else:
                assert abs(e - e_ref) <= 1e-10
                assert np.abs(g - g_ref).max() <= 1e-10
    e, g = gb.grad(c, w.theta, obs, gb.C128, gb.FUSED)
    for j in w.extra["fd_indices"]:
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[j] += 1e-5
        tm[j] -= 1e-5
        ep = gb.grad(c, tp, obs, gb.C128, gb.FUSED)[0]
        em = gb.grad(c, tm, obs, gb.C128, gb.FUSED)[0]
        assert abs((ep - em) / 2e-5 - g[j]) < 1e-7


def test_rqc24_matches_oracle():
    w = I.precision_24q()
    ref = O.apply_circuit(w.circuit, w.theta)
    c = gb.circuit_create(w.circuit)
    for dtype, mode in ((gb.C128, gb.FUSED), (gb.C128, gb.PLAIN), (gb.C64, gb.FUSED)):
        sv = gb.sv_alloc(24, dtype)
        gb.apply_circuit(sv, c, (), mode)
        got = gb.sv_get(sv).astype(np.complex128)
        sv.free()
        if dtype == gb.C128:
            assert np.abs(got - ref).max() <= 1e-12
        else:
            f = abs(np.vdot(got, ref)) ** 2 / np.vdot(got, got).real
            assert f >= 1 - 1e-6
            assert np.abs(got - ref).max() <= 2e-5


def test_rqc28_precision():
    import torch
    w = I.precision_28q()
    c = gb.circuit_create(w.circuit)
    n = 28
    s64 = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    s128 = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    s64[0] = 1
    s128[0] = 1
    sv64, sv128 = gb.sv_wrap(s64, n), gb.sv_wrap(s128, n)
    gb.apply_circuit(sv64, c, (), gb.FUSED)
    gb.apply_circuit(sv128, c, (), gb.FUSED)
    torch.cuda.synchronize()
    norm = torch.vdot(s128, s128).real.item()
    assert abs(norm - 1) < 1e-12
    a = s64.to(torch.complex128)
    n64 = torch.vdot(a, a).real.item()
    fid = abs(torch.vdot(a, s128).item()) ** 2 / (n64 * norm)
    print(f"28q complex64: fidelity {fid:.10f}, norm drift {n64 - 1:.3e}")
    assert fid >= 1 - 1e-6          # fidelity of the normalised states
    assert abs(n64 - 1) <= 1e-4     # FP32-rounded matrices are unitary to ~1e-7 each
    pt = (2 ** n) * torch.sum(torch.abs(s128) ** 4).item()
    assert 1.8 < pt < 2.2  # Porter-Thomas: 2^n sum |psi|^4 -> 2 for random circuits
    sv64.free()
    del s64
    plain = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    plain[0] = 1
    svp = gb.sv_wrap(plain, n)
    gb.apply_circuit(svp, c, (), gb.PLAIN)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(plain - s128)).item() <= 1e-12
    svp.free()
    sv128.free()


def test_noisy13_full():
    w = I.noisy_13q()
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 13)
    e128, g128 = gb.grad(c, w.theta, obs, gb.C128, gb.PLAIN)
    e128f, g128f = gb.grad(c, w.theta, obs, gb.C128, gb.FUSED)
    e64, g64 = gb.grad(c, w.theta, obs, gb.C64, gb.FUSED)
    gmax = np.abs(g128).max()
    assert abs(e128f - e128) <= 1e-10 and np.abs(g128f - g128).max() <= 1e-10 * max(1, gmax)
    assert abs(e64 - e128) <= 1e-5 * max(1.0, abs(e128))
    assert np.abs(g64 - g128).max() <= 1e-4 * gmax
    # parameter shift of the complex128 energy (exact for U(theta) (x) conj U(theta))
    for j in (0, 155, 311):
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[j] += math.pi / 2
        tm[j] -= math.pi / 2
        ep = gb.grad(c, tp, obs, gb.C128, gb.FUSED)[0]
        em = gb.grad(c, tm, obs, gb.C128, gb.FUSED)[0]
        assert abs(0.5 * (ep - em) - g128[j]) <= 1e-10
    sv = gb.sv_alloc(13, gb.C128, True)
    gb.apply_circuit(sv, c, w.theta, gb.FUSED)
    assert abs(gb.expect(sv, gb.obs_create([(1.0, ())], 13)) - 1.0) < 1e-12
    assert abs(gb.expect(sv, obs) - e128) < 1e-10


def test_ghz32_largest_state():
    import torch
    n = 32
    ops = [I.Op("H", (0,))] + [I.Op("CNOT", (i, i + 1)) for i in range(n - 1)]
    c = gb.circuit_create(I.Circuit(n, ops, 0))
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    st[0] = 1
    sv = gb.sv_wrap(st, n)
    gb.apply_circuit(sv, c, (), gb.FUSED)
    torch.cuda.synchronize()
    r = 1 / math.sqrt(2)
    assert abs(st[0].item() - r) < 1e-6 and abs(st[-1].item() - r) < 1e-6
    assert abs(torch.sum(torch.abs(st) ** 2).item() - 1) < 1e-5
    assert torch.count_nonzero(st).item() == 2
    sv.free()
