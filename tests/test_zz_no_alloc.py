"""GPU test of expect_noalloc, the expectation entry point that allocates nothing.

It serves callers that cannot allocate device memory (inside CUDA-graph stream capture,
or under a framework that owns the memory budget).  The test calls it through the C ABI
on caller-owned CUDA tensors and checks it against the handle-based `expect`, within
the tolerances of the other parity tests, on two calls in a row (the fixed scratch
array is reused, so the second call must see a clean counter), checks that the library
makes no device allocation during those calls (its allocation counter is unchanged), and
checks that inputs beyond its stated maximum are rejected with an error.
"""
import numpy as np
import pytest

import paper_2406_19212_gb300 as gb
from paper_2406_19212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,n", [(gb.C64, 16), (gb.C128, 16), (gb.C64, 9), (gb.C128, 21)])
def test_expect_noalloc_matches_expect(dtype, n):
    import torch
    tdt = torch.complex64 if dtype == gb.C64 else torch.complex128
    psi = torch.tensor(I.random_state(n, 41 + n), dtype=tdt, device="cuda")
    terms = I.ising_chain(n, np.linspace(-1, 1, n)) + I.heisenberg_1d(min(n, 6), 0.3, -0.7) + \
        [(0.25, tuple((q, "Y") for q in range(0, n, 3)))]
    assert len(terms) <= 64
    sv = gb.sv_wrap(psi, n)
    ref = gb.expect(sv, gb.obs_create(terms, n))
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        before = gb.mem_info()
        gb.expect_noalloc(psi, n, terms, out)
        torch.cuda.synchronize()
        assert gb.mem_info() == before   # the library made no device allocation
        got = float(out.item())
        if dtype == gb.C64:
            assert abs(got - ref) <= 1e-5 * max(1.0, abs(ref))
        else:
            assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref))
    sv.free()


def test_expect_noalloc_rejects_oversize():
    import torch
    psi = torch.zeros(1 << 4, dtype=torch.complex64, device="cuda")
    psi[0] = 1
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbvqcError) as ei:
        gb.expect_noalloc(psi, 4, [(1.0, ((0, "Z"),))] * 65, out)
    assert ei.value.status == 1 and "64" in str(ei.value)
    with pytest.raises(gb.GbvqcError):
        gb.expect_noalloc(psi, 4, [(1.0, ((5, "Z"),))], out)
