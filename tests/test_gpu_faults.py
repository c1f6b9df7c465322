"""Error paths on the GPU that leave the CUDA context usable: the allocation cap
(host-side fault injection of out-of-memory) and the argument checks of the tensor
wrappers.  Nothing here faults, traps or hangs a GPU: every failure is made on the host
before a kernel sees a bad pointer."""
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2406_19212_gb300 as gb
from paper_2406_19212_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_allocation_cap_on_gpu_keeps_context_usable():
    """With a 64 MiB cap a 20-qubit state fits and a 24-qubit one does not: sv_alloc and
    grad return ERR_OOM, and the same process then still evaluates the small case."""
    code = """
import numpy as np
import paper_2406_19212_gb300 as gb
from paper_2406_19212_gb300 import inputs as I
small = gb.sv_alloc(20)
try:
    gb.sv_alloc(24)
    print('no error')
except gb.GbvqcError as e:
    print('big', e.status)
w = I.precision_24q()
c = gb.circuit_create(w.circuit)
try:
    gb.apply_circuit(gb.sv_alloc(24), c, w.theta)
except gb.GbvqcError as e:
    print('apply', e.status)
w = I.plain_10q()
e, g = gb.grad(gb.circuit_create(w.circuit), w.theta, gb.obs_create(w.observable, 10), gb.C128, gb.PLAIN)
print('grad', np.isfinite(e) and np.all(np.isfinite(g)))
print('norm', gb.expect(small, gb.obs_create([(1.0, ())], 20)))
"""
    env = dict(os.environ, GBVQC_DEVICE_ALLOC_LIMIT=str(64 << 20))
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr
    lines = res.stdout.split("\n")
    assert "big 2" in lines and "apply 2" in lines and "grad True" in lines, res.stdout
    assert abs(float([l for l in lines if l.startswith("norm")][0].split()[1]) - 1.0) < 1e-6


def test_wrappers_reject_bad_cuda_tensors():
    import torch
    n = 6
    good = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    good[0] = 1
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    terms = [(1.0, ((0, "Z"),))]
    bad_psi = [torch.zeros(1 << (n - 1), dtype=torch.complex64, device="cuda"),       # short
               torch.zeros(2 << n, dtype=torch.complex64, device="cuda")[::2],        # strided
               torch.zeros(1 << n, dtype=torch.float32, device="cuda")]               # not complex
    for psi in bad_psi:
        for call in (lambda: gb.sv_wrap(psi, n), lambda: gb.expect_noalloc(psi, n, terms, out)):
            with pytest.raises(gb.GbvqcError) as ei:
                call()
            assert ei.value.status == 1
    for o in (torch.zeros(1, dtype=torch.float32, device="cuda"), torch.zeros(1, dtype=torch.float64),
              torch.zeros(0, dtype=torch.float64, device="cuda")):
        with pytest.raises(gb.GbvqcError) as ei:
            gb.expect_noalloc(good, n, terms, o)
        assert ei.value.status == 1
    with pytest.raises(gb.GbvqcError):
        gb.sv_wrap(good, n, is_density=True)   # a density matrix of 6 qubits needs 2^12
    gb.expect_noalloc(good, n, terms, out)       # the valid call still works
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(1.0)
