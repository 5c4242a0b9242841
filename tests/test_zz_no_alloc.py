"""The allocation-free far-field solve (hs_solve_noalloc).

It exists for callers whose device memory belongs to another allocator and
who therefore cannot let the library call cudaMalloc during the call.  The
test calls it twice in a row through the C ABI and checks each result
against hs_solve_dev (the solve that uses the context's own workspace) with
the far-field tolerance of the parity tests; it also checks that device free
memory does not move across the second call and that a request larger than
the fixed scratch is refused.  The file is named to be collected last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FAR_TOL = 1e-10  # far-field bar of tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_solve_matches_solve_dev_twice(hs):
    import torch
    c = synth.random_coeffs(5, 5, seed=17, scale=0.05)
    solver = hs.Solver(4, 5, 5).build(c, 5.0)
    cases = [(synth.directions(16), synth.receivers(32)), (synth.directions(7) + 0.1, synth.receivers(9))]
    free_after = []
    for al, th in cases:
        a = torch.tensor(al, device="cuda")
        t = torch.tensor(th, device="cuda")
        ref = torch.zeros((len(al), len(th), 2), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(ref)
        hs.hs_solve_dev(solver.ctx, a, t, ref)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        hs.hs_solve_noalloc(solver.ctx, a, t, out)
        torch.cuda.synchronize()
        free_after.append((free_before, torch.cuda.mem_get_info()[0]))
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < FAR_TOL
    # the second call (scratch address already looked up) leaves free memory unchanged
    assert free_after[1][0] == free_after[1][1]


def test_noalloc_rejects_requests_beyond_the_scratch(hs):
    import torch
    solver = hs.Solver(32, 2, 2).build(np.zeros((2, 2)), 10.0)
    # 16 * (56*32) * (6*128 + 2*256) bytes > 16 MiB
    a = torch.zeros(128, dtype=torch.float64, device="cuda")
    t = torch.zeros(256, dtype=torch.float64, device="cuda")
    out = torch.zeros((128, 256, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HSError) as e:
        hs.hs_solve_noalloc(solver.ctx, a, t, out)
    assert e.value.code == hs.HS_EINVAL
    assert "scratch" in str(e.value)
