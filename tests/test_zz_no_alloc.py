"""The allocation-free far-field solve (hs_solve_noalloc).

It exists for callers whose device memory belongs to another allocator and
who therefore cannot let the library call cudaMalloc during the call.  The
test calls it twice in a row through the C ABI and checks each result
against hs_solve_dev (the solve that uses the context's own workspace) with
the far-field tolerance of the parity tests; it also checks that torch's
caching allocator reserves nothing more across the calls, that device free
memory does not move across the second call (retried once, since other
processes on a shared GPU move it too), that a request larger than the fixed
scratch is refused and that a mixed-precision context is refused.  The file
is named to be collected last.
"""
import numpy as np
import pytest

import synth
from parity import rel

pytestmark = pytest.mark.gpu

FAR_TOL = 1e-10  # far-field bar of tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod


def test_noalloc_solve_matches_solve_dev_twice(hs):
    import torch
    c = synth.random_coeffs(5, 5, seed=17, scale=0.05)
    solver = hs.Solver(4, 5, 5).build(c, 5.0)
    cases = [(synth.directions(16), synth.receivers(32)), (synth.directions(7) + 0.1, synth.receivers(9))]
    for i, (al, th) in enumerate(cases):
        a = torch.tensor(al, device="cuda")
        t = torch.tensor(th, device="cuda")
        ref = torch.zeros((len(al), len(th), 2), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(ref)
        hs.hs_solve_dev(solver.ctx, a, t, ref)
        torch.cuda.synchronize()
        reserved = torch.cuda.memory_reserved()
        for attempt in range(2):
            free_before = torch.cuda.mem_get_info()[0]
            hs.hs_solve_noalloc(solver.ctx, a, t, out)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            if i == 0 or free_after == free_before:
                break
        assert torch.cuda.memory_reserved() == reserved
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) < FAR_TOL
        if i == 1:
            # the second call (scratch address already looked up) moves no device memory
            assert free_after == free_before


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


def test_noalloc_refuses_a_mixed_precision_context(hs):
    import torch
    solver = hs.Solver(4, 3, 3, precision=hs.HS_MIXED).build(np.zeros((3, 3)), 5.0)
    a = torch.tensor(synth.directions(4), device="cuda")
    t = torch.tensor(synth.receivers(6), device="cuda")
    out = torch.zeros((4, 6, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HSError) as e:
        hs.hs_solve_noalloc(solver.ctx, a, t, out)
    assert e.value.code == hs.HS_EINVAL
    solver.close()
