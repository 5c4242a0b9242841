"""Failure detection (the status codes of include/hs.h), all made on the host.

Nothing here faults, traps or hangs the GPU: the refinement is given a
tolerance it cannot reach in the passes it is allowed (HS_ENOCONV), the
library's next device allocation is refused by a test hook before cudaMalloc
is called (HS_ENOMEM), and the tensor-core timeout flag is set from the host
exactly as a bounded device wait that gave up would set it (HS_ETIMEOUT).
Each case then checks that the context is still usable and gives the same
answer as before.
"""
import numpy as np
import pytest

import synth
from parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod


def _problem():
    return synth.random_coeffs(4, 4, seed=12, scale=0.04), synth.directions(5), synth.receivers(7)


def test_refinement_that_cannot_converge_reports_enoconv(hs):
    c, al, th = _problem()
    s = hs.Solver(4, 4, 4, precision=hs.HS_MIXED, refine_tol=1e-300, refine_max_iter=1).build(c, 5.0)
    with pytest.raises(hs.HSError) as e:
        s.solve(al, th)
    assert e.value.code == hs.HS_ENOCONV
    assert "refinement" in str(e.value)
    s.close()
    ok = hs.Solver(4, 4, 4, precision=hs.HS_MIXED).build(c, 5.0)
    ref = hs.Solver(4, 4, 4).build(c, 5.0)
    assert rel(ok.solve(al, th), ref.solve(al, th)) < 1e-8
    ok.close()
    ref.close()


def test_refused_workspace_allocation_reports_enomem(hs):
    c, al, th = _problem()
    s = hs.Solver(4, 4, 4).build(c, 5.0)
    try:
        hs.hs_fail_next_allocs(1)
        with pytest.raises(hs.HSError) as e:
            s.solve(al, th)
        assert e.value.code == hs.HS_ENOMEM
        assert "injected" in str(e.value)
    finally:
        hs.hs_fail_next_allocs(0)
    first = s.solve(al, th)  # the context is intact: the next call allocates and solves
    assert rel(s.solve(al, th), first) == 0.0
    s.close()


def test_refused_allocation_at_create_reports_enomem(hs):
    try:
        hs.hs_fail_next_allocs(1)
        with pytest.raises(hs.HSError) as e:
            hs.Solver(2, 3, 3)
        assert e.value.code == hs.HS_ENOMEM
    finally:
        hs.hs_fail_next_allocs(0)
    c, al, th = _problem()
    s = hs.Solver(2, 4, 4).build(c, 3.0)
    assert np.all(np.isfinite(s.solve(al, th)))
    s.close()


def test_tensor_core_timeout_flag_reports_etimeout(hs):
    c, al, th = _problem()
    s = hs.Solver(4, 4, 4, precision=hs.HS_MIXED).build(c, 5.0)
    before = s.solve(al, th)
    hs.hs_raise_tc_timeout(0)
    with pytest.raises(hs.HSError) as e:
        s.solve(al, th)
    assert e.value.code == hs.HS_ETIMEOUT
    # the flag is cleared once reported: the same context solves again, unchanged
    assert rel(s.solve(al, th), before) < 1e-14
    s.close()
