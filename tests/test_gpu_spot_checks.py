"""Oracle spot checks of the two recursive-linearization sweeps at the low
frequencies the CPU oracle reaches (the k = 1..40 plan and the paper-scale
k = 1..70 plan; above k ~ 20 the oracle's dense exterior block does not fit in
seconds, so those frequencies are checked against the FP64 GPU path instead).

At each checked frequency the plan's own tree, contrast and angles are used,
and the far fields of every 16th incidence (0, 16, 32, ...) on all receivers
are compared with the oracle's: 1e-10 for the FP64 path, 1e-8 for the
mixed-precision path.
"""
import math

import numpy as np
import pytest

import synth
from oracle import forward as F
from parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod


def _check(hs, p, qfun):
    al_all = 2 * np.pi * np.arange(p.M) / p.M
    al, th = al_all[::16], 2 * np.pi * np.arange(p.P) / p.P
    ref, _ = F.forward_from_function(qfun, p.k, p.leaves_per_side, p.R).solve_plane(al, th)
    for prec, bar in ((hs.HS_FP64, 1e-10), (hs.HS_MIXED, 1e-8)):
        s = hs.Solver(p.leaves_per_side, 2, 2, p.R, prec)
        x, y = s.node_coords()
        s.build_nodes(qfun(x, y), p.k)
        assert rel(s.solve(al, th), ref) < bar, (p.k, prec)
        s.close()


@pytest.mark.parametrize("k", [1.0, 5.0, 10.0])
def test_sweep_k40_plan_low_frequencies_match_oracle(hs, k):
    """plan_ceil: S = ceil(1.6k), M = P = ceil(4k), 4 x 4 leaves up to k = 5, 8 x 8 at k = 10;
    blurred-ellipse phantom of seed 7."""
    from paper_1608_06871_gb300 import sweep as SW
    _check(hs, SW.plan_ceil(k), synth.ellipse_phantom(7))


@pytest.mark.parametrize("k", [1.0, 2.5])
def test_paper_scale_plan_low_frequencies_match_oracle(hs, k):
    """plan_c5: S = floor(2k), M = P = ceil(4k), 4 x 4 leaves at k = 1, 8 x 8 at k = 2.5;
    the 40-inclusion contrast of seed 5 scaled to max |q| = 0.5 on the 140 x 140 modes."""
    from paper_1608_06871_gb300 import sweep as SW
    qfun = synth.inclusions(5)
    c_top = synth.scaled_sine_coeffs(qfun, 140, 0.5)
    scale = c_top[0, 0] / synth.project_sine(qfun, 1, 1, nq=640)[0, 0]
    _check(hs, SW.plan_c5(k), lambda x, y: scale * qfun(x, y))
