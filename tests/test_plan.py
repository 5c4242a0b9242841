"""Frequency plans of the sweep driver (host logic, no GPU)."""
import math

import numpy as np

from paper_1608_06871_gb300 import sweep as SW


def dirichlet_eigenvalues(kmax):
    """sqrt(a^2 + b^2), a, b >= 1, of the square [-pi/2, pi/2]^2 (brute force)."""
    n = int(kmax) + 2
    return np.array(sorted({math.hypot(a, b) for a in range(1, n) for b in range(1, n) if math.hypot(a, b) <= kmax}))


def test_paper_grid_is_moved_off_the_square_resonances():
    ks = 1.0 + np.arange(0, 277) / 4.0  # k = 1, 1.25, ..., 70
    ev = dirichlet_eigenvalues(71.0)
    moved = [k for k in ks if SW.square_safe(k) != k]
    assert moved[:7] == [5.0, 10.0, 13.0, 15.0, 17.0, 18.25, 20.0]  # 18.25: 0.0017 from sqrt(333)
    on = [k for k in ks if np.abs(ev - k).min() < 1e-12]
    assert set(on) <= set(moved)  # every exact hit is moved (and the near ones)
    for k in ks:
        ks_ = SW.square_safe(k)
        assert abs(ks_ - k) <= 0.02
        assert np.abs(ev - ks_).min() >= 0.002, k


def test_plan_paper_counts():
    """Table 2's columns: Modes = S(S-1)/2 with S = floor(2k), M = floor(2k), M*P = 8 k^2 at integer k."""
    for k, modes, m, mp in ((1, 1, 2, 8), (2, 6, 4, 32), (4, 28, 8, 128), (8, 120, 16, 512), (16, 496, 32, 2048),
                            (32, 2016, 64, 8192), (64, 8128, 128, 32768)):
        p = SW.plan_paper(float(k))
        assert int(p.mask().sum()) == modes and p.M == m and p.M * p.P == mp
        assert abs(p.R - 40.0 / math.pi) < 1e-12


def test_plan_c5_top_and_resonances():
    p = SW.plan_c5(70.0)
    assert (p.leaves_per_side, p.S, p.M, p.P) == (128, 140, 280, 280)
    ks = np.arange(1.0, 70.0 + 1e-9, 0.25)
    ev = (math.pi / 2) * dirichlet_eigenvalues(46.0)
    for k in ks:
        pk = SW.plan_c5(float(k))
        assert abs(pk.k - k) <= 0.02 and np.abs(ev - pk.k).min() >= 0.002, k
    assert SW.plan_c5(40.75).k != 40.75


def test_example1_contrast_is_outside_the_sine_band_near_the_boundary():
    """Example 1 (Sec. 4) under the sign reading of its contrast, q = -1.5 exp(-|x|^2/50) on
    [-pi/2, pi/2]^2: q is -1.5 .. -1.36 over the whole square and does not vanish on its
    boundary, where every sine mode does.  So even the best L2 approximation in the paper's
    final basis (k = 14.25: m1 + m2 <= 28, 378 modes) stays a sizable fraction of ||q|| away,
    and a reconstruction in that basis cannot converge to q the way the paper's smooth
    examples do; Example 2's contrast, which decays inside the square, is approximated to
    well under 1% by the same basis."""
    import math

    import numpy as np

    import synth
    from paper_1608_06871_gb300 import sweep as SW
    p = SW.plan_paper(14.25)
    g = (np.arange(512) + 0.5) / 256.0 - 1.0
    X, Y = np.meshgrid(g, g, indexing="ij")
    bx = np.sin(np.outer(np.arange(1, p.S + 1), g + 1.0) * (math.pi / 2.0))
    cell = (math.pi / 512.0) ** 2
    out = {}
    for which in (1, 2):
        q = synth.paper_example(which)
        best = synth.project_sine(q, p.S, p.S, nq=512) * p.mask()
        err = math.sqrt(np.sum((bx.T @ best @ bx - q(X, Y)) ** 2) * cell)
        out[which] = err / math.sqrt(np.sum(q(X, Y) ** 2) * cell)
    assert int(p.mask().sum()) == 378
    assert out[1] > 0.1
    assert out[2] < 0.01


def test_combined_field_plans_keep_the_paper_frequencies():
    """With combined-field exterior rows (bm_eta > 0) the plans keep the resonant frequencies:
    k = 5 on the paper's domain is pi k / 2 on [-1, 1]^2, where 5 = sqrt(3^2 + 4^2)."""
    p = SW.plan_paper(5.0, avoid_resonance=False)
    assert p.k == math.pi * 5.0 / 2.0 and SW.plan_paper(5.0).k != p.k
    assert SW.plan_c5(40.75, avoid_resonance=False).k == 40.75
