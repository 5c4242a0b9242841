"""Leaf elimination through the impedance system (hs_config.leaf_impedance; Sec. 2's HPS
leaves) on FP64 and mixed contexts against the CPU oracle, whose global collocation system is
the same discrete problem solved without any leaf elimination.

The Dirichlet-block route needs A_ii nonsingular, i.e. k sqrt(1 - q) h away from the leaf's
Dirichlet eigenvalues pi sqrt(a^2 + b^2); the impedance system is solvable at every k h.  Bars:
far field 1e-10 (FP64) and 1e-8 (mixed: FP32 factors, FP64 refinement, whose particular solves
and transposed leaf rows then use the impedance system's particular-solution operator),
Jacobian 1e-9.  The eigenvalue cases put a leaf with
q ~ 0 (a narrow radial bump elsewhere) exactly at its lowest Dirichlet eigenvalue, which on the
4 x 4 tree is also a Dirichlet eigenvalue of the whole square, so they use the combined-field
exterior rows (bm_eta = 1) as well.
"""
import math

import numpy as np
import pytest

import synth
from parity import rel
from oracle import forward as F

pytestmark = pytest.mark.gpu

K_LEAF = math.pi * math.sqrt(2.0) / 0.5  # (1, 1) Dirichlet eigenvalue of a leaf of side 0.5 (4 x 4 leaves)


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod


def _bump(x, y, sig=0.15, q0=0.3):
    return q0 * np.exp(-(x * x + y * y) / (2 * sig * sig))


def _prec(hs, prec):
    return (hs.HS_FP64, 1e-10) if prec == "fp64" else (hs.HS_MIXED, 1e-8)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nL,k", [(1, 3.0), (2, 4.0), (4, 9.3), (2, 6.0)])
def test_farfield_matches_oracle_and_dirichlet_route(hs, nL, k, prec):
    """Regular k, including k h = 6 (beyond the leaf's first Dirichlet eigenvalue, pi sqrt(2))."""
    p, bar = _prec(hs, prec)
    c = synth.random_coeffs(4, 3, seed=31, scale=0.05)
    al, th = np.linspace(0.1, 6.0, 5), np.linspace(0.2, 6.1, 9)
    u_imp = hs.Solver(nL, 4, 3, precision=p, leaf_impedance=True).build(c, k).solve(al, th)
    u_dir = hs.Solver(nL, 4, 3, precision=p).build(c, k).solve(al, th)
    ref, _ = F.forward_from_coeffs(c, k, nL).solve_plane(al, th)
    assert rel(u_imp, ref) < bar
    assert rel(u_imp, u_dir) < bar


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_farfield_at_a_leaf_dirichlet_eigenvalue(hs, prec):
    p, bar = _prec(hs, prec)
    al, th = synth.directions(4), synth.receivers(12)
    S = hs.Solver(4, 2, 2, precision=p, leaf_impedance=True, bm_eta=1.0)
    x, y = S.node_coords()
    uf = S.build_nodes(_bump(x, y), K_LEAF).solve(al, th)
    if prec == "mixed":
        it, _, est = hs.hs_refine_stats(S.ctx)
        assert it <= 5 and est <= 1e-9
    S.close()
    ref, _ = F.forward_from_function(_bump, K_LEAF, 4, eta=1.0).solve_plane(al, th)
    assert rel(uf, ref) < bar


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_jacobian_at_a_leaf_dirichlet_eigenvalue(hs, prec):
    """FP64: the adjoint body-load operator Q from the transposed impedance system; mixed: the
    refined adjoint's transposed leaf solve P^T."""
    p, _ = _prec(hs, prec)
    al, th = synth.directions(3), synth.receivers(5)
    S = hs.Solver(4, 3, 3, precision=p, leaf_impedance=True, bm_eta=1.0)
    x, y = S.node_coords()
    S.build_nodes(_bump(x, y), K_LEAF)
    J = S.jacobian(al, th)
    S.close()
    ref = F.forward_from_function(_bump, K_LEAF, 4, eta=1.0).jacobian(al, th, 3, 3)
    assert rel(J, ref) < 1e-9
