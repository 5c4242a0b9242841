"""Leaf elimination through the impedance system (hs_config.leaf_impedance, FP64 contexts;
Sec. 2's HPS leaves) against the CPU oracle, whose global collocation system is the same
discrete problem solved without any leaf elimination.

The Dirichlet-block route needs A_ii nonsingular, i.e. k sqrt(1 - q) h away from the leaf's
Dirichlet eigenvalues pi sqrt(a^2 + b^2); the impedance system is solvable at every k h.  Bars:
far field 1e-10, Jacobian 1e-9 (the FP64 parity bars).  The eigenvalue cases put a leaf with
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


@pytest.mark.parametrize("nL,k", [(1, 3.0), (2, 4.0), (4, 9.3), (2, 6.0)])
def test_farfield_matches_oracle_and_dirichlet_route(hs, nL, k):
    """Regular k, including k h = 6 (beyond the leaf's first Dirichlet eigenvalue, pi sqrt(2))."""
    c = synth.random_coeffs(4, 3, seed=31, scale=0.05)
    al, th = np.linspace(0.1, 6.0, 5), np.linspace(0.2, 6.1, 9)
    u_imp = hs.Solver(nL, 4, 3, leaf_impedance=True).build(c, k).solve(al, th)
    u_dir = hs.Solver(nL, 4, 3).build(c, k).solve(al, th)
    ref, _ = F.forward_from_coeffs(c, k, nL).solve_plane(al, th)
    assert rel(u_imp, ref) < 1e-10
    assert rel(u_imp, u_dir) < 1e-10


def test_farfield_at_a_leaf_dirichlet_eigenvalue(hs):
    al, th = synth.directions(4), synth.receivers(12)
    S = hs.Solver(4, 2, 2, leaf_impedance=True, bm_eta=1.0)
    x, y = S.node_coords()
    uf = S.build_nodes(_bump(x, y), K_LEAF).solve(al, th)
    S.close()
    ref, _ = F.forward_from_function(_bump, K_LEAF, 4, eta=1.0).solve_plane(al, th)
    assert rel(uf, ref) < 1e-10


def test_jacobian_at_a_leaf_dirichlet_eigenvalue(hs):
    """The adjoint body-load operator Q from the transposed impedance system."""
    al, th = synth.directions(3), synth.receivers(5)
    c = np.zeros((3, 3))
    S = hs.Solver(4, 3, 3, leaf_impedance=True, bm_eta=1.0)
    x, y = S.node_coords()
    S.build_nodes(_bump(x, y), K_LEAF)
    J = S.jacobian(al, th)
    S.close()
    ref = F.forward_from_function(_bump, K_LEAF, 4, eta=1.0).jacobian(al, th, 3, 3)
    assert rel(J, ref) < 1e-9
