"""Combined-field exterior rows (hs_config.bm_eta > 0; Sec. 2, Remark, read with the
Burton-Miller combination, alpha = i eta / k) on the GPU against the CPU oracle's same rows.

Bars as in the other parity tests: far field 1e-10 on FP64 contexts and 1e-8 on mixed ones
(FP32 factors, FP64 refinement), Jacobian 1e-9.  At k^2 = (pi/2)^2 (a^2 + b^2), a Dirichlet
eigenvalue of the square [-1, 1]^2, Green's identity alone is singular; with the combined rows
both paths give the radial contrast's far field within 1e-8 of its separated-variables ODE
reference, and the mixed refinement converges there.
"""
import math

import numpy as np
import pytest

import closed_forms as CF
import synth
from parity import rel
from oracle import forward as F

pytestmark = pytest.mark.gpu

K_EIG = 0.5 * math.pi * math.sqrt(5.0)  # (a, b) = (1, 2)


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod


def _radial(sig=0.15, q0=0.3):
    return (lambda x, y: q0 * np.exp(-(x * x + y * y) / (2 * sig * sig)),
            lambda r: q0 * math.exp(-r * r / (2 * sig * sig)))


@pytest.mark.parametrize("nL,k", [(2, 4.0), (4, 5.0), (4, K_EIG), (8, 2 * K_EIG)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_farfield_matches_oracle(hs, nL, k, prec):
    c = synth.random_coeffs(4, 3, seed=21, scale=0.05)
    al, th = np.linspace(0.1, 6.0, 5), np.linspace(0.2, 6.1, 9)
    p = hs.HS_FP64 if prec == "fp64" else hs.HS_MIXED
    S = hs.Solver(nL, 4, 3, precision=p, bm_eta=1.0).build(c, k)
    uf = S.solve(al, th)
    S.close()
    ref, _ = F.forward_from_coeffs(c, k, nL, eta=1.0).solve_plane(al, th)
    assert rel(uf, ref) < (1e-10 if prec == "fp64" else 1e-8)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_radial_contrast_at_a_dirichlet_eigenvalue(hs, prec):
    qxy, qr = _radial()
    alpha = np.array([0.3])
    th = synth.receivers(12)
    ref = CF.radial_scattered(K_EIG, qr, 1.0, 0.3, th, 3.0, nmax=30)
    p = hs.HS_FP64 if prec == "fp64" else hs.HS_MIXED
    S = hs.Solver(8, 2, 2, precision=p, bm_eta=1.0)
    x, y = S.node_coords()
    uf = S.build_nodes(qxy(x, y), K_EIG).solve(alpha, th)
    if prec == "mixed":
        it, _, est = hs.hs_refine_stats(S.ctx)
        assert it <= 5 and est <= 1e-9
    S.close()
    assert rel(uf[0], ref) < 1e-8


def test_green_and_combined_rows_agree_off_resonance(hs):
    """At a regular k both exterior forms describe the same radiating field: far fields within
    the discretisation error of the combined rows' normal-derivative identity."""
    c = synth.random_coeffs(4, 4, seed=5, scale=0.05)
    al, th = synth.directions(4), synth.receivers(8)
    u0 = hs.Solver(8, 4, 4).build(c, 9.3).solve(al, th)
    u1 = hs.Solver(8, 4, 4, bm_eta=1.0).build(c, 9.3).solve(al, th)
    assert rel(u1, u0) < 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_jacobian_matches_oracle(hs, prec):
    """Discrete adjoint through the transposed combined rows (FP64 root solve, or the refined
    adjoint's transposed exterior residual on mixed contexts) against the oracle's
    column-by-column Frechet solves, at the Dirichlet eigenvalue."""
    c = synth.random_coeffs(3, 3, seed=8, scale=0.05)
    al, th = synth.directions(3), synth.receivers(5)
    p = hs.HS_FP64 if prec == "fp64" else hs.HS_MIXED
    S = hs.Solver(4, 3, 3, precision=p, bm_eta=1.0).build(c, K_EIG)
    J = S.jacobian(al, th)
    S.close()
    ref = F.forward_from_coeffs(c, K_EIG, 4, eta=1.0).jacobian(al, th, 3, 3)
    assert rel(J, ref) < 1e-9
