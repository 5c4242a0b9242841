"""Jacobian contraction (Theorem 3.1 through the discrete adjoint of Theorem 3.2):
chunked Khatri-Rao rows projected on the sine basis.

Bars: against the oracle's column-by-column Frechet solves 1e-9 (relative
2-norm, as the other Jacobian parity test); chunkings of the same product
agree to 1e-13; at the k = 20 gradient workload (no CPU oracle in seconds at
that size) the Jacobian satisfies Re J^H (F - data) = hs_gradient to 1e-10
and matches central differences of the far field (h = 1e-5: truncation
~h^2 |F'''|, rounding ~1e-16 / h) to 1e-6 on seeded columns.
"""
import numpy as np
import pytest

import synth
from parity import rel
from oracle import forward as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    yield mod
    mod.hs_set_contract_budget(0)




def test_ragged_chunks_match_oracle(hs):
    """4 x 4 leaves, 5 x 4 modes, 4 x 6 data: a budget of 7 pairs gives chunks 7, 7, 7, 3."""
    S1, S2, k, nL = 5, 4, 5.0, 4
    c = synth.random_coeffs(S1, S2, seed=51, scale=0.05)
    al, th = synth.directions(4), synth.receivers(6)
    nX = 14 * nL
    per_pair = 16 * (nX * nX + nX * S1)
    S = hs.Solver(nL, S1, S2).build(c, k)
    hs.hs_set_contract_budget(7 * per_pair)
    J7 = S.jacobian(al, th)
    hs.hs_set_contract_budget(1 * per_pair)
    J1 = S.jacobian(al, th)
    hs.hs_set_contract_budget(0)
    Jall = S.jacobian(al, th)
    S.close()
    Jo = F.forward_from_coeffs(c, k, nL).jacobian(al, th, S1, S2)
    assert rel(J7, Jo) < 1e-9
    assert rel(J7, Jall) < 1e-13
    assert rel(J1, Jall) < 1e-13


def test_full_size_k20_adjoint_identity_and_differences(hs):
    """k = 20 gradient workload (16 x 16 leaves, 40 x 40 modes, 64 x 128 data; 8 chunks at the
    default budget): the explicit Jacobian against the gradient kernel and against differences."""
    w = synth.WORKLOADS["grad_k20"]
    c0 = synth.project_sine(synth.ellipse_phantom(3), w.S, w.S)
    al, th = synth.directions(w.M), synth.receivers(w.P)
    rng = np.random.default_rng(45)
    data = 0.05 * (rng.standard_normal((w.M, w.P)) + 1j * rng.standard_normal((w.M, w.P)))
    S = hs.Solver(w.n_leaf_side, w.S, w.S, w.R).build(c0, w.k)
    J = S.jacobian(al, th)
    Fc = S.solve(al, th)
    g, _ = S.gradient(data, al, th)
    gJ = (J.conj().T @ (Fc - data).ravel()).real
    assert rel(gJ, g.ravel()) < 1e-10
    h = 1e-5
    for m in np.random.default_rng(46).choice(w.S * w.S, size=3, replace=False):
        cp, cm = c0.copy(), c0.copy()
        cp.flat[m] += h
        cm.flat[m] -= h
        fd = (S.build(cp, w.k).solve(al, th) - S.build(cm, w.k).solve(al, th)).ravel() / (2 * h)
        assert rel(J[:, m], fd) < 1e-6
    S.close()
