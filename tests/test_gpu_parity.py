"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Floating-point bars (relative 2-norm unless stated):
  * far field, FP64 path:                 1e-10 (the stated FP64 target);
  * interior fields:                      1e-9  (collocation rounding, cond ~1e6);
  * Jacobian (discrete adjoint vs the oracle's column-by-column Frechet solves): 1e-9;
  * Gauss-Newton coefficients:            1e-7  (the stated target);
  * misfit gradient:                      1e-9.
"""
import math

import numpy as np
import pytest

import closed_forms as CF
import synth
from parity import rel
from oracle import forward as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod




def test_forward_gaussian_bumps_k5(hs):
    """Data workload of the k = 5 Gauss-Newton step: 4 x 4 leaves, 16 directions, 32 receivers."""
    w = synth.WORKLOADS["gn_k5"]
    qt = synth.gaussian_bumps(1)
    al, th = synth.directions(w.M), synth.receivers(w.P)
    S = hs.Solver(w.n_leaf_side, 2, 2, w.R)
    x, y = S.node_coords()
    S.build_nodes(qt(x, y), w.k)
    uf = S.solve(al, th)
    ref, _ = F.forward_from_function(qt, w.k, w.n_leaf_side, w.R).solve_plane(al, th)
    assert rel(uf, ref) < 1e-10


@pytest.mark.parametrize("nL,k,S1,S2,M,P", [(1, 3.0, 3, 2, 3, 5), (2, 4.0, 4, 3, 2, 9), (8, 9.3, 7, 5, 5, 7)])
def test_forward_sine_series_ragged(hs, nL, k, S1, S2, M, P):
    c = synth.random_coeffs(S1, S2, seed=11, scale=0.05)
    al = np.linspace(0.1, 6.0, M)
    th = np.linspace(0.2, 6.1, P)
    uf = hs.Solver(nL, S1, S2).build(c, k).solve(al, th)
    ref, _ = F.forward_from_coeffs(c, k, nL).solve_plane(al, th)
    assert rel(uf, ref) < 1e-10


def test_fields_match_oracle(hs):
    import torch
    c = synth.random_coeffs(4, 4, seed=12, scale=0.05)
    k, nL = 5.0, 4
    al = synth.directions(3)
    S = hs.Solver(nL, 4, 4).build(c, k)
    u = torch.empty((3, nL * nL, 256, 2), dtype=torch.float64, device="cuda")
    hs.hs_fields_dev(S.ctx, torch.tensor(al, device="cuda"), u)
    torch.cuda.synchronize()
    ug = u.cpu().numpy()
    ug = (ug[..., 0] + 1j * ug[..., 1]).reshape(3, nL * nL, 16, 16)
    _, uo = F.forward_from_coeffs(c, k, nL).solve_plane(al, synth.receivers(4))
    m = np.ones((16, 16), bool)
    m[0, 0] = m[0, -1] = m[-1, 0] = m[-1, -1] = False
    assert rel(ug[:, :, m], uo[:, :, m]) < 1e-9
    assert np.all(ug[:, :, ~m] == 0)


def test_zero_contrast_full_size(hs):
    """q = 0 scatters nothing, at the k = 40 benchmark size (32 x 32 leaves, 128 x 256 data)."""
    w = synth.WORKLOADS["fwd_k40"]
    S = hs.Solver(w.n_leaf_side, 4, 4, w.R).build(np.zeros((4, 4)), w.k)
    uf = S.solve(synth.directions(w.M), synth.receivers(w.P))
    assert np.abs(uf).max() < 1e-9


def test_radial_gaussian_full_size_matches_ode(hs):
    """Radially symmetric contrast at the k = 40 benchmark size against the separated-variables reference."""
    w = synth.WORKLOADS["fwd_k40"]
    sig, q0 = 0.15, 0.3
    S = hs.Solver(w.n_leaf_side, 2, 2, w.R)
    x, y = S.node_coords()
    S.build_nodes(q0 * np.exp(-(x * x + y * y) / (2 * sig * sig)), w.k)
    th = synth.receivers(w.P)
    al = np.array([0.0, 1.3])
    uf = S.solve(al, th)
    for i, a in enumerate(al):
        ref = CF.radial_scattered(w.k, lambda r: q0 * math.exp(-r * r / (2 * sig * sig)), 1.0, a, th, w.R,
                                  nmax=75)
        assert rel(uf[i], ref) < 1e-8


def test_solve_dev_matches_host(hs):
    import torch
    c = synth.random_coeffs(3, 3, seed=13, scale=0.05)
    S = hs.Solver(4, 3, 3).build(c, 6.0)
    al, th = synth.directions(5), synth.receivers(7)
    host = S.solve(al, th)
    out = torch.empty((5, 7, 2), dtype=torch.float64, device="cuda")
    hs.hs_solve_dev(S.ctx, torch.tensor(al, device="cuda"), torch.tensor(th, device="cuda"), out)
    torch.cuda.synchronize()
    dev = out.cpu().numpy()
    assert np.array_equal(dev[..., 0] + 1j * dev[..., 1], host)


def test_jacobian_matches_frechet_columns(hs):
    S1 = S2 = 5
    k, nL = 5.0, 4
    c = synth.random_coeffs(S1, S2, seed=5, scale=0.05)
    al, th = synth.directions(4), synth.receivers(6)
    J = hs.Solver(nL, S1, S2).build(c, k).jacobian(al, th)
    Jo = F.forward_from_coeffs(c, k, nL).jacobian(al, th, S1, S2)
    assert rel(J, Jo) < 1e-9


def test_gn_step_k5_matches_oracle(hs):
    """One Gauss-Newton step of the k = 5 workload from q = 0 (eq. normaleq, lambda_rel = 1e-4)."""
    w = synth.WORKLOADS["gn_k5"]
    qt = synth.gaussian_bumps(1)
    al, th = synth.directions(w.M), synth.receivers(w.P)
    data, _ = F.forward_from_function(qt, w.k, w.n_leaf_side, w.R).solve_plane(al, th)
    c0 = np.zeros((w.S, w.S))
    lam_rel = 1e-4
    S = hs.Solver(w.n_leaf_side, w.S, w.S, w.R).build(c0, w.k)
    c1, rn = S.gn_step(data, al, th, lam_rel, c0)
    fw0 = F.forward_from_coeffs(c0, w.k, w.n_leaf_side, w.R)
    J = fw0.jacobian(al, th, w.S, w.S)
    F0, _ = fw0.solve_plane(al, th)
    r = (data - F0).ravel()
    A = (J.conj().T @ J).real
    lam = lam_rel * np.trace(A) / A.shape[0]
    ref = F.gn_step(J, r, lam)
    assert abs(rn - np.linalg.norm(r)) < 1e-10 * np.linalg.norm(r)
    assert rel(c1.ravel(), ref) < 1e-7


def test_gradient_matches_oracle(hs):
    S1 = S2 = 4
    k, nL = 5.0, 4
    c = synth.random_coeffs(S1, S2, seed=21, scale=0.04)
    al, th = synth.directions(3), synth.receivers(5)
    qt = synth.gaussian_bumps(2)
    data, _ = F.forward_from_function(qt, k, nL).solve_plane(al, th)
    g, mis = hs.Solver(nL, S1, S2).build(c, k).gradient(data, al, th)
    fw = F.forward_from_coeffs(c, k, nL)
    Fc, _ = fw.solve_plane(al, th)
    J = fw.jacobian(al, th, S1, S2)
    gref = F.misfit_gradient(J, Fc.ravel(), data.ravel())
    assert rel(g.ravel(), gref) < 1e-9
    assert abs(mis - 0.5 * np.linalg.norm(Fc - data) ** 2) < 1e-10 * mis


def test_error_paths(hs):
    S = hs.Solver(2, 2, 2)
    with pytest.raises(hs.HSError) as e:
        S.solve([0.0], [0.0])
    assert e.value.code == hs.HS_ENOTBUILT
    with pytest.raises(hs.HSError) as e:
        S.build(np.full((2, 2), 5.0), 3.0)  # 1 - q <= 0 somewhere
    assert e.value.code == hs.HS_EINVAL
    with pytest.raises(hs.HSError) as e:
        S.build(np.full((2, 2), np.nan), 3.0)
    assert e.value.code == hs.HS_EINVAL
    S.build(np.zeros((2, 2)), 3.0)
    assert S.launch_count() > 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_degenerate_one_of_everything(hs, prec):
    """1 x 1 leaf, one sine mode, one incidence, one receiver, low frequency: far field, Jacobian,
    gradient and both Gauss-Newton steps against the oracle, on FP64 and mixed contexts (the mixed
    adjoint is refined on a tree without merge levels)."""
    k, nL = 0.7, 1
    c = np.array([[0.05]])
    al, th = np.array([0.3]), np.array([2.0])
    fw = F.forward_from_coeffs(c, k, nL)
    ref, _ = fw.solve_plane(al, th)
    S = hs.Solver(nL, 1, 1, 3.0, hs.HS_FP64 if prec == "fp64" else hs.HS_MIXED).build(c, k)
    assert rel(S.solve(al, th), ref) < (1e-10 if prec == "fp64" else 1e-8)
    J = S.jacobian(al, th)
    Jo = fw.jacobian(al, th, 1, 1)
    assert rel(J, Jo) < 1e-9
    data = ref * 1.1
    g, _ = S.gradient(data, al, th)
    assert rel(g.ravel(), F.misfit_gradient(Jo, ref.ravel(), data.ravel())) < 1e-9
    c1, _ = S.gn_step(data, al, th, 0.0, c)
    dc_ref = F.gn_step(Jo, (data - ref).ravel(), 0.0)
    assert rel(c1.ravel() - c.ravel(), dc_ref) < 1e-7
    c2, _, it = S.gn_step_lsqr(data, al, th, c, tol=1e-12, max_iter=5)
    assert it == 1 and rel(c2.ravel() - c.ravel(), dc_ref) < 1e-7  # one unknown: one iteration is exact
    if prec == "mixed":  # the explicit FP32 Jacobian in the LSQR products: FP32 accuracy
        c3, _, it = S.gn_step_lsqr(data, al, th, c, tol=1e-12, max_iter=5, products=hs.HS_MIXED)
        assert it == 1 and rel(c3.ravel() - c.ravel(), dc_ref) < 1e-4
    S.close()
