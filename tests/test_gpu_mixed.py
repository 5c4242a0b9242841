"""Mixed precision: FP32 factors and sweeps, FP64 iterative refinement.

The bar (the stated mixed-precision target): far field within 1e-8 (relative
2-norm) of the FP64 result, against both the FP64 GPU path and the CPU oracle.
"""
import numpy as np
import pytest

import synth
from parity import rel
from oracle import forward as F

pytestmark = pytest.mark.gpu
MIXED_TOL = 1e-8


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod




def test_mixed_gaussian_bumps_k5_vs_oracle(hs):
    w = synth.WORKLOADS["gn_k5"]
    qt = synth.gaussian_bumps(1)
    al, th = synth.directions(w.M), synth.receivers(w.P)
    S = hs.Solver(w.n_leaf_side, 2, 2, w.R, precision=hs.HS_MIXED)
    x, y = S.node_coords()
    S.build_nodes(qt(x, y), w.k)
    uf = S.solve(al, th)
    it, upd, est = hs.hs_refine_stats(S.ctx)
    ref, _ = F.forward_from_function(qt, w.k, w.n_leaf_side, w.R).solve_plane(al, th)
    assert rel(uf, ref) < MIXED_TOL
    assert 2 <= it <= 8 and 0 <= est <= 1e-9 and upd >= 0


@pytest.mark.parametrize("nL,k,M,P", [(1, 3.0, 3, 5), (2, 4.0, 2, 9), (8, 9.3, 5, 7)])
def test_mixed_matches_fp64_ragged(hs, nL, k, M, P):
    c = synth.random_coeffs(5, 4, seed=31, scale=0.05)
    al, th = np.linspace(0.1, 6.0, M), np.linspace(0.2, 6.1, P)
    u64 = hs.Solver(nL, 5, 4).build(c, k).solve(al, th)
    u32 = hs.Solver(nL, 5, 4, precision=hs.HS_MIXED).build(c, k).solve(al, th)
    assert rel(u32, u64) < MIXED_TOL


def test_mixed_full_size_k40_matches_fp64(hs):
    """The benchmark workload: k = 40, 32 x 32 leaves, 128 incidences, 256 receivers."""
    w = synth.WORKLOADS["fwd_k40"]
    c = synth.smooth_random_coeffs(w.S, seed=2, qmax=0.3)
    al, th = synth.directions(w.M), synth.receivers(w.P)
    u64 = hs.Solver(w.n_leaf_side, w.S, w.S, w.R).build(c, w.k).solve(al, th)
    S = hs.Solver(w.n_leaf_side, w.S, w.S, w.R, precision=hs.HS_MIXED).build(c, w.k)
    u32 = S.solve(al, th)
    assert rel(u32, u64) < MIXED_TOL


def test_mixed_fields_match_fp64(hs):
    import torch
    c = synth.random_coeffs(4, 4, seed=32, scale=0.05)
    k, nL, M = 6.0, 4, 3
    al = torch.tensor(synth.directions(M), device="cuda")
    out = []
    for prec in (hs.HS_FP64, hs.HS_MIXED):
        S = hs.Solver(nL, 4, 4, precision=prec).build(c, k)
        u = torch.zeros((M, nL * nL, 256, 2), dtype=torch.float64, device="cuda")
        hs.hs_fields_dev(S.ctx, al, u)
        torch.cuda.synchronize()
        out.append(u.cpu().numpy())
    assert rel(out[1], out[0]) < MIXED_TOL


def test_forward_dev_both_precisions(hs):
    """hs_forward_dev returns the far field of hs_solve and the fields of hs_fields_dev in one call."""
    import torch
    c = synth.random_coeffs(4, 4, seed=33, scale=0.05)
    k, nL, M, P = 5.5, 4, 4, 6
    al_np, th_np = synth.directions(M), synth.receivers(P)
    al, th = torch.tensor(al_np, device="cuda"), torch.tensor(th_np, device="cuda")
    res = {}
    for prec in (hs.HS_FP64, hs.HS_MIXED):
        S = hs.Solver(nL, 4, 4, precision=prec).build(c, k)
        uf = torch.zeros((M, P, 2), dtype=torch.float64, device="cuda")
        u = torch.zeros((M, nL * nL, 256, 2), dtype=torch.float64, device="cuda")
        hs.hs_forward_dev(S.ctx, al, th, uf, u)
        u2 = torch.zeros_like(u)
        hs.hs_fields_dev(S.ctx, al, u2)
        torch.cuda.synchronize()
        ufn = uf.cpu().numpy()
        res[prec] = (ufn[..., 0] + 1j * ufn[..., 1], u.cpu().numpy())
        assert rel(res[prec][0], S.solve(al_np, th_np)) < 1e-12
        assert rel(res[prec][1], u2.cpu().numpy()) < 1e-12
    ref, _ = F.forward_from_coeffs(c, k, nL).solve_plane(al_np, th_np)
    assert rel(res[hs.HS_FP64][0], ref) < 1e-10
    assert rel(res[hs.HS_MIXED][0], ref) < MIXED_TOL


def test_mixed_gn_step_k5_matches_oracle(hs):
    """The direct Gauss-Newton step of the k = 5 workload (eq. normaleq, lambda_rel = 1e-4) on a
    mixed-precision context: refined far field, refined forward and adjoint fields, FP64
    contraction and normal equations; the step within 1e-7 of the oracle's."""
    w = synth.WORKLOADS["gn_k5"]
    al, th = synth.directions(w.M), synth.receivers(w.P)
    data, _ = F.forward_from_function(synth.gaussian_bumps(1), w.k, w.n_leaf_side, w.R).solve_plane(al, th)
    c0 = np.zeros((w.S, w.S))
    S = hs.Solver(w.n_leaf_side, w.S, w.S, w.R, hs.HS_MIXED).build(c0, w.k)
    c1, rn = S.gn_step(data, al, th, 1e-4, c0)
    it, upd, est = hs.hs_adjoint_refine_stats(S.ctx)
    S.close()
    fw0 = F.forward_from_coeffs(c0, w.k, w.n_leaf_side, w.R)
    J = fw0.jacobian(al, th, w.S, w.S)
    F0, _ = fw0.solve_plane(al, th)
    r = (data - F0).ravel()
    A = (J.conj().T @ J).real
    ref = F.gn_step(J, r, 1e-4 * np.trace(A) / A.shape[0])
    assert abs(rn - np.linalg.norm(r)) < 1e-9 * np.linalg.norm(r)
    assert rel(c1.ravel(), ref) < 1e-7
    assert 2 <= it <= 8 and 0 <= est <= 1e-9


def test_factor_graph_replay_bitwise(hs):
    """Every build after a context's first replays one captured CUDA graph of the
    factorisation (the kernels read k from device memory), at the same k and at a new
    one: the far fields must be bitwise identical to the launch-by-launch builds, and
    the launch count per build the same."""
    w = synth.WORKLOADS["grad_k20"]
    c = synth.smooth_random_coeffs(w.S, seed=4, qmax=0.3)
    al, th = synth.directions(16), synth.receivers(24)
    outs, counts = [], []
    for graphs in (False, True):
        hs.hs_set_graphs(graphs)
        try:
            S = hs.Solver(w.n_leaf_side, w.S, w.S, w.R, precision=hs.HS_MIXED)
            for _ in range(3):  # first build eager (new k), then capture, then replay
                n0 = S.launch_count()
                S.build(c, w.k)
                counts.append(S.launch_count() - n0)
            outs.append(S.solve(al, th))
            S.build(0.5 * c, w.k)  # a different contrast through the same graph
            outs.append(S.solve(al, th))
            S.build(c, w.k + 1.5)  # a new frequency through the same graphs
            outs.append(S.solve(al, th))
            S.close()
        finally:
            hs.hs_set_graphs(True)
    assert all(np.array_equal(outs[i], outs[i + 3]) for i in range(3))
    assert counts[1] == counts[4] and counts[2] == counts[5]
    assert not np.array_equal(outs[0], outs[1]) and not np.array_equal(outs[0], outs[2])


def test_mixed_gradient_k20(hs):
    """Misfit gradient on a mixed-precision context (refined forward and adjoint fields) against
    the FP64 context at the k = 20 gradient workload: misfit to 1e-8 (the refined far field),
    gradient to 1e-9 (the bar of the FP64 gradient against the oracle)."""
    w = synth.WORKLOADS["grad_k20"]
    c = synth.project_sine(synth.ellipse_phantom(3), w.S, w.S)
    rng = np.random.default_rng(44)
    data = 0.05 * (rng.standard_normal((w.M, w.P)) + 1j * rng.standard_normal((w.M, w.P)))
    al, th = synth.directions(w.M), synth.receivers(w.P)
    out = {}
    for prec in (hs.HS_FP64, hs.HS_MIXED):
        S = hs.Solver(w.n_leaf_side, w.S, w.S, w.R, prec).build(c, w.k)
        out[prec] = S.gradient(data, al, th)
        S.close()
    (g64, m64), (g32, m32) = out[hs.HS_FP64], out[hs.HS_MIXED]
    assert abs(m32 - m64) < 1e-8 * m64
    assert rel(g32, g64) < 1e-9


@pytest.mark.parametrize("case", ["k5", "k20"])
def test_mixed_jacobian(hs, case):
    """Explicit Jacobian on a mixed-precision context (refined forward and adjoint fields, FP64
    contraction) against the FP64 context and, at k = 5, against the oracle's Frechet columns:
    bar 1e-9, the FP64 Jacobian's."""
    if case == "k5":
        nL, S, k, M, P = 4, 6, 5.0, 8, 12
        c = synth.random_coeffs(S, S, seed=5, scale=0.05)
    else:
        w = synth.WORKLOADS["grad_k20"]
        nL, S, k, M, P = w.n_leaf_side, 16, w.k, 32, 48
        c = synth.project_sine(synth.ellipse_phantom(3), S, S)
    al, th = synth.directions(M), synth.receivers(P)
    J = {}
    for prec in (hs.HS_FP64, hs.HS_MIXED):
        Sv = hs.Solver(nL, S, S, 3.0, prec).build(c, k)
        J[prec] = Sv.jacobian(al, th)
        if prec == hs.HS_MIXED:
            it, upd, est = hs.hs_adjoint_refine_stats(Sv.ctx)
            assert 2 <= it <= 8 and 0 <= est <= 1e-9
        Sv.close()
    assert rel(J[hs.HS_MIXED], J[hs.HS_FP64]) < 1e-9
    if case == "k5":
        Jo = F.forward_from_coeffs(c, k, nL).jacobian(al, th, S, S)
        assert rel(J[hs.HS_MIXED], Jo) < 1e-9
