"""Tensor-core complex FP32 GEMM (tcgen05, 3xTF32) of the mixed-precision path.

The kernel is checked against a plain PyTorch complex128 product of the same
FP32 inputs, entry by entry, within a componentwise bound
|C - A B| <= gamma (|A| |B|): the split x = hi + lo into two TF32 parts leaves
a relative error of at most 2**-22 per operand and drops the lo*lo product
(together below 2**-20 per product), and the FP32 accumulation in tensor
memory rounds once per MMA (K = 8 reals) and per split term, at most 2**-23
each.  A wrong operand layout or sign gives O(1) errors.  The mixed solver
(Sec. 2 merges, root system and sweeps with FP32 factors, FP64 refinement)
must give the same far field with the tensor cores on and off.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    yield mod
    mod.hs_set_tensor_cores(True)


def _rand(shape, gen):
    re = torch.randn(shape, generator=gen, dtype=torch.float32)
    im = torch.randn(shape, generator=gen, dtype=torch.float32)
    return torch.complex(re, im)


# (batch, m, n, k): exact tiles, ragged m/n/k tails, the shapes of the merge
# and sweep products of a 32 x 32 leaf tree (k = ne = 64 .. 1792)
SHAPES = [
    (1, 128, 64, 64),
    (3, 200, 100, 70),
    (2, 257, 130, 129),
    (1, 1000, 512, 448),
    (4, 448, 128, 896),
    (1, 256, 64, 4100),  # many chunks through the copy ring, ragged k, split over a cluster
]


def _gamma(k):
    nacc = 3 * ((2 * k + 7) // 8)
    return 2.0 ** -20 + nacc * 2.0 ** -23


def _check_bound(got, A, B, k):
    A64, B64 = A.cpu().to(torch.complex128), B.cpu().to(torch.complex128)
    ref = torch.matmul(A64, B64)
    absAB = torch.matmul(A64.abs(), B64.abs())
    ratio = ((got.cpu().to(torch.complex128) - ref).abs() / absAB).max().item()
    assert ratio <= _gamma(k), (ratio, _gamma(k))
    return ratio


@pytest.mark.parametrize("batch,m,n,k", SHAPES)
def test_cgemm_tc_vs_torch(hs, batch, m, n, k):
    gen = torch.Generator().manual_seed(1000 + m + n + k)
    A = _rand((batch, m, k), gen)
    B = _rand((batch, k, n), gen)
    out = torch.full((batch, m, n), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    used = hs.hs_cgemm32(A.cuda(), B.cuda(), out)
    assert used, "shape should be eligible for the tensor-core kernel"
    _check_bound(out, A, B, k)


def test_cgemm_tc_matches_simt(hs):
    gen = torch.Generator().manual_seed(7)
    A = _rand((2, 300, 260), gen)
    B = _rand((2, 260, 96), gen)
    dA, dB = A.cuda(), B.cuda()
    o1 = torch.empty((2, 300, 96), dtype=torch.complex64, device="cuda")
    o2 = torch.empty_like(o1)
    assert hs.hs_cgemm32(dA, dB, o1)
    hs.hs_set_tensor_cores(False)
    try:
        assert not hs.hs_cgemm32(dA, dB, o2)
    finally:
        hs.hs_set_tensor_cores(True)
    _check_bound(o1, A, B, 260)
    _check_bound(o2, A, B, 260)


def test_small_shapes_not_eligible(hs):
    gen = torch.Generator().manual_seed(3)
    A = _rand((1, 100, 64), gen).cuda()
    B = _rand((1, 64, 64), gen).cuda()
    out = torch.empty((1, 100, 64), dtype=torch.complex64, device="cuda")
    assert not hs.hs_cgemm32(A, B, out)
    _check_bound(out, A, B, 64)


def test_mixed_solve_tc_on_off(hs):
    import synth
    w = synth.WORKLOADS["grad_k20"]
    c = synth.smooth_random_coeffs(w.S, seed=5, qmax=0.3)
    al, th = synth.directions(w.M), synth.receivers(w.P)
    outs = []
    for tc in (True, False):
        hs.hs_set_tensor_cores(tc)
        try:
            S = hs.Solver(w.n_leaf_side, w.S, w.S, w.R, precision=hs.HS_MIXED).build(c, w.k)
            outs.append(S.solve(al, th))
            it, upd, est = hs.hs_refine_stats(S.ctx)
            assert 2 <= it <= 8 and 0 <= est <= 1e-9 and upd >= 0
        finally:
            hs.hs_set_tensor_cores(True)
    rel = np.abs(outs[0] - outs[1]).max() / np.abs(outs[1]).max()
    assert rel < 1e-8, rel  # both within the 1e-8 mixed-precision bar of the FP64 result
