"""Tensor-core FP32 products of the mixed-precision path (tcgen05, split TF32).

Each operand entry is split exactly x = hi + mid + lo into three TF32 parts;
the tensor cores accumulate the six products of weight >= 2**-22 in FP32.  The
kernel is checked against a plain PyTorch float64 / complex128 product of the
same FP32 inputs, entry by entry, within the componentwise bound
|C - A B| <= gamma (|A| |B|): the three dropped products are below 3 * 2**-33
of each product, and every MMA (K = 8 of the real operand) rounds its FP32
accumulation once per term (six per k step), at most 2**-24 each.  That is
the FP32 product's own accuracy; a two-term split (22 bits per operand) fails
the bound on long k, and a wrong operand layout, sign or plane gives O(1)
errors.  Rows and columns scaled over thirty decades, and entries spread over
twelve decades inside a row, check that no entry loses its low parts (a split
into FP16 parts would).  The mixed solver (Sec. 2 merges, root system and
sweeps with FP32 factors, FP64 refinement) must give the same far field with
the tensor cores on and off.
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
    mod.hs_set_tensor_cores(2)  # every supported product on the tensor cores
    yield mod
    mod.hs_set_tensor_cores(1)


def _rand(shape, gen, cplx=True):
    re = torch.randn(shape, generator=gen, dtype=torch.float32)
    if not cplx:
        return re
    im = torch.randn(shape, generator=gen, dtype=torch.float32)
    return torch.complex(re, im)


# (batch, m, n, k): exact tiles, ragged m / n / k tails, few tiles with a long k
# (split over k pieces), the merge, root and sweep products of a 32 x 32 leaf tree
SHAPES = [
    (1, 128, 64, 64),
    (3, 200, 100, 70),
    (2, 257, 130, 129),
    (1, 1000, 512, 448),
    (4, 448, 128, 896),
    (1, 256, 64, 4100),
    (1, 1792, 128, 1792),
    (16, 196, 56, 196),
]


def _gamma(kprime):
    nacc = 6 * ((kprime + 7) // 8)
    return 2.0 ** -22 + nacc * 2.0 ** -24


def _check_bound(got, A, B, kprime):
    dt = torch.complex128 if (A.is_complex() or B.is_complex()) else torch.float64
    A64, B64 = A.cpu().to(dt), B.cpu().to(dt)
    ref = torch.matmul(A64, B64)
    absAB = torch.matmul(A64.abs(), B64.abs())
    err = (got.cpu().to(dt) - ref).abs()
    ratio = (err / absAB).max().item()
    assert ratio <= _gamma(kprime), (ratio, _gamma(kprime))
    return ratio


@pytest.mark.parametrize("batch,m,n,k", SHAPES)
@pytest.mark.parametrize("mode", [2, 1, 0])
def test_split_tf32_product_vs_torch(hs, mode, batch, m, n, k):
    gen = torch.Generator().manual_seed(1000 + 7 * mode + m + n + k)
    A = _rand((batch, m, k), gen, cplx=mode == 2)
    B = _rand((batch, k, n), gen, cplx=mode >= 1)
    out = torch.full((batch, m, n), 7.0, dtype=torch.complex64 if mode else torch.float32, device="cuda")
    used = hs.hs_gemm32(A.cuda(), B.cuda(), out)
    assert used, "the product should run on the tensor cores"
    _check_bound(out, A, B, 2 * k if mode == 2 else k)


@pytest.mark.parametrize("mode", [2, 1, 0])
def test_scaled_rows_and_columns(hs, mode):
    """Rows of A and columns of B spread over 1e-15 .. 1e15: each gets its own exponent."""
    gen = torch.Generator().manual_seed(55 + mode)
    batch, m, n, k = 2, 300, 150, 333
    A = _rand((batch, m, k), gen, cplx=mode == 2)
    B = _rand((batch, k, n), gen, cplx=mode >= 1)
    ra = 10.0 ** (30 * torch.rand((batch, m, 1), generator=gen) - 15)
    cb = 10.0 ** (30 * torch.rand((batch, 1, n), generator=gen) - 15)
    A = A * ra.to(torch.float32)
    B = B * cb.to(torch.float32)
    out = torch.empty((batch, m, n), dtype=torch.complex64 if mode else torch.float32, device="cuda")
    assert hs.hs_gemm32(A.cuda(), B.cuda(), out)
    _check_bound(out, A, B, 2 * k if mode == 2 else k)


@pytest.mark.parametrize("mode", [2, 0])
def test_entries_spread_inside_rows(hs, mode):
    """Entries of one row spread over 1e-12 .. 1: the componentwise bound holds for each."""
    gen = torch.Generator().manual_seed(77 + mode)
    batch, m, n, k = 1, 256, 128, 300
    A = _rand((batch, m, k), gen, cplx=mode == 2)
    B = _rand((batch, k, n), gen, cplx=mode >= 1)
    A = A * (10.0 ** (-12 * torch.rand((batch, m, k), generator=gen))).to(torch.float32)
    B = B * (10.0 ** (-12 * torch.rand((batch, k, n), generator=gen))).to(torch.float32)
    out = torch.empty((batch, m, n), dtype=torch.complex64 if mode else torch.float32, device="cuda")
    assert hs.hs_gemm32(A.cuda(), B.cuda(), out)
    _check_bound(out, A, B, 2 * k if mode == 2 else k)


def test_shared_right_operand(hs):
    """One B for every batch item (batch stride 0), as the leaf and sweep products use."""
    gen = torch.Generator().manual_seed(9)
    A = _rand((5, 196, 196), gen, cplx=False)
    B = _rand((1, 196, 64), gen)
    out = torch.empty((5, 196, 64), dtype=torch.complex64, device="cuda")
    assert hs.hs_gemm32(A.cuda(), B.cuda(), out, b_shared=True)
    _check_bound(out, A, B.expand(5, 196, 64), 196)


def test_tensor_cores_off_and_autotuned(hs):
    gen = torch.Generator().manual_seed(7)
    A = _rand((2, 300, 260), gen)
    B = _rand((2, 260, 96), gen)
    dA, dB = A.cuda(), B.cuda()
    o1 = torch.empty((2, 300, 96), dtype=torch.complex64, device="cuda")
    o2 = torch.empty_like(o1)
    o3 = torch.empty_like(o1)
    assert hs.hs_gemm32(dA, dB, o1)
    try:
        hs.hs_set_tensor_cores(0)
        assert not hs.hs_gemm32(dA, dB, o2)
        hs.hs_set_tensor_cores(1)
        hs.hs_gemm32(dA, dB, o3)  # either path, measured once for this shape
    finally:
        hs.hs_set_tensor_cores(2)
    for o in (o1, o2, o3):
        _check_bound(o, A, B, 520)


@pytest.mark.parametrize("batch,m,n,k", [(1, 1792, 128, 3584), (2, 700, 300, 1000), (1, 256, 64, 4100)])
def test_simt_split_k_products(hs, batch, m, n, k):
    """The SIMT FP32 products (tensor cores off) on few-tile shapes with a long k, which the
    dispatch splits over a thread-block cluster (64 x 64 and 32 x 32 tiles), within the same
    componentwise bound."""
    gen = torch.Generator().manual_seed(31 + m + k)
    A = _rand((batch, m, k), gen)
    B = _rand((batch, k, n), gen)
    out = torch.empty((batch, m, n), dtype=torch.complex64, device="cuda")
    try:
        hs.hs_set_tensor_cores(0)
        assert not hs.hs_gemm32(A.cuda(), B.cuda(), out)
    finally:
        hs.hs_set_tensor_cores(2)
    _check_bound(out, A, B, 2 * k)


def test_mixed_solve_tc_on_off(hs):
    import synth
    w = synth.WORKLOADS["grad_k20"]
    c = synth.smooth_random_coeffs(w.S, seed=5, qmax=0.3)
    al, th = synth.directions(w.M), synth.receivers(w.P)
    outs = []
    for tc in (2, 0):
        hs.hs_set_tensor_cores(tc)
        try:
            S = hs.Solver(w.n_leaf_side, w.S, w.S, w.R, precision=hs.HS_MIXED).build(c, w.k)
            outs.append(S.solve(al, th))
            it, upd, est = hs.hs_refine_stats(S.ctx)
            assert 2 <= it <= 8 and 0 <= est <= 1e-9 and upd >= 0
            S.close()
        finally:
            hs.hs_set_tensor_cores(2)
    rel = np.abs(outs[0] - outs[1]).max() / np.abs(outs[1]).max()
    assert rel < 1e-8, rel  # both within the 1e-8 mixed-precision bar of the FP64 result
