"""The emulated FP64 product on the tensor cores (csrc/ozaki.cu): exact BF16
slices of the scaled rows of A and columns of B, exact FP32 accumulation of
the slice products per anti-diagonal, exact integer recombination.

Checked entry by entry against the FP64 product within the FP64 GEMM's own
error bound 2 k u |A| |B| (u = 2^-53), on ragged shapes (partial tiles in
m, n and k), batches, k longer than one launch (split and accumulated in
FP64), rows and columns of very different magnitudes (the per-row and
per-column scaling), exact zeros, and integer inputs whose products reach
the largest partial sums the exact accumulation allows.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def hs():
    from paper_1608_06871_gb300.build import build
    build()
    import paper_1608_06871_gb300 as mod
    return mod


def _check(hs, A, B, factor=2.0):
    C = torch.empty((A.shape[0], A.shape[1], B.shape[2]), dtype=torch.float64, device="cuda")
    hs.hs_dgemm_emulated(A, B, C)
    torch.cuda.synchronize()
    ref = torch.bmm(A, B)
    bound = factor * A.shape[2] * U * torch.bmm(A.abs(), B.abs())
    err = (C - ref).abs()
    worst = float((err / bound.clamp_min(1e-300)).max())
    assert bool((err <= bound).all()), worst
    return worst


@pytest.mark.parametrize("batch,m,n,k", [(1, 128, 64, 32), (1, 300, 70, 448), (3, 129, 65, 33), (2, 256, 128, 1000),
                                         (1, 200, 64, 3584)])
def test_random_products_within_fp64_bound(hs, batch, m, n, k):
    g = torch.Generator(device="cuda").manual_seed(batch * 1000 + m + n + k)
    A = torch.randn((batch, m, k), dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn((batch, k, n), dtype=torch.float64, device="cuda", generator=g)
    _check(hs, A, B)


def test_scaled_rows_columns_and_zeros(hs):
    g = torch.Generator(device="cuda").manual_seed(7)
    m, n, k = 256, 128, 448
    A = torch.randn((1, m, k), dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn((1, k, n), dtype=torch.float64, device="cuda", generator=g)
    A *= torch.logspace(-200, 200, m, base=2.0, dtype=torch.float64, device="cuda")[None, :, None]
    B *= torch.logspace(150, -150, n, base=2.0, dtype=torch.float64, device="cuda")[None, None, :]
    A[0, 5, :] = 0.0
    B[0, :, 7] = 0.0
    A[0, 9, ::3] = 0.0
    _check(hs, A, B)


def test_largest_exact_partial_sums(hs):
    """Entries whose first slice is the extreme integer +-128 on every row and column, k = 384
    (the longest single launch) and k = 1632 (five pieces): the top diagonal's partial sums
    reach 384 * 128^2; the product must still be exact up to the FP64 roundings."""
    for k in (384, 1632):
        _extreme(hs, k)


def _extreme(hs, k):
    m, n = 128, 64
    rng = np.random.default_rng(3)
    sgn_a = rng.choice([-1.0, 1.0], size=(m, k))
    sgn_b = rng.choice([-1.0, 1.0], size=(k, n))
    A = torch.tensor(sgn_a * (1.0 - 2.0 ** -30), device="cuda")[None]
    B = torch.tensor(sgn_b * (1.0 - 2.0 ** -30), device="cuda")[None]
    A[0, :, 0] = 1.0 - 2.0 ** -52  # rows and columns scale to values just below 1
    B[0, 0, :] = 1.0 - 2.0 ** -52
    C = torch.empty((1, m, n), dtype=torch.float64, device="cuda")
    hs.hs_dgemm_emulated(A, B, C)
    torch.cuda.synchronize()
    exact = np.einsum("ik,kj->ij", A[0].cpu().numpy().astype(np.longdouble), B[0].cpu().numpy().astype(np.longdouble))
    err = np.abs(C[0].cpu().numpy().astype(np.longdouble) - exact)
    assert float(np.max(err / (k * U * np.abs(exact).max()))) < 1.0


def _emulation(hs, on):
    hs.hs_set_fp64_emulation(on)


def test_jacobian_with_and_without_emulation(hs):
    """The Jacobian contraction (k = 20, 16 x 16 leaves, 16 x 16 modes) with the emulated products
    and with the FP64 SIMT GEMMs agrees to rounding."""
    import synth
    from parity import rel
    c = synth.project_sine(synth.ellipse_phantom(3), 16, 16)
    al, th = synth.directions(24), synth.receivers(32)
    out = []
    for on in (True, False):
        _emulation(hs, on)
        try:
            s = hs.Solver(16, 16, 16).build(c, 20.0)
            out.append(s.jacobian(al, th))
            s.close()
        finally:
            _emulation(hs, True)
    assert rel(out[0], out[1]) < 1e-12


def test_lsqr_and_mixed_solve_with_and_without_emulation(hs):
    """LSQR with FP64 products (explicit emulated J vs. products from the fields) at equal
    iteration counts, and the mixed-precision forward solve (emulated vs. SIMT exterior residual
    and far field), at k = 5 on 4 x 4 leaves."""
    import synth
    from parity import rel
    from oracle import forward as F
    al, th = synth.directions(8), synth.receivers(12)
    data, _ = F.forward_from_function(synth.gaussian_bumps(1), 5.0, 4).solve_plane(al, th)
    c = synth.random_coeffs(6, 6, seed=4, scale=0.02)
    steps, fars = [], []
    for on in (True, False):
        _emulation(hs, on)
        try:
            s = hs.Solver(4, 6, 6).build(c, 5.0)
            steps.append(s.gn_step_lsqr(data, al, th, c, tol=0.0, max_iter=8)[0] - c)
            s.close()
            m = hs.Solver(4, 6, 6, precision=hs.HS_MIXED).build(c, 5.0)
            fars.append(m.solve(al, th))
            m.close()
        finally:
            _emulation(hs, True)
    assert rel(steps[0], steps[1]) < 1e-9
    assert rel(fars[0], fars[1]) < 1e-10
