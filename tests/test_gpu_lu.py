"""Batched LU with row pivoting (shared-memory panels; tournament pivoting for
panels taller than 256 rows) and the triangular solves, through hs_lu_solve.

Checked by the normwise backward error eta = |A x - b| / (|A| |x| + |b|) of
every solution (infinity norms, evaluated in complex128 on the host), bounded
by 8 n u with u the unit roundoff of the arithmetic (2**-53 for complex128,
2**-24 for complex64): the classical bound for LU with a modest growth factor.
A wrong permutation, multiplier or update gives eta of order one.
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
    return mod


def _eta(A, X, B):
    A, X, B = (t.cpu().to(torch.complex128).numpy() for t in (A, X, B))
    worst = 0.0
    for a, x, b in zip(A, X, B):
        r = a @ x - b
        nA = np.abs(a).sum(axis=1).max()
        worst = max(worst, np.abs(r).max() / (nA * np.abs(x).max() + np.abs(b).max()))
    return worst


def _solve(hs, A, B, dtype):
    dA = A.to(dtype).cuda().contiguous()
    dB = B.to(dtype).cuda().contiguous()
    hs.hs_lu_solve(dA, dB)
    torch.cuda.synchronize()
    return dB


@pytest.mark.parametrize("dtype,u", [(torch.complex128, 2.0 ** -53), (torch.complex64, 2.0 ** -24)])
@pytest.mark.parametrize("batch,n,nrhs", [(4, 37, 3), (2, 256, 5), (3, 257, 4), (2, 600, 7), (1, 1792, 16)])
def test_lu_solve_random(hs, dtype, u, batch, n, nrhs):
    g = torch.Generator().manual_seed(n * 7 + batch)
    A = torch.complex(torch.randn(batch, n, n, generator=g, dtype=torch.float64),
                      torch.randn(batch, n, n, generator=g, dtype=torch.float64))
    B = torch.complex(torch.randn(batch, n, nrhs, generator=g, dtype=torch.float64),
                      torch.randn(batch, n, nrhs, generator=g, dtype=torch.float64))
    A, B = A.to(dtype), B.to(dtype)  # the solver's own inputs, exactly
    X = _solve(hs, A, B, dtype)
    eta = _eta(A, X, B)
    assert eta <= 8 * n * u, (eta, 8 * n * u)


@pytest.mark.parametrize("n", [200, 700])
def test_lu_needs_pivoting(hs, n):
    """Zero diagonal and tiny leading rows: without row exchanges the
    factorisation breaks down; the pivots must come from far below."""
    g = torch.Generator().manual_seed(11)
    M = torch.randn(n, n, generator=g, dtype=torch.float64) + 4 * n ** 0.5 * torch.eye(n, dtype=torch.float64)
    perm = torch.arange(n - 1, -1, -1)  # row reversal: every diagonal entry of A is off the dominant band
    A = M[perm].to(torch.complex128)
    A[: n // 2] *= 1e-6
    B = torch.randn(n, 3, generator=g, dtype=torch.float64).to(torch.complex128)
    X = _solve(hs, A[None], B[None], torch.complex128)
    assert _eta(A[None], X, B[None]) <= 8 * n * 2.0 ** -53


def test_lu_singular_reports(hs):
    n = 300
    g = torch.Generator().manual_seed(5)
    A = torch.complex(torch.randn(1, n, n, generator=g, dtype=torch.float64),
                      torch.randn(1, n, n, generator=g, dtype=torch.float64))
    A[0, :, 40] = 0  # a zero column: exactly singular
    B = torch.ones(1, n, 1, dtype=torch.complex128)
    with pytest.raises(hs.HSError) as e:
        _solve(hs, A, B, torch.complex128)
    assert e.value.code == hs.HS_ESINGULAR
