"""Pins of the oracle's LSQR (Paige and Saunders' algorithm, the solver of the
paper's Gauss-Newton subproblems, Sec. 4) against facts that do not reuse its
recurrences:

* converged, it is the least-squares solution (LAPACK lstsq), and with damping
  the Tikhonov solution of the normal equations;
* its first iterate is the exact line minimiser along A^T b,
  x_1 = (|A^T b|^2 / |A A^T b|^2) A^T b;
* its k-th iterate minimises |b - A x| over the Krylov space
  span{g, (A^T A) g, ..., (A^T A)^{k-1} g}, g = A^T b (brute force: an
  orthonormal basis of that space and a small dense least-squares solve);
* its relative-residual test is the true relative residual of the returned
  iterate, and its normal-equations test is within a factor 2 of the true one.
"""
import numpy as np

from oracle import lsqr as L


def problem(m=60, n=20, seed=0, cond=1e3):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.logspace(0, -np.log10(cond), n)
    A = U @ np.diag(s) @ V.T
    b = rng.standard_normal(m)
    return A, b


def run(A, b, tol, it, damp=0.0):
    return L.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, A.shape[1], tol, it, damp)


def test_converged_equals_lstsq():
    A, b = problem()
    x, it, _ = run(A, b, 1e-15, 500)
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x - ref) < 1e-10 * np.linalg.norm(ref)


def test_damped_equals_tikhonov_normal_equations():
    A, b = problem(seed=1)
    d = 0.05
    x, _, _ = run(A, b, 1e-15, 500, damp=d)
    ref = np.linalg.solve(A.T @ A + d * d * np.eye(A.shape[1]), A.T @ b)
    assert np.linalg.norm(x - ref) < 1e-10 * np.linalg.norm(ref)


def test_first_iterate_is_line_minimiser():
    A, b = problem(seed=2)
    x, it, _ = run(A, b, 0.0, 1)
    g = A.T @ b
    ref = (g @ g) / np.linalg.norm(A @ g) ** 2 * g
    assert it == 1
    assert np.linalg.norm(x - ref) < 1e-13 * np.linalg.norm(ref)


def test_iterates_minimise_over_krylov_spaces():
    A, b = problem(seed=3, cond=30.0)
    g = A.T @ b
    for k in (2, 3, 5):
        x, it, _ = run(A, b, 0.0, k)
        K = np.empty((A.shape[1], k))
        v = g.copy()
        for j in range(k):
            K[:, j] = v / np.linalg.norm(v)
            v = A.T @ (A @ K[:, j])
        Q, _ = np.linalg.qr(K)
        y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
        ref = Q @ y
        assert it == k
        assert np.linalg.norm(x - ref) < 1e-9 * np.linalg.norm(ref)


def test_stopping_tests_match_the_returned_iterate():
    A, b = problem(seed=4, cond=1e4)
    x, it, hist = run(A, b, 1e-3, 1000)
    r = b - A @ x
    test1 = np.linalg.norm(r) / np.linalg.norm(b)
    test2 = np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r))
    assert min(hist[-1]) <= 1e-3 and it < 1000
    assert abs(hist[-1][0] - test1) < 1e-8 * test1
    # the normal-equations test uses recurrence estimates of |A^T r| and of |A|_F (the
    # Frobenius norm of the bidiagonal so far), which drift without reorthogonalisation:
    # same order of magnitude as the true quantity, not equal
    assert 0.5 * test2 <= hist[-1][1] <= 2.0 * test2


def test_gn_step_lsqr_masks_columns():
    rng = np.random.default_rng(5)
    J = rng.standard_normal((30, 12)) + 1j * rng.standard_normal((30, 12))
    r = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    mask = np.zeros(12, bool)
    mask[[0, 3, 4, 9]] = True
    dc, _ = L.gn_step_lsqr(J, r, 1e-15, 200, mask)
    A = np.vstack([J.real[:, mask], J.imag[:, mask]])
    ref = np.linalg.lstsq(A, np.concatenate([r.real, r.imag]), rcond=None)[0]
    assert np.all(dc[~mask] == 0)
    assert np.linalg.norm(dc[mask] - ref) < 1e-10 * np.linalg.norm(ref)
