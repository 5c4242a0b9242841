"""LSQR for the linearized least-squares problem (test infrastructure only).

The paper solves each Gauss-Newton subproblem (Sec. 3.3, eq. normaleq) with
LSQR (Paige and Saunders, ACM TOMS 8 (1982), Algorithm LSQR) stopped at a
tolerance of 1e-3 (Sec. 4, Table 2).  This is a plain restatement of that
published algorithm -- Golub-Kahan bidiagonalisation of A started from b,
with the plane rotations that update the iterate -- over explicit callables
for A v and A^T u, in NumPy FP64.

Stopping rule (the paper names the tolerance only; reading): stop after
iteration k when the relative residual ||b - A x_k|| / ||b|| or the relative
normal-equations residual ||A^T (b - A x_k)|| / (||A||_F ||b - A x_k||) is at
most tol, with the norms replaced by LSQR's own recurrence estimates
(||A||_F accumulated from the bidiagonal entries), or after max_iter
iterations.  With damp > 0 the problem is min ||A x - b||^2 + damp^2 ||x||^2.

Only tests/, the smoke entry and the benchmark's CPU baseline may use this
module.
"""
from __future__ import annotations

import math

import numpy as np


def lsqr(matvec, rmatvec, b: np.ndarray, n: int, tol: float, max_iter: int, damp: float = 0.0):
    """Returns (x, iterations, history) with history[k] = (relative residual, normal-equations test)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n)
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return x, 0, []
    u = b / beta
    v = np.asarray(rmatvec(u), dtype=np.float64)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return x, 0, []
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    beta1 = beta
    anorm2 = 0.0
    res2 = 0.0  # the damp part of the residual norm
    history = []
    it = 0
    while it < max_iter:
        it += 1
        # bidiagonalisation: beta u = A v - alpha u, alpha v = A^T u - beta v
        u = np.asarray(matvec(v), dtype=np.float64) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0.0:
            u = u / beta
        anorm2 += alpha * alpha + beta * beta + damp * damp
        v = np.asarray(rmatvec(u), dtype=np.float64) - beta * v
        alpha = float(np.linalg.norm(v))
        if alpha > 0.0:
            v = v / alpha
        # rotation eliminating the damping term, then the one eliminating beta
        rhobar1 = math.hypot(rhobar, damp)
        c1, s1 = rhobar / rhobar1, damp / rhobar1
        psi = s1 * phibar
        phibar = c1 * phibar
        rho = math.hypot(rhobar1, beta)
        c, s = rhobar1 / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        # iterate and search direction
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        res2 += psi * psi
        rnorm = math.sqrt(phibar * phibar + res2)
        arnorm = alpha * abs(c) * abs(phibar)
        test1 = rnorm / beta1
        test2 = arnorm / (math.sqrt(anorm2) * rnorm) if rnorm > 0.0 else 0.0
        history.append((test1, test2))
        if test1 <= tol or test2 <= tol or alpha == 0.0 or beta == 0.0:
            break
    return x, it, history


def gn_step_lsqr(J: np.ndarray, resid: np.ndarray, tol: float, max_iter: int, mask=None, damp: float = 0.0):
    """Gauss-Newton step in the real coefficients (eq. normaleq read as a least-squares
    problem): min over real dc supported on `mask` of ||J dc - r||, i.e. LSQR on
    A = [Re J; Im J] (columns in mask), b = [Re r; Im r].  Returns (dc, iterations)."""
    J = np.asarray(J)
    nm = J.shape[1]
    cols = np.arange(nm) if mask is None else np.flatnonzero(np.ravel(mask))
    A = np.vstack([J.real[:, cols], J.imag[:, cols]])
    b = np.concatenate([np.real(resid), np.imag(resid)]).ravel()
    y, it, _ = lsqr(lambda v: A @ v, lambda u: A.T @ u, b, len(cols), tol, max_iter, damp)
    dc = np.zeros(nm)
    dc[cols] = y
    return dc, it
