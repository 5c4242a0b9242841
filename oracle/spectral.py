"""One-dimensional spectral building blocks of the oracle (test infrastructure).

* Chebyshev-Lobatto nodes t_a = -cos(pi a / (p-1)), a = 0..p-1 (ascending),
  the nodes of the K x K tensor leaf grids of Sec. 2 (K = 16).
* The differentiation matrix of the degree p-1 interpolant through them,
  written from the barycentric form of the Lagrange basis.
* Interpolatory quadrature weights for the p-2 interior nodes (the nodes the
  boundary panels and the leaf quadrature use), from polynomial moments.
* Lagrange basis evaluation on an arbitrary node set.
* Gauss-Legendre rules are taken from SciPy (a library primitive).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import roots_legendre


def lobatto_nodes(p: int) -> np.ndarray:
    """Ascending Chebyshev-Lobatto points on [-1, 1]."""
    return -np.cos(math.pi * np.arange(p) / (p - 1))


def barycentric_weights(t: np.ndarray) -> np.ndarray:
    """lambda_j = 1 / prod_{l != j} (t_j - t_l)."""
    n = len(t)
    lam = np.empty(n)
    for j in range(n):
        diff = t[j] - np.delete(t, j)
        lam[j] = 1.0 / np.prod(diff)
    return lam


def diff_matrix(t: np.ndarray) -> np.ndarray:
    """D[i, j] = L_j'(t_i) for the Lagrange basis on nodes t.

    Off-diagonal: (lambda_j / lambda_i) / (t_i - t_j); diagonal: minus the row sum
    (the derivative of a constant is zero).
    """
    lam = barycentric_weights(t)
    n = len(t)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (t[i] - t[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def interp_quad_weights(t: np.ndarray) -> np.ndarray:
    """Weights w with sum_j w_j f(t_j) = int_{-1}^{1} f for every polynomial of degree < len(t).

    Moments of Legendre polynomials: int P_0 = 2, int P_n = 0 for n >= 1; the
    weights solve V^T w = moments with V[j, n] = P_n(t_j) (well conditioned).
    """
    n = len(t)
    V = np.polynomial.legendre.legvander(t, n - 1)  # (n, n)
    mom = np.zeros(n)
    mom[0] = 2.0
    return np.linalg.solve(V.T, mom)


def lagrange_eval(t: np.ndarray, s: np.ndarray) -> np.ndarray:
    """L[q, j] = L_j(s_q) for the Lagrange basis on nodes t (product form)."""
    s = np.asarray(s, dtype=np.float64)
    n = len(t)
    L = np.ones((s.size, n))
    for j in range(n):
        for l in range(n):
            if l != j:
                L[:, j] *= (s.ravel() - t[l]) / (t[j] - t[l])
    return L


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [-1, 1] (SciPy)."""
    x, w = roots_legendre(n)
    return np.asarray(x), np.asarray(w)
