"""Boundary of Omega: panels, layer potentials and the field on the receiver circle.

Test infrastructure only.  Follows Sec. 2 (Remark): the scattered field
outside Omega satisfies Green's representation u_s = D u_s - S d_n u_s with

    S phi(x) = int G(x, y) phi(y) ds_y,
    D phi(x) = int d/dn_y G(x, y) phi(y) ds_y,
    G(x, y)  = (i/4) H_0^(1)(k |x - y|),

and, on the boundary, the jump relations give (D - I/2) u_s = S d_n u_s.  The
same representation evaluated at x_p = R (cos theta_p, sin theta_p) gives the
measured field u_far(theta_p) of Sec. 1 (eq. farfielddef).

Discretisation (a reading: the paper gives none): the boundary panels are the
leaf edges lying on the boundary; each carries the 14 interior
Chebyshev-Lobatto nodes of its leaf edge.  Densities are represented by their
degree-13 interpolant on each panel.  Entries for a target and a source panel
closer than one panel length use product integration of the exact kernel
against the Lagrange basis (dyadically graded Gauss-Legendre toward the
nearest point, which resolves the logarithmic singularity); all other pairs
use the interpolatory rule on the panel nodes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.special import hankel1

from .spectral import gauss_legendre, interp_quad_weights, lagrange_eval, lobatto_nodes

P_LEAF = 16            # Chebyshev-Lobatto points per leaf side
GRADE_LEVELS = 56      # dyadic levels toward the nearest point (2^-56 ~ 1.4e-17)
GRADE_GL = 16          # Gauss-Legendre points per graded interval


@dataclass
class Boundary:
    """Panel geometry of the boundary of [-1,1]^2 for n_L leaves per side."""

    n_leaf: int
    h: float
    t: np.ndarray        # (14,) panel nodes on [-1,1]
    wq: np.ndarray       # (14,) interpolatory weights on [-1,1]
    start: np.ndarray    # (n_panels, 2)
    tangent: np.ndarray  # (n_panels, 2)
    normal: np.ndarray   # (n_panels, 2) outward
    nodes: np.ndarray    # (n_panels*14, 2)
    node_normal: np.ndarray
    node_weight: np.ndarray  # ds weights: wq * h / 2
    panel_of: np.ndarray     # (n_panels*14,) panel index


def make_boundary(n_leaf: int) -> Boundary:
    h = 2.0 / n_leaf
    t = lobatto_nodes(P_LEAF)[1:-1]
    wq = interp_quad_weights(t)
    starts, tans, norms = [], [], []
    for i in range(n_leaf):  # south side y = -1, left to right
        starts.append((-1.0 + i * h, -1.0)); tans.append((1.0, 0.0)); norms.append((0.0, -1.0))
    for i in range(n_leaf):  # east side x = 1, bottom to top
        starts.append((1.0, -1.0 + i * h)); tans.append((0.0, 1.0)); norms.append((1.0, 0.0))
    for i in range(n_leaf):  # north side y = 1, left to right
        starts.append((-1.0 + i * h, 1.0)); tans.append((1.0, 0.0)); norms.append((0.0, 1.0))
    for i in range(n_leaf):  # west side x = -1, bottom to top
        starts.append((-1.0, -1.0 + i * h)); tans.append((0.0, 1.0)); norms.append((-1.0, 0.0))
    start = np.array(starts)
    tangent = np.array(tans)
    normal = np.array(norms)
    s = (t + 1.0) * h / 2.0
    nodes = (start[:, None, :] + s[None, :, None] * tangent[:, None, :]).reshape(-1, 2)
    node_normal = np.repeat(normal, len(t), axis=0)
    node_weight = np.tile(wq * h / 2.0, len(start))
    panel_of = np.repeat(np.arange(len(start)), len(t))
    return Boundary(n_leaf, h, t, wq, start, tangent, normal, nodes, node_normal,
                    node_weight, panel_of)


def green(k: float, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """G(x, y) = (i/4) H_0^(1)(k |x - y|) (Sec. 1, below eq. inteqscat)."""
    r = np.linalg.norm(x - y, axis=-1)
    return 0.25j * hankel1(0, k * r)


def green_dny(k: float, x: np.ndarray, y: np.ndarray, ny: np.ndarray) -> np.ndarray:
    """d/dn_y G(x, y) = (i k / 4) H_1^(1)(k r) (x - y).n_y / r, r = |x - y|."""
    d = x - y
    r = np.linalg.norm(d, axis=-1)
    return 0.25j * k * hankel1(1, k * r) * np.sum(d * ny, axis=-1) / r


def _segment_distance(a0, a1, b0, b1) -> float:
    """Distance between two axis-aligned segments (sampled exactly at endpoints)."""
    def pt_seg(p, s0, s1):
        d = s1 - s0
        u = np.clip(np.dot(p - s0, d) / np.dot(d, d), 0.0, 1.0)
        return np.linalg.norm(p - (s0 + u * d))
    return min(pt_seg(a0, b0, b1), pt_seg(a1, b0, b1), pt_seg(b0, a0, a1), pt_seg(b1, a0, a1))


def near_panels(bd: Boundary) -> list[list[int]]:
    """For each panel, the panels at distance <= one panel length (itself included)."""
    n = len(bd.start)
    ends = bd.start + bd.h * bd.tangent
    out = []
    for p in range(n):
        row = []
        for q in range(n):
            if _segment_distance(bd.start[p], ends[p], bd.start[q], ends[q]) <= bd.h * (1 + 1e-9):
                row.append(q)
        out.append(row)
    return out


def _graded_rule(h: float, s_star: float):
    """Offsets sigma (from s_star) and weights on [0, h], dyadically graded toward s_star.

    Offsets are generated directly (never as s - s_star) so that |x - y| stays
    exact down to the finest level.
    """
    xg, wg = gauss_legendre(GRADE_GL)
    offs, weights = [], []
    for d in (-s_star, h - s_star):
        if d == 0.0:
            continue
        edges = [d * 2.0 ** (-j) for j in range(GRADE_LEVELS + 1)] + [0.0]
        for lo, hi in zip(edges[1:], edges[:-1]):
            mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
            offs.append(mid + half * xg)
            weights.append(np.abs(half) * wg)
    return np.concatenate(offs), np.concatenate(weights)


def product_weights(bd: Boundary, k: float, x: np.ndarray, q: int):
    """int_panel K(x, y(s)) L_j(s) ds for K = G and K = dG/dn_y, j over the panel nodes."""
    y0, tau, ny = bd.start[q], bd.tangent[q], bd.normal[q]
    s_star = float(np.clip(np.dot(x - y0, tau), 0.0, bd.h))
    sig, w = _graded_rule(bd.h, s_star)
    perp = x - (y0 + s_star * tau)                  # x - y(s_star)
    dvec = perp[None, :] - sig[:, None] * tau[None, :]  # x - y(s_star + sigma)
    r = np.sqrt(np.sum(dvec * dvec, axis=-1))
    L = lagrange_eval(bd.t, 2.0 * (s_star + sig) / bd.h - 1.0)  # (nq, 14)
    g = 0.25j * hankel1(0, k * r) * w
    dg = 0.25j * k * hankel1(1, k * r) * (dvec @ ny) / r * w
    return g @ L, dg @ L


def layer_matrices(bd: Boundary, k: float):
    """Nystrom matrices S, D (N_b x N_b) on the boundary nodes (Sec. 2, Remark)."""
    X = bd.nodes
    n = len(X)
    S = green(k, X[:, None, :], X[None, :, :]) * bd.node_weight[None, :]
    Dm = green_dny(k, X[:, None, :], X[None, :, :], bd.node_normal[None, :, :]) * bd.node_weight[None, :]
    np.fill_diagonal(S, 0.0)
    np.fill_diagonal(Dm, 0.0)
    npn = len(bd.t)
    near = near_panels(bd)
    for i in range(n):
        p = bd.panel_of[i]
        for q in near[p]:
            ws, wd = product_weights(bd, k, X[i], q)
            S[i, q * npn:(q + 1) * npn] = ws
            Dm[i, q * npn:(q + 1) * npn] = wd
    return S, Dm


def receiver_points(thetas: np.ndarray, R: float) -> np.ndarray:
    return R * np.stack([np.cos(thetas), np.sin(thetas)], axis=-1)


def farfield_matrices(bd: Boundary, k: float, thetas: np.ndarray, R: float):
    """(A_phi, A_psi) with u_s(x_p) = A_phi @ u_s|bd + A_psi @ d_n u_s|bd (Green's representation)."""
    xp = receiver_points(thetas, R)
    X = bd.nodes
    A_phi = green_dny(k, xp[:, None, :], X[None, :, :], bd.node_normal[None, :, :]) * bd.node_weight[None, :]
    A_psi = -green(k, xp[:, None, :], X[None, :, :]) * bd.node_weight[None, :]
    return A_phi, A_psi
