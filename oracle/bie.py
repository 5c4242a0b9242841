"""Boundary of Omega: panels, layer potentials and the field on the receiver circle.

Test infrastructure only.  Follows Sec. 2 (Remark): the scattered field
outside Omega satisfies Green's representation u_s = D u_s - S d_n u_s with

    S phi(x) = int G(x, y) phi(y) ds_y,
    D phi(x) = int d/dn_y G(x, y) phi(y) ds_y,
    G(x, y)  = (i/4) H_0^(1)(k |x - y|),

and, on the boundary, the jump relations give (D - I/2) u_s = S d_n u_s.  The
same representation evaluated at x_p = R (cos theta_p, sin theta_p) gives the
measured field u_far(theta_p) of Sec. 1 (eq. farfielddef).

That identity alone is singular where k^2 is a Dirichlet eigenvalue of the
square (S has a null space there).  Its normal derivative, with
K' phi(x) = int d/dn_x G phi ds_y and T = d/dn_x D, is T u_s = (K' + I/2) d_n u_s;
the Burton-Miller combination of the two with coupling alpha = i eta / k
(exterior_rows, eta > 0) is uniquely solvable at every k > 0 (the reading of
the combined-field exterior used here).  T comes from Maue's identity,
T phi = d/dt_x S(d phi/dt) + k^2 n_x . S(n phi), with the tangential
derivative of S integrated as a principal value on the target's own panel.

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

from .spectral import diff_matrix, gauss_legendre, interp_quad_weights, lagrange_eval, lobatto_nodes

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


_RULES: dict = {}


def _graded_basis(t: np.ndarray, h: float, s_star: float):
    """(_graded_rule(h, s_star), the panel's Lagrange basis at its points), computed once per
    distinct (panel nodes, h, s_star): the targets of a boundary meet only a few offsets s_star
    (the panel nodes and the panel ends), so the rule is shared by every target at that offset.
    The arrays are shared: callers only read them."""
    key = (tuple(t), h, s_star)
    if key not in _RULES:
        sig, w = _graded_rule(h, s_star)
        _RULES[key] = (sig, w, lagrange_eval(t, 2.0 * (s_star + sig) / h - 1.0))
    return _RULES[key]


def product_weights(bd: Boundary, k: float, x: np.ndarray, q: int):
    """int_panel K(x, y(s)) L_j(s) ds for K = G and K = dG/dn_y, j over the panel nodes."""
    y0, tau, ny = bd.start[q], bd.tangent[q], bd.normal[q]
    s_star = float(np.clip(np.dot(x - y0, tau), 0.0, bd.h))
    sig, w, L = _graded_basis(bd.t, bd.h, s_star)     # L: (nq, 14) Lagrange basis at the points
    perp = x - (y0 + s_star * tau)                  # x - y(s_star)
    dvec = perp[None, :] - sig[:, None] * tau[None, :]  # x - y(s_star + sigma)
    r = np.sqrt(np.sum(dvec * dvec, axis=-1))
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


def ccw_sign(bd: Boundary) -> np.ndarray:
    """+1 where a panel's tangent runs counter-clockwise around Omega (tangent = normal turned
    by +90 degrees), -1 where it runs the other way (north and west sides)."""
    ccw = np.stack([-bd.normal[:, 1], bd.normal[:, 0]], axis=-1)
    return np.sign(np.sum(ccw * bd.tangent, axis=-1))


def normal_tangent_matrices(bd: Boundary, k: float):
    """Nystrom matrices of the kernels d/dn_x G and d/dt_x G (t_x the counter-clockwise tangent at
    the target), on the same panels and near rule as layer_matrices.

    K'[i, j] ~ int dG/dn_x(x_i, y) L_j(y) ds_y: zero on the target's own side (the side is
    straight).  H[i, j] ~ PV int dG/dt_x(x_i, y) L_j(y) ds_y: on the target's own panel the kernel
    is -sgn/(2 pi (s_x - s)) plus a remainder with a logarithmic singularity; the Cauchy part is
    integrated in closed form, PV int_0^h f(s)/(s_x - s) ds = f(s_x) log(s_x / (h - s_x))
    + int_0^h (f(s) - f(s_x)) / (s_x - s) ds (the last integrand a polynomial: Gauss-Legendre),
    and the remainder by the graded rule.
    """
    X = bd.nodes
    n = len(X)
    sgn = ccw_sign(bd)
    tx = np.repeat(sgn[:, None] * bd.tangent, len(bd.t), axis=0)  # counter-clockwise tangents
    d = X[:, None, :] - X[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    np.fill_diagonal(r, 1.0)
    h1 = -0.25j * k * hankel1(1, k * r) / r * bd.node_weight[None, :]
    Kp = h1 * np.sum(d * bd.node_normal[:, None, :], axis=-1)
    H = h1 * np.sum(d * tx[:, None, :], axis=-1)
    np.fill_diagonal(Kp, 0.0)
    np.fill_diagonal(H, 0.0)
    npn = len(bd.t)
    near = near_panels(bd)
    xg, wg = gauss_legendre(GRADE_GL)
    for i in range(n):
        p = bd.panel_of[i]
        nx, txi = bd.node_normal[i], tx[i]
        for q in near[p]:
            y0, tau = bd.start[q], bd.tangent[q]
            s_star = float(np.clip(np.dot(X[i] - y0, tau), 0.0, bd.h))
            sig, w, L = _graded_basis(bd.t, bd.h, s_star)
            perp = X[i] - (y0 + s_star * tau)
            dvec = perp[None, :] - sig[:, None] * tau[None, :]
            rr = np.sqrt(np.sum(dvec * dvec, axis=-1))
            base = -0.25j * k * hankel1(1, k * rr) / rr * w
            Kp[i, q * npn:(q + 1) * npn] = (base * (dvec @ nx)) @ L
            kt = base * (dvec @ txi)
            if q == p:  # own panel: subtract the Cauchy part, sgn * (-1 / (2 pi (s_x - s)))
                s_x = s_star
                delta = -sig                                   # s_x - s
                kt = kt - sgn[p] * (-1.0 / (2.0 * np.pi * delta)) * w
                hv = kt @ L
                # closed-form principal value of the Cauchy part against each L_j
                sg = 0.5 * bd.h * (xg + 1.0)                   # Gauss-Legendre on [0, h]
                wgs = 0.5 * bd.h * wg
                Lg = lagrange_eval(bd.t, 2.0 * sg / bd.h - 1.0)       # (16, 14)
                Lx = lagrange_eval(bd.t, np.array([2.0 * s_x / bd.h - 1.0]))[0]  # (14,)
                pv = Lx * np.log(s_x / (bd.h - s_x)) + ((Lg - Lx[None, :]) / (s_x - sg)[:, None]).T @ wgs
                H[i, q * npn:(q + 1) * npn] = hv + sgn[p] * (-1.0 / (2.0 * np.pi)) * pv
            else:
                H[i, q * npn:(q + 1) * npn] = kt @ L
    return Kp, H


def hypersingular_matrix(bd: Boundary, k: float, S: np.ndarray, H: np.ndarray) -> np.ndarray:
    """T = d/dn_x D (the normal derivative of the double layer) by Maue's identity,
    T phi = d/dt_x S (d phi / dt) + k^2 n_x . S (n phi), with d/dt the counter-clockwise
    tangential derivative: H (d/dt_x S, from normal_tangent_matrices) times the panel-wise
    differentiation of phi's degree-13 interpolant."""
    sgn = ccw_sign(bd)
    Dref = diff_matrix(bd.t) * (2.0 / bd.h)
    Dt = np.kron(np.diag(sgn), Dref)
    Nx, Ny = bd.node_normal[:, 0], bd.node_normal[:, 1]
    return H @ Dt + k * k * (Nx[:, None] * S * Nx[None, :] + Ny[:, None] * S * Ny[None, :])


def exterior_rows(bd: Boundary, k: float, S: np.ndarray, Dl: np.ndarray, eta: float = 0.0):
    """(A_u, A_psi) of the exterior relation A_u u_s = A_psi d_n u_s on the boundary nodes.

    eta = 0: Green's identity, (D - I/2) u_s = S d_n u_s (singular where k^2 is a Dirichlet
    eigenvalue of the square).  eta > 0: the Burton-Miller combination of it with its normal
    derivative T u_s = (K' + I/2) d_n u_s, coupling alpha = i eta / k:
    (D - I/2 + alpha T) u_s = (S + alpha (K' + I/2)) d_n u_s, uniquely solvable at every k > 0.
    """
    I = np.eye(len(bd.nodes))
    A_u, A_psi = Dl - 0.5 * I, S.copy()
    if eta > 0.0:
        alpha = 1j * eta / k
        Kp, H = normal_tangent_matrices(bd, k)
        A_u = A_u + alpha * hypersingular_matrix(bd, k, S, H)
        A_psi = A_psi + alpha * (Kp + 0.5 * I)
    return A_u, A_psi


def receiver_points(thetas: np.ndarray, R: float) -> np.ndarray:
    return R * np.stack([np.cos(thetas), np.sin(thetas)], axis=-1)


def farfield_matrices(bd: Boundary, k: float, thetas: np.ndarray, R: float):
    """(A_phi, A_psi) with u_s(x_p) = A_phi @ u_s|bd + A_psi @ d_n u_s|bd (Green's representation)."""
    xp = receiver_points(thetas, R)
    X = bd.nodes
    A_phi = green_dny(k, xp[:, None, :], X[None, :, :], bd.node_normal[None, :, :]) * bd.node_weight[None, :]
    A_psi = -green(k, xp[:, None, :], X[None, :, :]) * bd.node_weight[None, :]
    return A_phi, A_psi
