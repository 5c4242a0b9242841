"""Forward scattering, its Frechet derivative and the Gauss-Newton step (oracle).

Test infrastructure only.  One frequency k, contrast q on Omega = [-1, 1]^2.

Forward problem (Sec. 1, eqs. origpde/fscatprob/srad; Sec. 2): the total field
u = u_inc + u_s solves  Lap u + k^2 (1 - q) u = 0  in Omega, and outside
Omega the scattered part is radiating, which on the boundary is the identity
(D - I/2) u_s = S d_n u_s of Sec. 2 (Remark).  Discretised as ONE global
collocation system (see the package docstring):

* unknowns: u at the 16 x 16 Chebyshev-Lobatto nodes of every leaf (corner
  nodes carry the dummy equation u = 0: no other equation touches them) and
  psi = d_n u at every boundary node;
* at every interior leaf node: the spectral Laplacian + k^2 (1 - q) u = 0;
* at every interior leaf edge node shared by leaves alpha (west/south) and
  beta (east/north): u_alpha = u_beta on alpha's row, d_n u_alpha + d_n u_beta
  = 0 on beta's row (each normal derivative by its own leaf's spectral
  differentiation);
* at every boundary node: psi = d_n u (leaf differentiation) and the exterior
  identity applied to u_s = u - u_inc, d_n u_s = psi - d_n u_inc: Green's
  identity (eta = 0), or its Burton-Miller combination with the normal
  derivative identity (eta > 0, bie.exterior_rows), which stays solvable at
  the square's Dirichlet eigenvalues.

Measured data (eq. farfielddef): u_s at x_p = R (cos theta_p, sin theta_p) by
Green's representation from the boundary data.  Jacobian (Theorem 3.1, eq.
vdef): one solve of the same system per (mode, direction) with body load
k^2 phi_m u_0 and no incident field.  Gauss-Newton (eq. normaleq): normal
equations in the real sine coefficients.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import hankel1

from . import bie
from .spectral import diff_matrix, lobatto_nodes

P = 16


def sine_basis(m: np.ndarray, t: np.ndarray) -> np.ndarray:
    """s_m(t) = sin(m pi (t + 1) / 2): the sine series of Sec. 3.2 (eq. sineseries) on [-1, 1]."""
    return np.sin(np.outer(m, np.asarray(t) + 1.0) * (math.pi / 2.0))


def sine_eval(c: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """E_k: q(x, y) = sum_{m1, m2} c[m1-1, m2-1] s_m1(x) s_m2(y) at points (x, y) (Definition, Sec. 3.2)."""
    S1, S2 = c.shape
    sx = sine_basis(np.arange(1, S1 + 1), x.ravel())  # (S1, n)
    sy = sine_basis(np.arange(1, S2 + 1), y.ravel())
    return np.einsum("ij,in,jn->n", c, sx, sy).reshape(np.shape(x))


class Grid:
    """Leaf grids of the uniform quadtree: leaf (ix, iy) has id iy * n + ix."""

    def __init__(self, n_leaf: int):
        self.n = n_leaf
        self.h = 2.0 / n_leaf
        self.t = lobatto_nodes(P)
        self.D = diff_matrix(self.t) * (2.0 / self.h)  # d/dx on one leaf
        self.D2 = self.D @ self.D
        nl = n_leaf * n_leaf
        ix = np.arange(nl) % n_leaf
        iy = np.arange(nl) // n_leaf
        xs = -1.0 + ix[:, None] * self.h + (self.t[None, :] + 1.0) * self.h / 2.0  # (nl, 16)
        ys = -1.0 + iy[:, None] * self.h + (self.t[None, :] + 1.0) * self.h / 2.0
        self.X = np.broadcast_to(xs[:, :, None], (nl, P, P)).copy()  # X[l, a, b] = x_a
        self.Y = np.broadcast_to(ys[:, None, :], (nl, P, P)).copy()  # Y[l, a, b] = y_b
        self.nleaves = nl

    def idx(self, leaf, a, b):
        return (leaf * P + a) * P + b

    def leaf_id(self, ix, iy):
        return iy * self.n + ix


def _normal_row(grid: Grid, leaf: int, a: int, b: int):
    """Column indices and coefficients of the outward normal derivative at edge node (a, b)."""
    D = grid.D
    c = np.arange(P)
    if a == 0:
        return grid.idx(leaf, c, b), -D[0, :]
    if a == P - 1:
        return grid.idx(leaf, c, b), D[P - 1, :]
    if b == 0:
        return grid.idx(leaf, a, c), -D[0, :]
    if b == P - 1:
        return grid.idx(leaf, a, c), D[P - 1, :]
    raise ValueError("not an edge node")


def boundary_leaf_nodes(grid: Grid) -> np.ndarray:
    """Global unknown index of each boundary node, in the panel order of bie.make_boundary."""
    n = grid.n
    out = []
    for i in range(n):  # south
        out += [grid.idx(grid.leaf_id(i, 0), a, 0) for a in range(1, P - 1)]
    for i in range(n):  # east
        out += [grid.idx(grid.leaf_id(n - 1, i), P - 1, b) for b in range(1, P - 1)]
    for i in range(n):  # north
        out += [grid.idx(grid.leaf_id(i, n - 1), a, P - 1) for a in range(1, P - 1)]
    for i in range(n):  # west
        out += [grid.idx(grid.leaf_id(0, i), 0, b) for b in range(1, P - 1)]
    return np.array(out)


class Forward:
    """Factored global system for one (q, k).  q_nodes: q at every leaf node, shape (n_L^2, 16, 16)."""

    def __init__(self, k: float, n_leaf: int, q_nodes: np.ndarray, R: float = 3.0, eta: float = 0.0):
        self.k = float(k)
        self.R = float(R)
        self.eta = float(eta)  # 0: Green's identity exterior rows; > 0: Burton-Miller, alpha = i eta / k
        self.grid = g = Grid(n_leaf)
        self.bd = bd = bie.make_boundary(n_leaf)
        self.q = np.asarray(q_nodes, dtype=np.float64).reshape(g.nleaves, P, P)
        self.bnodes = boundary_leaf_nodes(g)
        # consistency: boundary panel nodes coincide with the leaf nodes they sit on
        xy = np.stack([g.X.ravel()[self.bnodes], g.Y.ravel()[self.bnodes]], axis=-1)
        assert np.allclose(xy, bd.nodes, atol=1e-13)
        self.nu = g.nleaves * P * P
        self.nb = len(self.bnodes)
        self.S, self.Dl = bie.layer_matrices(bd, self.k)
        self.A_u, self.A_psi = bie.exterior_rows(bd, self.k, self.S, self.Dl, self.eta)
        self._assemble()
        self.lu = spla.splu(self.A.tocsc())

    # -- assembly -------------------------------------------------------------
    def _assemble(self):
        g, k = self.grid, self.k
        rows, cols, vals = [], [], []

        def add(r, c, v):
            rows.append(np.broadcast_to(r, np.shape(c)).ravel())
            cols.append(np.ravel(c))
            vals.append(np.ravel(v).astype(np.complex128))

        c = np.arange(P)
        bset = {int(j): i for i, j in enumerate(self.bnodes)}
        for leaf in range(g.nleaves):
            ix, iy = leaf % g.n, leaf // g.n
            for a in range(P):
                for b in range(P):
                    r = g.idx(leaf, a, b)
                    corner = a in (0, P - 1) and b in (0, P - 1)
                    if corner:
                        add(r, [r], [1.0])
                        continue
                    if 0 < a < P - 1 and 0 < b < P - 1:
                        # spectral Laplacian + k^2 (1 - q)
                        add(r, g.idx(leaf, c, b), g.D2[a, :])
                        add(r, g.idx(leaf, a, c), g.D2[b, :])
                        add(r, [r], [k * k * (1.0 - self.q[leaf, a, b])])
                        continue
                    if r in bset:
                        continue  # exterior rows are added below
                    # interface node: find the neighbour leaf and its matching node
                    if a == P - 1:
                        nb_leaf, na, nbb, alpha = g.leaf_id(ix + 1, iy), 0, b, True
                    elif a == 0:
                        nb_leaf, na, nbb, alpha = g.leaf_id(ix - 1, iy), P - 1, b, False
                    elif b == P - 1:
                        nb_leaf, na, nbb, alpha = g.leaf_id(ix, iy + 1), a, 0, True
                    else:
                        nb_leaf, na, nbb, alpha = g.leaf_id(ix, iy - 1), a, P - 1, False
                    if alpha:   # continuity of u
                        add(r, [r, g.idx(nb_leaf, na, nbb)], [1.0, -1.0])
                    else:       # continuity of the flux: sum of outward normal derivatives
                        c1, v1 = _normal_row(g, leaf, a, b)
                        c2, v2 = _normal_row(g, nb_leaf, na, nbb)
                        add(r, c1, v1)
                        add(r, c2, v2)
        # boundary rows: psi_j - d_n u_j = 0 and the exterior identity
        nu, nb = self.nu, self.nb
        for j, gj in enumerate(self.bnodes):
            leaf, rem = divmod(int(gj), P * P)
            a, b = divmod(rem, P)
            cj, vj = _normal_row(g, leaf, a, b)
            add(nu + j, [nu + j], [1.0])
            add(nu + j, cj, -vj)
        for i, gi in enumerate(self.bnodes):
            add(int(gi), self.bnodes, self.A_u[i, :])
            add(int(gi), nu + np.arange(nb), -self.A_psi[i, :])
        n = nu + nb
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(n, n))

    # -- solves ---------------------------------------------------------------
    def solve_incident(self, ui_bd: np.ndarray, dni_bd: np.ndarray):
        """Total field for incident traces on the boundary nodes (columns = right-hand sides)."""
        rhs = np.zeros((self.nu + self.nb, ui_bd.shape[1]), dtype=np.complex128)
        rhs[self.bnodes, :] = self.A_u @ ui_bd - self.A_psi @ dni_bd
        return self.lu.solve(rhs)

    def split(self, sol: np.ndarray):
        """(u on leaf nodes (nrhs, n_L^2, 16, 16), u on boundary, psi on boundary)."""
        u = sol[: self.nu].T.reshape(-1, self.grid.nleaves, P, P)
        return u, sol[self.bnodes].T, sol[self.nu:].T

    def plane_traces(self, alphas: np.ndarray):
        """u_inc = exp(i k x.d) and d_n u_inc on the boundary nodes, d = (cos alpha, sin alpha)."""
        d = np.stack([np.cos(alphas), np.sin(alphas)], axis=-1)  # (M, 2)
        X = self.bd.nodes
        ui = np.exp(1j * self.k * (X @ d.T))                      # (nb, M)
        dni = 1j * self.k * (self.bd.node_normal @ d.T) * ui
        return ui, dni

    def point_traces(self, src: np.ndarray):
        """u_inc = G(x, x_src) and d_n u_inc on the boundary nodes, one column per source."""
        X = self.bd.nodes
        dvec = X[:, None, :] - src[None, :, :]
        r = np.linalg.norm(dvec, axis=-1)
        ui = 0.25j * hankel1(0, self.k * r)
        dni = -0.25j * self.k * hankel1(1, self.k * r) * np.sum(dvec * self.bd.node_normal[:, None, :], -1) / r
        return ui, dni

    def farfield(self, phi_s: np.ndarray, psi_s: np.ndarray, thetas: np.ndarray) -> np.ndarray:
        """u_s(R cos theta_p, R sin theta_p) from scattered boundary data (rows = right-hand sides)."""
        A_phi, A_psi = bie.farfield_matrices(self.bd, self.k, thetas, self.R)
        return phi_s @ A_phi.T + psi_s @ A_psi.T

    def solve_plane(self, alphas: np.ndarray, thetas: np.ndarray):
        """u_far[m, p] for incidence alpha_m and receiver theta_p; also the interior total fields."""
        ui, dni = self.plane_traces(alphas)
        u, ub, psi = self.split(self.solve_incident(ui, dni))
        ufar = self.farfield(ub - ui.T, psi - dni.T, thetas)
        return ufar, u

    # -- Frechet derivative (Theorem 3.1) ---------------------------------------
    def jacobian(self, alphas: np.ndarray, thetas: np.ndarray, S1: int, S2: int) -> np.ndarray:
        """J[(m*P + p), (m1-1)*S2 + (m2-1)] = v_far for Lap v + k^2(1-q) v = k^2 phi_m u_m."""
        g, k = self.grid, self.k
        _, u0 = self.solve_plane(alphas, thetas)  # (M, nl, 16, 16)
        M, Pn = len(alphas), len(thetas)
        sx = sine_basis(np.arange(1, S1 + 1), g.X.ravel()).reshape(S1, g.nleaves, P, P)
        sy = sine_basis(np.arange(1, S2 + 1), g.Y.ravel()).reshape(S2, g.nleaves, P, P)
        interior = np.zeros((P, P), dtype=bool)
        interior[1:-1, 1:-1] = True
        J = np.zeros((M * Pn, S1 * S2), dtype=np.complex128)
        A_phi, A_psi = bie.farfield_matrices(self.bd, k, thetas, self.R)
        for m1 in range(S1):
            for m2 in range(S2):
                phi = (sx[m1] * sy[m2]) * interior  # (nl, 16, 16), zero off the PDE rows
                rhs = np.zeros((self.nu + self.nb, M), dtype=np.complex128)
                rhs[: self.nu, :] = (k * k * phi[None] * u0).reshape(M, -1).T
                v = self.lu.solve(rhs)
                vfar = v[self.bnodes].T @ A_phi.T + v[self.nu:].T @ A_psi.T  # (M, P)
                J[:, m1 * S2 + m2] = vfar.ravel()
        return J


def forward_from_coeffs(c: np.ndarray, k: float, n_leaf: int, R: float = 3.0, eta: float = 0.0) -> Forward:
    g = Grid(n_leaf)
    return Forward(k, n_leaf, sine_eval(c, g.X, g.Y), R, eta)


def forward_from_function(qfun, k: float, n_leaf: int, R: float = 3.0, eta: float = 0.0) -> Forward:
    g = Grid(n_leaf)
    return Forward(k, n_leaf, qfun(g.X, g.Y), R, eta)


def gn_step(J: np.ndarray, resid: np.ndarray, lam: float) -> np.ndarray:
    """Real update from the normal equations (eq. normaleq): (Re J^H J + lam I) dc = Re J^H r."""
    A = (J.conj().T @ J).real + lam * np.eye(J.shape[1])
    b = (J.conj().T @ resid).real
    return np.linalg.solve(A, b)


def misfit_gradient(J: np.ndarray, F: np.ndarray, data: np.ndarray) -> np.ndarray:
    """d/dc of 0.5 ||F(c) - data||^2 = Re J^H (F - data) (Theorem 3.2 read on the sine coefficients)."""
    return (J.conj().T @ (F - data)).real
