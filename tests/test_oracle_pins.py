"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each pin is chosen so that a plausible mistake in the oracle (a dropped term,
a sign, a transposed operand, a wrong normal, a wrong weight) fails one of
them: closed forms (disk and radial media), a brute-force integral (Born
Jacobian), finite differences, Green's-function symmetry, reciprocity of the
far-field pattern, energy conservation (the optical theorem), a library
least-squares solve and the grid-size column the paper prints (Table 1).
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import hankel1

import closed_forms as CF
import synth
from oracle import bie
from oracle import forward as F
from oracle.spectral import (diff_matrix, interp_quad_weights, lagrange_eval,
                             lobatto_nodes)

K5 = 5.0


@pytest.fixture(scope="module")
def fw_zero():
    return F.forward_from_coeffs(np.zeros((5, 5)), K5, 4)


# --- 1-D spectral pieces ------------------------------------------------------
def test_diff_matrix_exact_on_polynomials():
    t = lobatto_nodes(16)
    D = diff_matrix(t)
    for deg in range(16):
        err = np.abs(D @ t**deg - (deg * t ** (deg - 1) if deg else 0 * t)).max()
        assert err < 1e-11 * max(1, deg) ** 2


def test_interior_quadrature_exact_to_degree_13():
    t = lobatto_nodes(16)[1:-1]
    w = interp_quad_weights(t)
    assert np.all(w > 0)  # Fejer's second rule has positive weights
    for deg in range(14):
        exact = (1 - (-1) ** (deg + 1)) / (deg + 1)
        assert abs(w @ t**deg - exact) < 1e-14


def test_lagrange_basis_is_cardinal():
    t = lobatto_nodes(16)[1:-1]
    assert np.allclose(lagrange_eval(t, t), np.eye(14), atol=1e-13)


def test_grid_point_counts_match_table1():
    """Distinct points of 2^l x 2^l leaves of 16 x 16 Chebyshev nodes (paper Table 1, column N)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_grid_points.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for nl, N in rows:
        g = F.Grid(int(nl)) if int(nl) <= 16 else None
        if g is None:
            continue
        pts = np.unique(np.round(np.stack([g.X.ravel(), g.Y.ravel()], -1), 12), axis=0)
        assert len(pts) == int(N)


def test_sine_eval_matches_direct_sum():
    rng = np.random.default_rng(0)
    c = rng.standard_normal((4, 3))
    x, y = rng.uniform(-1, 1, 7), rng.uniform(-1, 1, 7)
    ref = [sum(c[a, b] * math.sin((a + 1) * math.pi * (xi + 1) / 2) * math.sin((b + 1) * math.pi * (yi + 1) / 2)
               for a in range(4) for b in range(3)) for xi, yi in zip(x, y)]
    assert np.allclose(F.sine_eval(c, x, y), ref, atol=1e-14)


# --- boundary integral pieces -------------------------------------------------
def test_product_weights_match_quadpack():
    """Singular and near-singular panel integrals against QUADPACK with the singular point given."""
    bd = bie.make_boundary(4)
    k = K5
    i = 3  # a node on panel 0
    x = bd.nodes[i]
    for q in (0, 1, 15):  # self, neighbour on the same side, neighbour across the corner
        ws, wd = bie.product_weights(bd, k, x, q)
        y0, tau, ny = bd.start[q], bd.tangent[q], bd.normal[q]
        for j in (0, 6, 13):
            def f(s, part, kern):
                y = y0 + s * tau
                d = x - y
                r = math.hypot(*d)
                Lj = lagrange_eval(bd.t, np.array([2 * s / bd.h - 1]))[0, j]
                if kern == "S":
                    val = 0.25j * hankel1(0, k * r)
                else:
                    val = 0.25j * k * hankel1(1, k * r) * (d @ ny) / r
                return (val.real if part == 0 else val.imag) * Lj
            sing = [float(np.clip((x - y0) @ tau, 0, bd.h))]
            for kern, w in (("S", ws), ("D", wd)):
                re = quad(f, 0, bd.h, args=(0, kern), points=sing, limit=200, epsabs=1e-15, epsrel=1e-13)[0]
                im = quad(f, 0, bd.h, args=(1, kern), points=sing, limit=200, epsabs=1e-15, epsrel=1e-13)[0]
                assert abs(w[j] - (re + 1j * im)) < 1e-12, (q, j, kern)


def test_normal_and_tangential_weights_match_quadpack():
    """d/dn_x G and d/dt_x G panel weights (normal_tangent_matrices) against QUADPACK: the near
    panels by adaptive quadrature with the singular point given, the target's own panel for the
    tangential kernel as a Cauchy principal value (QAWC, weight 1/(s - s_x))."""
    bd = bie.make_boundary(4)
    k = K5
    Kp, H = bie.normal_tangent_matrices(bd, k)
    sgn = bie.ccw_sign(bd)
    npn = len(bd.t)
    for i in (3, 12, 9 * npn + 5):  # south side (two panels), north side (clockwise panel tangent)
        x = bd.nodes[i]
        p = bd.panel_of[i]
        nx, tx = bd.node_normal[i], sgn[p] * bd.tangent[p]
        for q in bie.near_panels(bd)[p]:  # the panels the product rule covers (own, same side, across a corner)
            y0, tau = bd.start[q], bd.tangent[q]
            s_x = float(np.clip((x - y0) @ tau, 0, bd.h))
            for j in (0, 6, 13):
                def f(s, part, kern, pv):
                    d = x - (y0 + s * tau)
                    r = math.hypot(*d)
                    Lj = lagrange_eval(bd.t, np.array([2 * s / bd.h - 1]))[0, j]
                    val = -0.25j * k * hankel1(1, k * r) * (d @ (nx if kern == "K'" else tx)) / r
                    if pv:
                        val = val * (s - s_x)  # QAWC divides by (s - s_x)
                    return (val.real if part == 0 else val.imag) * Lj
                for kern, M in (("K'", Kp), ("H", H)):
                    got = M[i, q * npn + j]
                    if q == p and kern == "K'":
                        assert got == 0.0  # the side is straight: (x - y) . n_x = 0
                        continue
                    if q == p:
                        kw = dict(weight="cauchy", wvar=s_x, limit=200, epsabs=1e-15, epsrel=1e-13)
                        re = quad(f, 0, bd.h, args=(0, kern, True), **kw)[0]
                        im = quad(f, 0, bd.h, args=(1, kern, True), **kw)[0]
                    else:
                        kw = dict(points=[s_x], limit=200, epsabs=1e-15, epsrel=1e-13)
                        re = quad(f, 0, bd.h, args=(0, kern, False), **kw)[0]
                        im = quad(f, 0, bd.h, args=(1, kern, False), **kw)[0]
                    assert abs(got - (re + 1j * im)) < 1e-11, (i, q, j, kern, got, re + 1j * im)


def test_normal_derivative_identity_for_radiating_source(fw_zero):
    """T u = (K' + I/2) d_n u on the boundary (the normal derivative of Green's representation;
    T by Maue's identity from the tangential-derivative kernel) for u = G(., x0), x0 in Omega:
    pins T, K' and the tangent orientation at every node, the corner panels included."""
    fw = fw_zero
    Kp, H = bie.normal_tangent_matrices(fw.bd, K5)
    T = bie.hypersingular_matrix(fw.bd, K5, fw.S, H)
    for x0 in (np.array([[0.2, -0.3]]), np.array([[-0.5, 0.4]])):
        ui, dni = fw.point_traces(x0)
        res = T @ ui - (Kp + 0.5 * np.eye(fw.nb)) @ dni
        assert np.abs(res).max() < 1e-7 * np.abs(dni).max()  # measured 5e-11 and 2e-8 (source 0.5 from the side)


def test_combined_field_at_a_dirichlet_eigenvalue():
    """At k^2 = (pi/2)^2 (1 + 4), a Dirichlet eigenvalue of [-1, 1]^2, Green's identity alone
    leaves the exterior relation singular (far field off by O(1)); the Burton-Miller rows
    (eta = 1) give the radial ODE reference to the discretisation error, and agree with the
    Green rows at a regular k."""
    sig, q0, alpha = 0.15, 0.3, 0.3
    th = synth.receivers(12)
    qf = lambda x, y: q0 * np.exp(-(x * x + y * y) / (2 * sig * sig))
    k = 0.5 * math.pi * math.sqrt(5.0)
    ref = CF.radial_scattered(k, lambda r: q0 * math.exp(-r * r / (2 * sig * sig)), 1.0, alpha, th, 3.0, nmax=30)
    err = {}
    for eta in (0.0, 1.0):
        uf, _ = F.forward_from_function(qf, k, 8, eta=eta).solve_plane(np.array([alpha]), th)
        err[eta] = np.abs(uf[0] - ref).max() / np.abs(ref).max()
    assert err[1.0] < 2e-9 and err[0.0] > 1e-2, err
    u0, _ = F.forward_from_function(qf, K5, 4).solve_plane(np.array([alpha]), th)
    u1, _ = F.forward_from_function(qf, K5, 4, eta=1.0).solve_plane(np.array([alpha]), th)
    assert np.abs(u1 - u0).max() < 1e-7 * np.abs(u0).max()


def test_green_identity_for_radiating_source(fw_zero):
    """(D - I/2) u = S d_n u on the boundary, and Green's representation at R, for u = G(., x0), x0 in Omega."""
    fw = fw_zero
    x0 = np.array([[0.2, -0.3]])
    ui, dni = fw.point_traces(x0)
    res = (fw.Dl - 0.5 * np.eye(fw.nb)) @ ui - fw.S @ dni
    assert np.abs(res).max() < 1e-10 * np.abs(ui).max()
    th = synth.receivers(8)
    A_phi, A_psi = bie.farfield_matrices(fw.bd, K5, th, 3.0)
    xp = 3.0 * np.stack([np.cos(th), np.sin(th)], -1)
    exact = 0.25j * hankel1(0, K5 * np.linalg.norm(xp - x0, axis=-1))
    assert np.abs(A_phi @ ui[:, 0] + A_psi @ dni[:, 0] - exact).max() < 1e-10 * np.abs(exact).max()


# --- forward map ----------------------------------------------------------------
def test_zero_contrast_scatters_nothing(fw_zero):
    uf, u = fw_zero.solve_plane(synth.directions(4), synth.receivers(8))
    assert np.abs(uf).max() < 1e-10


def test_radial_gaussian_matches_ode_reference():
    sig, q0 = 0.15, 0.3
    th = synth.receivers(12)
    alpha = 0.3
    ref = CF.radial_scattered(K5, lambda r: q0 * math.exp(-r * r / (2 * sig * sig)), 1.0, alpha, th, 3.0, nmax=30)
    fw = F.forward_from_function(lambda x, y: q0 * np.exp(-(x * x + y * y) / (2 * sig * sig)), K5, 8)
    uf, _ = fw.solve_plane(np.array([alpha]), th)
    assert np.abs(uf[0] - ref).max() < 2e-9 * np.abs(ref).max()


def test_disk_matches_bessel_series():
    """Jump not aligned with leaves: algebraic convergence, so a loose bound (sign and scale check)."""
    a, q0, alpha = 0.55, 0.2, 0.3
    th = synth.receivers(12)
    ref = CF.disk_scattered(K5, q0, a, alpha, th, 3.0)
    fw = F.forward_from_function(lambda x, y: np.where(x * x + y * y < a * a, q0, 0.0), K5, 4)
    uf, _ = fw.solve_plane(np.array([alpha]), th)
    assert np.abs(uf[0] - ref).max() < 2e-2 * np.abs(ref).max()


def test_green_function_symmetry():
    """Scattered field at x_b from a source at x_a equals that at x_a from a source at x_b.

    The identity is exact for the continuous problem; the collocation scheme is
    not symmetric, so it holds to discretisation error (about 4e-9 here, with the
    contrast's jump at the corners of Omega); a transposed or mis-signed
    operand gives an O(1) mismatch.
    """
    qt = synth.gaussian_bumps(1)
    fw = F.forward_from_function(qt, K5, 4)
    th = np.array([0.4, 2.1])
    src = 3.0 * np.stack([np.cos(th), np.sin(th)], -1)
    ui, dni = fw.point_traces(src)
    _, ub, psi = fw.split(fw.solve_incident(ui, dni))
    us = fw.farfield(ub - ui.T, psi - dni.T, th)  # us[source, receiver]
    assert abs(us[0, 1] - us[1, 0]) < 5e-8 * abs(us[0, 1])


# --- Jacobian -------------------------------------------------------------------
def test_jacobian_at_zero_is_born_integral(fw_zero):
    al, th, S = synth.directions(4), synth.receivers(6), 5
    J = fw_zero.jacobian(al, th, S, S)
    J0 = CF.born_jacobian(K5, al, th, 3.0, S, S, nq=120)
    assert np.abs(J - J0).max() < 2e-9 * np.abs(J0).max()


def test_jacobian_matches_finite_differences():
    S, h = 4, 1e-5
    al, th = synth.directions(3), synth.receivers(5)
    c = synth.random_coeffs(S, S, seed=5, scale=0.03)
    J = F.forward_from_coeffs(c, K5, 4).jacobian(al, th, S, S)
    for m in (0, 6, 15):
        cp, cm = c.copy(), c.copy()
        cp.flat[m] += h
        cm.flat[m] -= h
        up, _ = F.forward_from_coeffs(cp, K5, 4).solve_plane(al, th)
        um, _ = F.forward_from_coeffs(cm, K5, 4).solve_plane(al, th)
        fd = ((up - um) / (2 * h)).ravel()
        assert np.abs(fd - J[:, m]).max() < 2e-6 * np.abs(J[:, m]).max()


def test_jacobian_with_combined_rows_at_an_eigenvalue_matches_finite_differences():
    """The oracle's Frechet Jacobian (one solve per mode of the assembled system) with the
    Burton-Miller exterior rows, at the Dirichlet eigenvalue k = (pi/2) sqrt(5) where the Green
    rows alone are singular, against central differences of its own forward map (2 x 2 leaves)."""
    S, h, k = 3, 1e-5, 0.5 * math.pi * math.sqrt(5.0)
    al, th = synth.directions(2), synth.receivers(4)
    c = synth.random_coeffs(S, S, seed=6, scale=0.03)
    J = F.forward_from_coeffs(c, k, 2, eta=1.0).jacobian(al, th, S, S)
    for m in (0, 4, 8):
        cp, cm = c.copy(), c.copy()
        cp.flat[m] += h
        cm.flat[m] -= h
        up, _ = F.forward_from_coeffs(cp, k, 2, eta=1.0).solve_plane(al, th)
        um, _ = F.forward_from_coeffs(cm, k, 2, eta=1.0).solve_plane(al, th)
        fd = ((up - um) / (2 * h)).ravel()
        assert np.abs(fd - J[:, m]).max() < 2e-6 * np.abs(J[:, m]).max()


def test_misfit_gradient_matches_finite_differences():
    """Central differences of 0.5 ||F(c) - d||^2 in single coefficients (k = 5, 4 x 4 leaves)
    against Re J^H (F - d): a dropped conjugate, a transposed J or a flipped residual sign fails.
    h = 1e-4 balances the h^2 truncation against the rounding of the two solves (both ~2e-8 here)."""
    S, h = 4, 1e-4
    al, th = synth.directions(3), synth.receivers(5)
    c = synth.random_coeffs(S, S, seed=5, scale=0.03)
    rng = np.random.default_rng(21)
    fw = F.forward_from_coeffs(c, K5, 4)
    Fc, _ = fw.solve_plane(al, th)
    d = Fc + 0.05 * (rng.standard_normal(Fc.shape) + 1j * rng.standard_normal(Fc.shape))
    J = fw.jacobian(al, th, S, S)
    g = F.misfit_gradient(J, Fc.ravel(), d.ravel())

    def phi(cc):
        u, _ = F.forward_from_coeffs(cc, K5, 4).solve_plane(al, th)
        return 0.5 * np.linalg.norm(u - d) ** 2

    for m in (0, 5, 10, 15):
        cp, cm = c.copy(), c.copy()
        cp.flat[m] += h
        cm.flat[m] -= h
        fd = (phi(cp) - phi(cm)) / (2 * h)
        assert abs(fd - g[m]) < 1e-7 * np.abs(g).max()


# --- Gauss-Newton step ------------------------------------------------------------
def test_normal_equations_equal_stacked_lstsq():
    rng = np.random.default_rng(3)
    J = rng.standard_normal((40, 6)) + 1j * rng.standard_normal((40, 6))
    r = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    lam = 0.1
    dc = F.gn_step(J, r, lam)
    Ast = np.vstack([J.real, J.imag, math.sqrt(lam) * np.eye(6)])
    bst = np.concatenate([r.real, r.imag, np.zeros(6)])
    ref = np.linalg.lstsq(Ast, bst, rcond=None)[0]
    assert np.abs(dc - ref).max() < 1e-12 * np.abs(ref).max()


def test_gn_recovers_coefficients_from_linearised_data(fw_zero):
    """Data exactly J c (Born regime, well-resolved low modes): one step returns c."""
    S = 3
    al, th = synth.directions(8), synth.receivers(12)
    J = fw_zero.jacobian(al, th, S, S)
    c = synth.random_coeffs(S, S, seed=9)
    dc = F.gn_step(J, J @ c.ravel(), 0.0)
    assert np.abs(dc - c.ravel()).max() < 1e-8 * np.abs(c).max()


def test_oracle_sweep_recovers_band_limited_contrast():
    """Exact data of a contrast inside the band limit: two frequencies of Newton steps recover it."""
    from types import SimpleNamespace
    from oracle import sweep as OS
    c_true = synth.random_coeffs(3, 3, seed=41, scale=0.05)
    plans = [SimpleNamespace(k=k, leaves_per_side=2, S=3, M=8, P=8, newton=3) for k in (2.0, 3.0)]
    data = {}

    def data_fn(p, al, th):
        if p.k not in data:
            data[p.k] = F.forward_from_coeffs(c_true, p.k, p.leaves_per_side).solve_plane(al, th)[0]
        return data[p.k]

    c, hist = OS.sweep(plans, data_fn, lambda_rel=1e-8)
    assert np.abs(c - c_true).max() < 1e-4 * np.abs(c_true).max()
    assert hist[0][-1] < 1e-3 * hist[0][0]


# --- far-field pattern: reciprocity and the optical theorem ----------------------
def pattern(fw, alphas, xhat_angles):
    """Far-field pattern u_inf(xhat; d) of u_s = exp(i k r)/sqrt(r) (u_inf + O(1/r)) from the
    oracle's scattered boundary data by Green's representation with the asymptotic kernel:
    u_inf(xhat) = e^{i pi/4}/sqrt(8 pi k) int (d_n_y e^{-i k xhat.y} u_s - e^{-i k xhat.y} d_n u_s) ds_y.
    Written here from the large-argument form of H_0, independently of the oracle's receivers."""
    k = fw.k
    ui, dni = fw.plane_traces(np.asarray(alphas))
    _, ub, psi = fw.split(fw.solve_incident(ui, dni))
    phi_s, psi_s = ub - ui.T, psi - dni.T  # (M, nb)
    xh = np.stack([np.cos(xhat_angles), np.sin(xhat_angles)], -1)  # (Q, 2)
    X, nrm, w = fw.bd.nodes, fw.bd.node_normal, fw.bd.node_weight
    e = np.exp(-1j * k * (xh @ X.T))  # (Q, nb)
    dne = -1j * k * (xh @ nrm.T) * e
    c = np.exp(1j * math.pi / 4) / math.sqrt(8 * math.pi * k)
    return c * ((phi_s * w) @ dne.T - (psi_s * w) @ e.T)  # (M, Q)


def test_far_field_pattern_reciprocity():
    """u_inf(xhat; d) = u_inf(-d; -xhat) (exact for the continuous problem; discretisation
    error here, as for the Green-function symmetry)."""
    fw = F.forward_from_function(synth.gaussian_bumps(1), K5, 4)
    a1, t1 = 0.4, 2.1
    u12 = pattern(fw, [a1], np.array([t1]))[0, 0]
    u21 = pattern(fw, [t1 + math.pi], np.array([a1 + math.pi]))[0, 0]
    assert abs(u12 - u21) < 5e-8 * abs(u12)


def test_optical_theorem_energy_conservation():
    """For real q no energy is absorbed: Im int conj(u) d_r u over a circle of radius rho -> oo
    vanishes for the total field u = u_i + u_s.  The scattered part gives k int |u_inf|^2; the
    cross terms, by stationary phase at xhat = d (int exp(i k rho (1 - cos t)) dt ~
    sqrt(2 pi / (k rho)) e^{i pi/4}; the contributions at xhat = -d cancel), give
    sqrt(8 pi k) Re(e^{i pi/4} u_inf(d)).  So k int |u_inf|^2 dxhat = -sqrt(8 pi k) Re(e^{i pi/4}
    u_inf(d)).  A wrong sign, normal or weight in the exterior representation breaks it at O(1)."""
    fw = F.forward_from_function(synth.gaussian_bumps(1), K5, 4)
    alpha = 0.7
    Q = 256
    th = 2 * math.pi * np.arange(Q) / Q
    u = pattern(fw, [alpha], th)[0]
    lhs = K5 * np.sum(np.abs(u) ** 2) * (2 * math.pi / Q)
    fwd = pattern(fw, [alpha], np.array([alpha]))[0, 0]
    rhs = -math.sqrt(8 * math.pi * K5) * (np.exp(1j * math.pi / 4) * fwd).real
    assert abs(lhs - rhs) < 1e-8 * abs(lhs)
