"""Closed forms and brute-force references that pin the oracle (no solver code).

* Constant-contrast disk: separation of variables in polar coordinates; the
  scattered field is a Bessel/Hankel series (the radially symmetric special
  case of the forward problem of Sec. 1, eqs. origpde and srad).
* Smooth radial contrast: the same separation with the radial ODE integrated
  numerically (DOP853) and matched to J_n + a_n H_n at the support radius.
* Born Jacobian at q = 0: Theorem 3.1 with q0 = 0 has the explicit solution
  v = -k^2 int G(x, y) dq(y) exp(i k d.y) dy (G of eq. inteqscat), which is a
  smooth integral for receivers outside Omega, done by tensor Gauss-Legendre.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp
from scipy.special import hankel1, jv, jvp, h1vp, roots_legendre


def disk_scattered(k, q0, a, alpha, thetas, R, nmax=60):
    """u_s(R cos theta, R sin theta) for q = q0 on |x| < a, plane wave of angle alpha."""
    k1 = k * math.sqrt(1.0 - q0)
    n = np.arange(-nmax, nmax + 1)
    num = k * jvp(n, k * a) * jv(n, k1 * a) - k1 * jv(n, k * a) * jvp(n, k1 * a)
    den = k1 * hankel1(n, k * a) * jvp(n, k1 * a) - k * h1vp(n, k * a) * jv(n, k1 * a)
    an = num / den
    th = np.asarray(thetas)[:, None]
    return np.sum((1j ** n) * an * hankel1(n, k * R) * np.exp(1j * n * (th - alpha)), axis=1)


def radial_scattered(k, qfun, a, alpha, thetas, R, nmax=40, r0=1e-3):
    """u_s on the circle of radius R for a radial contrast q(r) supported in r < a.

    Each Fourier mode u_n(r) of the total field solves
    r^2 u'' + r u' + (k^2 (1 - q(r)) r^2 - n^2) u = 0, regular at the origin;
    it is started from J_n(k sqrt(1 - q(0)) r) at r0 and integrated to a.
    """
    an = []
    q00 = qfun(0.0)
    for n in range(0, nmax + 1):
        ks = k * math.sqrt(1.0 - q00)
        y0 = [jv(n, ks * r0), ks * jvp(n, ks * r0)]
        scale = max(abs(y0[0]), abs(y0[1]), 1e-300)
        y0 = [y0[0] / scale, y0[1] / scale]

        def rhs(r, y, n=n):
            u, up = y
            return [up, -up / r - (k * k * (1.0 - qfun(r)) - n * n / (r * r)) * u]

        sol = solve_ivp(rhs, (r0, a), y0, method="DOP853", rtol=1e-13, atol=1e-300)
        ua, upa = sol.y[0, -1], sol.y[1, -1]
        num = k * jvp(n, k * a) * ua - jv(n, k * a) * upa
        den = hankel1(n, k * a) * upa - k * h1vp(n, k * a) * ua
        an.append(num / den)
    an = np.array(an)
    n = np.arange(-nmax, nmax + 1)
    a_full = np.concatenate([an[:0:-1], an])  # a_{-n} = a_n for a radial medium
    th = np.asarray(thetas)[:, None]
    return np.sum((1j ** n) * a_full * hankel1(n, k * R) * np.exp(1j * n * (th - alpha)), axis=1)


def born_jacobian(k, alphas, thetas, R, S1, S2, nq=200):
    """J0[(m*P + p), (m1-1)*S2 + m2-1] = -k^2 int_Omega G(x_p, y) s_m1(y1) s_m2(y2) e^{i k d_m.y} dy."""
    x, w = roots_legendre(nq)
    Y1, Y2 = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    s1 = np.sin(np.outer(np.arange(1, S1 + 1), x + 1.0) * math.pi / 2)  # (S1, nq)
    s2 = np.sin(np.outer(np.arange(1, S2 + 1), x + 1.0) * math.pi / 2)
    J = np.zeros((len(alphas) * len(thetas), S1 * S2), dtype=np.complex128)
    for mi, al in enumerate(alphas):
        inc = np.exp(1j * k * (Y1 * math.cos(al) + Y2 * math.sin(al)))
        for pi_, th in enumerate(thetas):
            xp = R * np.array([math.cos(th), math.sin(th)])
            r = np.hypot(xp[0] - Y1, xp[1] - Y2)
            f = -k * k * 0.25j * hankel1(0, k * r) * inc * W  # (nq, nq)
            J[mi * len(thetas) + pi_, :] = (s1 @ f @ s2.T).ravel()
    return J
