"""Recursive linearization over frequency, oracle version (test infrastructure only).

Sec. 3.4 ("Recursive Linearization using Newton's method"): for increasing
frequencies, start Newton's method at k_j from the contrast found at k_{j-1}
and take Gauss-Newton steps with the normal equations (eq. normaleq) at each
frequency.  The band limit grows with k; coefficients found at a lower
frequency are carried into the larger basis with the new modes at zero.
Built from the oracle's forward map, its column-by-column Frechet Jacobian
(Theorem 3.1) and gn_step; feasible only at low k.
"""
from __future__ import annotations

import numpy as np

from . import forward as F
from . import lsqr as L


def embed(c: np.ndarray, S1: int, S2: int) -> np.ndarray:
    out = np.zeros((S1, S2))
    a, b = min(S1, c.shape[0]), min(S2, c.shape[1])
    out[:a, :b] = c[:a, :b]
    return out


def sweep(plans, data_fn, lambda_rel: float, c0=None, R: float | None = None, solver: str = "direct",
          lsqr_tol: float = 1e-3, lsqr_max_iter: int = 200, eta: float = 0.0):
    """plans: objects with k, leaves_per_side, S, M, P, newton (increasing k), and
    optionally R and mask() (the unknown modes; None = all).

    data_fn(plan, alphas, thetas) -> measured far field (M x P complex).
    solver: "direct" = normal equations with lambda_rel (eq. normaleq); "lsqr" = the
    paper's LSQR at lsqr_tol on the plan's modes (Sec. 4).
    eta: exterior rows of the forward map (0 Green's identity, > 0 Burton-Miller, bie.exterior_rows).
    Returns the final coefficients and the residual norms per frequency.
    """
    c = np.zeros((plans[0].S, plans[0].S)) if c0 is None else np.asarray(c0, dtype=np.float64)
    history = []
    for p in plans:
        c = embed(c, p.S, p.S)
        al = 2 * np.pi * np.arange(p.M) / p.M
        th = 2 * np.pi * np.arange(p.P) / p.P
        data = data_fn(p, al, th)
        res = []
        radius = getattr(p, "R", 3.0) if R is None else R
        mask = p.mask() if hasattr(p, "mask") else None
        for _ in range(p.newton):
            fw = F.forward_from_coeffs(c, p.k, p.leaves_per_side, radius, eta)
            Fc, _ = fw.solve_plane(al, th)
            J = fw.jacobian(al, th, p.S, p.S)
            r = (data - Fc).ravel()
            if solver == "lsqr":
                dc, _ = L.gn_step_lsqr(J, r, lsqr_tol, lsqr_max_iter, None if mask is None else mask.ravel())
            else:
                A = (J.conj().T @ J).real
                lam = lambda_rel * np.trace(A) / A.shape[0]
                dc = F.gn_step(J, r, lam)
            c = c + dc.reshape(p.S, p.S)
            res.append(float(np.linalg.norm(r)))
        history.append(res)
    return c, history
