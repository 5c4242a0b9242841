"""Recursive linearization over frequency (Sec. 3.4, "Recursive Linearization using Newton's method").

Host-side driver: for k_1 < k_2 < ... < k_Q it builds the discretisation
for each frequency (quadtree size, sine band limit, incidences, receivers),
starts Newton's method at k_j from the contrast found at k_{j-1} (the sine
coefficients carried into the larger basis), and takes Gauss-Newton steps
with the library (hs_build + hs_gn_step, eq. normaleq).  Every step runs on
the GPU through the C ABI; the driver only moves coefficient arrays.

Checkpoint/resume: with ``checkpoint_dir`` set, the coefficients and the
residual history are saved after every frequency and a later call resumes at
the first frequency not yet done.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import HS_FP64, Solver


@dataclass
class FrequencyPlan:
    """Discretisation at one frequency."""

    k: float
    leaves_per_side: int
    S: int       # sine modes per axis
    M: int       # incidences
    P: int       # receivers
    newton: int  # Gauss-Newton steps
    R: float = 3.0                 # receiver radius on [-1, 1]^2
    triangle: int = 0              # > 0: only modes m1 + m2 <= triangle are unknowns
    k_label: float | None = None   # the frequency in the paper's units, when rescaled

    def mask(self):
        if self.triangle <= 0:
            return None
        m = np.arange(1, self.S + 1)
        return (m[:, None] + m[None, :]) <= self.triangle


def plan_ceil(k: float, mode_factor: float = 1.6, dir_factor: float = 4.0, newton: int = 1,
              min_leaves: int = 4, leaf_k: float = 0.8, max_leaves: int = 128) -> FrequencyPlan:
    """S = ceil(1.6 k), M = P = ceil(4 k), leaves 2^max(2, ceil(log2(0.8 k))) -- the k = 1..40 sweep's rule."""
    nl = 2 ** max(int(math.log2(min_leaves)), int(math.ceil(math.log2(max(leaf_k * k, 1.0)))))
    return FrequencyPlan(k, min(nl, max_leaves), int(math.ceil(mode_factor * k)), int(math.ceil(dir_factor * k)),
                         int(math.ceil(dir_factor * k)), newton)


def square_eigenvalues(lo: float, hi: float, unit: float = 1.0) -> list:
    """Dirichlet eigenvalues unit * sqrt(a^2 + b^2) (a, b >= 1) in [lo, hi]: those of the square
    [-pi/2, pi/2]^2 for unit = 1, of [-1, 1]^2 for unit = pi/2."""
    if unit != 1.0:
        return [unit * e for e in square_eigenvalues(lo / unit, hi / unit)]
    out = set()
    for a in range(1, int(math.floor(hi)) + 1):
        blo = math.sqrt(max(lo * lo - a * a, 1.0))
        for b in range(max(1, int(math.floor(blo))), int(math.floor(math.sqrt(max(hi * hi - a * a, 0.0)))) + 1):
            v = math.hypot(a, b)
            if lo <= v <= hi:
                out.add(v)
    return sorted(out)


def square_safe(k: float, near: float = 0.002, window: float = 0.02, unit: float = 1.0) -> float:
    """The paper's frequency on its square [-pi/2, pi/2]^2, moved when it lies within `near`
    of a Dirichlet eigenvalue sqrt(a^2 + b^2) (a, b >= 1) of that square: the exterior
    relation (D - I/2) u = S d_n u of Sec. 2 (the paper's T_ext = S^{-1}(D - I/2)) is
    singular there, and the paper's grid k = 1 + j/4 hits it exactly at every integer k
    that is the hypotenuse of a Pythagorean triple (5, 10, 13, 15, ...).  The new frequency
    is the midpoint of the widest gap between eigenvalues within `window` of k.  With
    unit = pi/2 the same for a frequency on [-1, 1]^2 (eigenvalues (pi/2) sqrt(a^2 + b^2))."""
    ev = square_eigenvalues(k - window, k + window, unit)
    if not ev or min(abs(e - k) for e in ev) >= near:
        return k
    pts = [k - window] + ev + [k + window]
    gaps = [(pts[i + 1] - pts[i], 0.5 * (pts[i] + pts[i + 1])) for i in range(len(pts) - 1)]
    return max(gaps)[1]


def plan_paper(k: float, R: float = 20.0, leaf_kh: float = 2.5, min_leaves: int = 4,
               max_leaves: int = 128, avoid_resonance: bool = True) -> FrequencyPlan:
    """The paper's experiment plan (Sec. 4) at its frequency k on its domain
    [-pi/2, pi/2]^2, read on [-1, 1]^2 by x = (pi/2) x_hat: the wavenumber becomes
    pi k / 2 and the receiver radius 2 R / pi (R = 20); M = floor(2k) incidences,
    P = floor(4k) receivers, unknowns the sine modes m1 + m2 <= floor(2k) (the
    basis sin(m (x + pi/2)) is sin(m pi (x_hat + 1) / 2)); one Gauss-Newton step.
    Leaves: the smallest power of two with (pi k / 2) h <= leaf_kh (h = 2 / n_L),
    which keeps the leaf Dirichlet blocks well away from resonance (the paper's
    own rule, 6-10 points per wavelength, is coarser).  Frequencies within 0.002
    of the square's Dirichlet eigenvalues are moved off them (square_safe), unless
    avoid_resonance is False (for solvers with combined-field exterior rows,
    bm_eta > 0, which are solvable there)."""
    kh = math.pi * (square_safe(k) if avoid_resonance else k) / 2.0
    nl = max(min_leaves, 2 ** int(math.ceil(math.log2(max(2.0 * kh / leaf_kh, 1.0)))))
    S = int(math.floor(2.0 * k))
    return FrequencyPlan(kh, min(nl, max_leaves), max(S - 1, 1), int(math.floor(2.0 * k)),
                         int(math.floor(4.0 * k)), 1, R=2.0 * R / math.pi, triangle=S, k_label=k)


def plan_table1(k: float, M: int = 64, R: float = 20.0) -> FrequencyPlan:
    """The forward benchmark of the paper's Table 1 (Sec. 2) at its frequency k in
    {1, 2, 4, ..., 128} on [-pi/2, pi/2]^2, read on [-1, 1]^2 like plan_paper
    (wavenumber pi k / 2, receiver radius 2 R / pi): max(4, k) x max(4, k) leaves of
    16 x 16 points, i.e. the table's N = (15 n_L + 1)^2 (3721 for k <= 4, 3,690,241 at
    k = 128) and a leaf of width pi / k (k h = pi, half a free-space wavelength).  The
    table's contrast is q = 1.5 exp(-|x|^2 / 50), read as entering with the opposite
    sign (synth.paper_example(1)): k sqrt(1 - q) h is then 4.83..4.97, between the
    first two Dirichlet eigenvalues pi sqrt(2), pi sqrt(5) of a leaf, so the leaf
    interior blocks stay nonsingular.  M incidences and M receivers time the solves."""
    nl = max(4, int(round(k)))
    return FrequencyPlan(math.pi * k / 2.0, nl, 1, M, M, 0, R=2.0 * R / math.pi, k_label=k)


def plan_c5(k: float, avoid_resonance: bool = True) -> FrequencyPlan:
    """The paper-scale reconstruction plan on [-1, 1]^2: S = floor(2k) sine modes per axis
    (140 x 140 = 19,600 at k = 70), M = P = ceil(4k) (280 at k = 70), leaves
    2^min(7, max(2, ceil(log2(128 k / 70)))) (128 x 128 at the top), one Gauss-Newton step;
    frequencies within 0.002 of a Dirichlet eigenvalue of the square are moved off it
    (square_safe with unit pi/2; the grid comes within 2e-5 of one at k = 40.75), unless
    avoid_resonance is False (combined-field exterior rows)."""
    nl = 2 ** min(7, max(2, int(math.ceil(math.log2(128.0 * k / 70.0)))))
    ks = square_safe(k, unit=math.pi / 2.0) if avoid_resonance else k
    return FrequencyPlan(ks, nl, int(math.floor(2.0 * k)), int(math.ceil(4.0 * k)), int(math.ceil(4.0 * k)), 1,
                         k_label=k)


def solver_kind_lsqr(solver_name: str) -> bool:
    if solver_name not in ("direct", "lsqr"):
        raise ValueError("solver must be 'direct' or 'lsqr'")
    return solver_name == "lsqr"


def embed(c: np.ndarray, S1: int, S2: int) -> np.ndarray:
    """Coefficients of a smaller band limit carried into an S1 x S2 basis (new modes start at 0)."""
    out = np.zeros((S1, S2))
    a, b = min(S1, c.shape[0]), min(S2, c.shape[1])
    out[:a, :b] = c[:a, :b]
    return out


@dataclass
class SweepResult:
    c: np.ndarray
    history: list = field(default_factory=list)


def recursive_linearization(plans, data_fn, lambda_rel: float = 1e-4, c0: np.ndarray | None = None,
                            R: float | None = None, precision: int = HS_FP64, device: int = 0,
                            checkpoint_dir: str | None = None, angles=None, solver: str = "direct",
                            lsqr_tol: float = 1e-3, lsqr_max_iter: int = 200,
                            lsqr_products: int = HS_FP64, bm_eta: float = 0.0,
                            leaf_impedance: bool = False) -> SweepResult:
    """Run the sweep.

    plans:   list of FrequencyPlan with increasing k.
    data_fn: data_fn(plan, alphas, thetas) -> measured far field (M x P complex) at plan.k.
    angles:  optional function plan -> (alphas, thetas); default equispaced 2 pi m / M, 2 pi p / P.
    solver:  "direct" (normal equations with lambda_rel, hs_gn_step) or "lsqr" (the paper's
             LSQR at lsqr_tol on the plan's modes, hs_gn_step_lsqr, products in lsqr_products).
    precision: HS_FP64, or HS_MIXED (FP32 factors; forward and adjoint fields refined in FP64).
    R:       receiver radius overriding the plans' own.
    bm_eta:  exterior rows of every solver (hs_config.bm_eta): 0 Green's identity, > 0 the
             combined-field rows, solvable at the square's Dirichlet eigenvalues.
    leaf_impedance: leaf elimination of every solver (hs_config.leaf_impedance): through the
             leaf's impedance system, solvable at every k h (plans with coarser leaves,
             e.g. plan_paper(k, leaf_kh=math.pi)), instead of the Dirichlet block.
    Each history entry records the build (factorisation) time t_f and the
    least-squares time t_l of every step in seconds, and the LSQR iterations.
    """
    use_lsqr = solver_kind_lsqr(solver)
    if angles is None:
        angles = lambda p: (2 * np.pi * np.arange(p.M) / p.M, 2 * np.pi * np.arange(p.P) / p.P)
    c = np.zeros((plans[0].S, plans[0].S)) if c0 is None else np.asarray(c0, dtype=np.float64)
    history = []
    start = 0
    if checkpoint_dir:
        os.makedirs(checkpoint_dir, exist_ok=True)
        meta = os.path.join(checkpoint_dir, "sweep.json")
        if os.path.exists(meta):
            saved = json.load(open(meta))
            start = saved["next"]
            history = saved["history"]
            c = np.load(os.path.join(checkpoint_dir, "c.npy"))
    solvers = {}
    for j in range(start, len(plans)):
        p = plans[j]
        c = embed(c, p.S, p.S)
        radius = p.R if R is None else R
        key = (p.leaves_per_side, p.S, radius)
        if key not in solvers:
            for old in solvers.values():
                old.close()
            solvers.clear()  # one tree at a time keeps device memory bounded
            solvers[key] = Solver(p.leaves_per_side, p.S, p.S, radius, precision, device, bm_eta=bm_eta,
                                  leaf_impedance=leaf_impedance)
        slv = solvers[key]
        al, th = angles(p)
        data = data_fn(p, al, th)
        res, t_f, t_l, its = [], [], [], []
        for _ in range(p.newton):
            t0 = time.perf_counter()
            slv.build(c, p.k)
            t1 = time.perf_counter()
            if use_lsqr:
                c, rn, it = slv.gn_step_lsqr(data, al, th, c, mask=p.mask(), tol=lsqr_tol, max_iter=lsqr_max_iter,
                                             products=lsqr_products)
                its.append(it)
            else:
                c, rn = slv.gn_step(data, al, th, lambda_rel, c)
            t2 = time.perf_counter()
            res.append(rn)
            t_f.append(t1 - t0)
            t_l.append(t2 - t1)
        modes = int(p.mask().sum()) if p.triangle > 0 else p.S * p.S
        history.append({"k": p.k if p.k_label is None else p.k_label, "k_solver": p.k,
                        "leaves": p.leaves_per_side, "N": (15 * p.leaves_per_side + 1) ** 2, "S": p.S,
                        "modes": modes, "M": p.M, "P": p.P, "residuals": res, "t_f": t_f, "t_l": t_l,
                        "lsqr_iterations": its})
        if checkpoint_dir:
            np.save(os.path.join(checkpoint_dir, "c.npy"), c)
            json.dump({"next": j + 1, "history": history}, open(os.path.join(checkpoint_dir, "sweep.json"), "w"))
    for s in solvers.values():
        s.close()
    return SweepResult(c, history)
