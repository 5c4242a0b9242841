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


def plan_ceil(k: float, mode_factor: float = 1.6, dir_factor: float = 4.0, newton: int = 1,
              min_leaves: int = 4, leaf_k: float = 0.8, max_leaves: int = 128) -> FrequencyPlan:
    """S = ceil(1.6 k), M = P = ceil(4 k), leaves 2^max(2, ceil(log2(0.8 k))) -- the k = 1..40 sweep's rule."""
    nl = 2 ** max(int(math.log2(min_leaves)), int(math.ceil(math.log2(max(leaf_k * k, 1.0)))))
    return FrequencyPlan(k, min(nl, max_leaves), int(math.ceil(mode_factor * k)), int(math.ceil(dir_factor * k)),
                         int(math.ceil(dir_factor * k)), newton)


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
                            R: float = 3.0, precision: int = HS_FP64, device: int = 0,
                            checkpoint_dir: str | None = None, angles=None) -> SweepResult:
    """Run the sweep.

    plans:   list of FrequencyPlan with increasing k.
    data_fn: data_fn(plan, alphas, thetas) -> measured far field (M x P complex) at plan.k.
    angles:  optional function plan -> (alphas, thetas); default equispaced 2 pi m / M, 2 pi p / P.
    """
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
        key = (p.leaves_per_side, p.S)
        if key not in solvers:
            solvers.clear()  # one tree at a time keeps device memory bounded
            solvers[key] = Solver(p.leaves_per_side, p.S, p.S, R, precision, device)
        solver = solvers[key]
        al, th = angles(p)
        data = data_fn(p, al, th)
        res = []
        for _ in range(p.newton):
            solver.build(c, p.k)
            c, rn = solver.gn_step(data, al, th, lambda_rel, c)
            res.append(rn)
        history.append({"k": p.k, "leaves": p.leaves_per_side, "S": p.S, "M": p.M, "P": p.P, "residuals": res})
        if checkpoint_dir:
            np.save(os.path.join(checkpoint_dir, "c.npy"), c)
            json.dump({"next": j + 1, "history": history}, open(os.path.join(checkpoint_dir, "sweep.json"), "w"))
    for s in solvers.values():
        s.close()
    return SweepResult(c, history)
