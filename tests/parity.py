"""Parity measure shared by the GPU tests.

rel(a, b) is the larger of two relative errors of a against the reference b:
the 2-norm error ||a - b|| / ||b|| and the max-entry error
max |a_i - b_i| / max |b_i|.  A bar on it therefore holds both for the array
as a whole and for every single entry measured against the array's scale, so
a handful of wrong receivers, modes or grid points cannot hide under a small
norm.
"""
import numpy as np


def rel(a, b) -> float:
    a = np.ravel(np.asarray(a))
    b = np.ravel(np.asarray(b))
    d = a - b
    nb = np.linalg.norm(b)
    mb = np.max(np.abs(b)) if b.size else 0.0
    if nb == 0.0 or mb == 0.0:
        return float(np.max(np.abs(d))) if d.size else 0.0
    return float(max(np.linalg.norm(d) / nb, np.max(np.abs(d)) / mb))
