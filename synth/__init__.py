"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds only input generation: contrasts q(x) given as plain
functions of position, sine-coefficient arrays, incidence angles and receiver
angles.  It contains none of the solver's arithmetic (no discretisation, no
Green's functions, no linear algebra), so that the CUDA path and the CPU
oracle can both draw their inputs from it without sharing any method code.

Workloads follow the paper's experiments (Sec. 4): plane-wave incidence from
equispaced directions d_m = (cos 2 pi m/M, sin 2 pi m/M) and receivers at
x_p = R (cos 2 pi p/P, sin 2 pi p/P) on a circle of radius R enclosing the
domain Omega = [-1, 1]^2; contrasts are smooth bumps or blurred inclusions of
the amplitudes used there, scaled so that 1 - q stays positive (Sec. 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "GaussianBumps",
    "gaussian_bumps",
    "smooth_random_coeffs",
    "directions",
    "receivers",
    "random_coeffs",
    "WORKLOADS",
    "Workload",
]


@dataclass(frozen=True)
class GaussianBumps:
    """q(x) = sum_i a_i exp(-|x - c_i|^2 / (2 w_i^2)) restricted to Omega."""

    centres: np.ndarray  # (n, 2)
    widths: np.ndarray   # (n,)
    amps: np.ndarray     # (n,)

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros(np.broadcast(x, y).shape)
        for (cx, cy), w, a in zip(self.centres, self.widths, self.amps):
            out = out + a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * w * w))
        inside = (np.abs(x) <= 1.0) & (np.abs(y) <= 1.0)
        return np.where(inside, out, 0.0)


def gaussian_bumps(seed: int = 1, n: int = 3, centre_box: float = 0.6,
                   width_range=(0.15, 0.3), amp_range=(0.1, 0.4)) -> GaussianBumps:
    """Sum of `n` Gaussian bumps with seeded centres, widths and amplitudes.

    Defaults: 3 bumps, centres U[-0.6, 0.6]^2, widths U[0.15, 0.3],
    amplitudes U[0.1, 0.4] (so max q < 1.2 only if bumps overlap strongly;
    1 - q > 0 is checked by the caller).
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-centre_box, centre_box, size=(n, 2))
    widths = rng.uniform(*width_range, size=n)
    amps = rng.uniform(*amp_range, size=n)
    return GaussianBumps(centres, widths, amps)


def smooth_random_coeffs(S: int, seed: int = 2, decay: float = 8.0,
                         qmax: float = 0.3, grid: int = 513) -> np.ndarray:
    """Sine coefficients c[m1-1, m2-1] ~ N(0,1) exp(-|m|/decay), |m| = sqrt(m1^2+m2^2).

    The array is scaled so that max |q| over a uniform `grid` x `grid` sample of
    Omega equals `qmax`, where q(x) = sum c[m1,m2] sin(m1 pi (x1+1)/2) sin(m2 pi (x2+1)/2)
    is the band-limited contrast of Sec. 3.2 (eq. sineseries) on [-1,1]^2.
    """
    rng = np.random.default_rng(seed)
    m = np.arange(1, S + 1, dtype=np.float64)
    mag = np.sqrt(m[:, None] ** 2 + m[None, :] ** 2)
    c = rng.standard_normal((S, S)) * np.exp(-mag / decay)
    t = np.linspace(-1.0, 1.0, grid)
    basis = np.sin(np.outer(m, t + 1.0) * (math.pi / 2.0))  # (S, grid)
    q = basis.T @ c @ basis
    return c * (qmax / np.max(np.abs(q)))


def random_coeffs(S1: int, S2: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Plain N(0, scale^2) coefficients (S1, S2) for perturbation tests."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((S1, S2))


@dataclass(frozen=True)
class EllipsePhantom:
    """Sum of ellipses with blurred edges: c_i * erfc(rho_i / (sqrt(2) w)) / 2, clipped at `clip`.

    rho_i = (sqrt((x'/a)^2 + (y'/b)^2) - 1) * min(a, b) in the ellipse's frame.
    """

    centres: np.ndarray
    axes: np.ndarray
    angles: np.ndarray
    contrasts: np.ndarray
    blur: float
    clip: float

    def __call__(self, x, y):
        from scipy.special import erfc
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros(np.broadcast(x, y).shape)
        for (cx, cy), (a, b), th, cval in zip(self.centres, self.axes, self.angles, self.contrasts):
            ct, st = math.cos(th), math.sin(th)
            xr = (x - cx) * ct + (y - cy) * st
            yr = -(x - cx) * st + (y - cy) * ct
            rho = (np.sqrt((xr / a) ** 2 + (yr / b) ** 2) - 1.0) * min(a, b)
            out = out + cval * 0.5 * erfc(rho / (math.sqrt(2.0) * self.blur))
        out = np.minimum(out, self.clip)
        inside = (np.abs(x) <= 1.0) & (np.abs(y) <= 1.0)
        return np.where(inside, out, 0.0)


def ellipse_phantom(seed: int = 3, n: int = 5, centre_box: float = 0.6, axes=(0.08, 0.35),
                    contrast=(0.05, 0.3), blur: float = 0.05, clip: float = 0.3) -> EllipsePhantom:
    """Seeded blurred-ellipse phantom (stand-in for the paper's head/thorax phantoms, Sec. 4)."""
    rng = np.random.default_rng(seed)
    return EllipsePhantom(rng.uniform(-centre_box, centre_box, size=(n, 2)), rng.uniform(*axes, size=(n, 2)),
                          rng.uniform(0.0, math.pi, size=n), rng.uniform(*contrast, size=n), blur, clip)


@dataclass(frozen=True)
class Inclusions:
    """Sum of contrast functions (Gaussian bumps and blurred ellipses), times `scale`."""

    parts: tuple
    scale: float = 1.0

    def __call__(self, x, y):
        out = 0.0
        for f in self.parts:
            out = out + f(x, y)
        return self.scale * out


def inclusions(seed: int = 5, n: int = 40, centre_box: float = 0.7) -> Inclusions:
    """Seeded random sum of n inclusions, half Gaussian bumps (widths U[0.03, 0.12],
    amplitudes U[0.1, 1]) and half blurred ellipses (semi-axes U[0.04, 0.2], contrast
    U[0.1, 1], edge blur 0.02), centres U[-0.7, 0.7]^2 (the paper-scale reconstruction
    contrast; scale it with `scaled_sine_coeffs`)."""
    rng = np.random.default_rng(seed)
    ng = n // 2
    ne = n - ng
    bumps = GaussianBumps(rng.uniform(-centre_box, centre_box, size=(ng, 2)), rng.uniform(0.03, 0.12, size=ng),
                          rng.uniform(0.1, 1.0, size=ng))
    ell = EllipsePhantom(rng.uniform(-centre_box, centre_box, size=(ne, 2)), rng.uniform(0.04, 0.2, size=(ne, 2)),
                         rng.uniform(0.0, math.pi, size=ne), rng.uniform(0.1, 1.0, size=ne), 0.02, np.inf)
    return Inclusions((bumps, ell))


def scaled_sine_coeffs(qfun, S: int, qmax: float, nq: int = 640, grid: int = 1025) -> np.ndarray:
    """Projection of q onto S x S sine modes, scaled so that max |q_S| over a uniform
    `grid` x `grid` sample of Omega equals qmax (q_S the band-limited series, eq. sineseries)."""
    c = project_sine(qfun, S, S, nq)
    t = np.linspace(-1.0, 1.0, grid)
    basis = np.sin(np.outer(np.arange(1, S + 1), t + 1.0) * (math.pi / 2.0))
    q = basis.T @ c @ basis
    return c * (qmax / np.max(np.abs(q)))


@dataclass(frozen=True)
class PaperExample:
    """The contrast of the paper's Example 1 (a single Gaussian) or Example 2 (a sum of
    Hermite functions, sigma = 0.5), Sec. 4, given on [-pi/2, pi/2]^2 and evaluated here on
    [-1, 1]^2 through x = (pi/2) x_hat.  Example 1's printed contrast 1.5 exp(-|x|^2/50)
    would make 1 - q negative everywhere under the equation of Sec. 1; it is read as
    entering with the opposite sign, q = -1.5 exp(-|x|^2/50) (refractive index squared
    1 + 1.5 exp(...))."""

    which: int

    def paper_q(self, x, y):
        if self.which == 1:
            return -1.5 * np.exp(-(x * x + y * y) / 50.0)
        s = 0.5
        xs, ys = x / s, y / s
        return (0.15 * (1.0 - xs) ** 2 * np.exp(-(xs ** 2 + (ys + 1.0) ** 2))
                - np.exp(-(ys ** 2 + (xs + 1.0) ** 2)) / 60.0
                - s * (0.4 * x - xs ** 3 - ys ** 5) * np.exp(-(x * x + y * y) / (s * s)))

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = self.paper_q(0.5 * math.pi * x, 0.5 * math.pi * y)
        inside = (np.abs(x) <= 1.0) & (np.abs(y) <= 1.0)
        return np.where(inside, out, 0.0)


def paper_example(which: int) -> PaperExample:
    if which not in (1, 2):
        raise ValueError("the paper's analytic examples are 1 and 2")
    return PaperExample(which)


def project_sine(qfun, S1: int, S2: int, nq: int = 256) -> np.ndarray:
    """Coefficients of the L2 projection of q onto s_m1(x) s_m2(y) on [-1,1]^2 (Gauss-Legendre, nq^2 points).

    The basis is orthogonal with int_{-1}^{1} s_m^2 = 1, so c = int q s_m1 s_m2.
    """
    from scipy.special import roots_legendre
    t, w = roots_legendre(nq)
    X, Y = np.meshgrid(t, t, indexing="ij")
    Q = qfun(X, Y) * np.outer(w, w)
    sx = np.sin(np.outer(np.arange(1, S1 + 1), t + 1.0) * (math.pi / 2.0))
    sy = np.sin(np.outer(np.arange(1, S2 + 1), t + 1.0) * (math.pi / 2.0))
    return sx @ Q @ sy.T


def add_noise(u: np.ndarray, delta: float, seed: int) -> np.ndarray:
    """Noisy data of Sec. 4: per incidence row u_d, u_d + delta ||u_d|| / ||eps|| eps, eps = eps1 + i eps2 ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    u = np.asarray(u, dtype=np.complex128)
    eps = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    scale = delta * np.linalg.norm(u, axis=-1, keepdims=True) / np.linalg.norm(eps, axis=-1, keepdims=True)
    return u + scale * eps


def directions(M: int) -> np.ndarray:
    """Incidence angles alpha_m = 2 pi m / M, m = 0..M-1 (d = (cos, sin))."""
    return 2.0 * math.pi * np.arange(M, dtype=np.float64) / M


def receivers(P: int) -> np.ndarray:
    """Receiver angles theta_p = 2 pi p / P, p = 0..P-1 on the circle of radius R."""
    return 2.0 * math.pi * np.arange(P, dtype=np.float64) / P


@dataclass(frozen=True)
class Workload:
    name: str
    k: float
    n_leaf_side: int
    S: int
    M: int
    P: int
    R: float = 3.0


# The workloads the tests and the benchmark use (sizes of the paper-shaped runs).
WORKLOADS = {
    # one Gauss-Newton step at k = 5 from q = 0, data from 3 Gaussian bumps
    "gn_k5": Workload("gn_k5_4x4leaves_100modes_16dirs_32recv", 5.0, 4, 10, 16, 32),
    # forward-only batched solve at k = 40 on 32 x 32 leaves
    "fwd_k40": Workload("fwd_k40_32x32leaves_128dirs_256recv", 40.0, 32, 40, 128, 256),
    # misfit gradient at k = 20 (1600 coefficients)
    "grad_k20": Workload("grad_k20_16x16leaves_1600modes_64dirs_128recv", 20.0, 16, 40, 64, 128),
    # one Gauss-Newton step at the top frequency of the k = 1..40 sweep:
    # S = ceil(1.6 k) = 64 modes per axis, M = P = ceil(4 k) = 160, 32 x 32 leaves
    "gn_k40": Workload("gn_k40_32x32leaves_4096modes_160dirs_160recv", 40.0, 32, 64, 160, 160),
    # forward batch at the top frequency of the paper-scale sweep: 140 x 140 = 19,600
    # sine unknowns, 128 x 128 leaves (N = (15*128 + 1)^2 = 3,690,241 distinct points),
    # 280 incidences and receivers
    "fwd_k70": Workload("fwd_k70_128x128leaves_19600modes_280dirs_280recv", 70.0, 128, 140, 280, 280),
}
