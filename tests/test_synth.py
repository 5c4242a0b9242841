"""Seeded input generators (no method arithmetic): determinism and the properties the
workloads rely on (1 - q > 0 for the contrasts, the stated amplitude scalings, the noise
level of Sec. 4)."""
import math

import numpy as np

import synth


def grid(n=401):
    t = np.linspace(-1.0, 1.0, n)
    return np.meshgrid(t, t, indexing="ij")


def series(c, X):
    S1, S2 = c.shape
    t = X[:, 0]
    b1 = np.sin(np.outer(np.arange(1, S1 + 1), t + 1.0) * math.pi / 2)
    b2 = np.sin(np.outer(np.arange(1, S2 + 1), t + 1.0) * math.pi / 2)
    return b1.T @ c @ b2


def test_generators_are_seeded():
    assert np.array_equal(synth.smooth_random_coeffs(12, seed=2), synth.smooth_random_coeffs(12, seed=2))
    assert not np.array_equal(synth.smooth_random_coeffs(12, seed=2), synth.smooth_random_coeffs(12, seed=3))
    X, Y = grid(64)
    assert np.array_equal(synth.inclusions(5)(X, Y), synth.inclusions(5)(X, Y))
    assert np.array_equal(synth.ellipse_phantom(7)(X, Y), synth.ellipse_phantom(7)(X, Y))


def test_contrasts_keep_one_minus_q_positive():
    X, Y = grid()
    c = synth.smooth_random_coeffs(40, seed=2, qmax=0.3)
    assert abs(np.abs(series(c, X)).max() - 0.3) < 5e-3  # scaled on a 513 grid, checked on 401
    for q in (synth.gaussian_bumps(1)(X, Y), synth.ellipse_phantom(3)(X, Y), synth.ellipse_phantom(7)(X, Y),
              synth.paper_example(1)(X, Y), synth.paper_example(2)(X, Y)):
        assert (1.0 - q).min() > 0.0
    ci = synth.scaled_sine_coeffs(synth.inclusions(5), 140, 0.5)
    qi = series(ci, X)
    assert abs(np.abs(qi).max() - 0.5) < 1e-3 and (1.0 - qi).min() > 0.0  # scaled on a 1025 grid


def test_paper_examples_on_their_domain():
    # Example 2 at a point, straight from its formula on [-pi/2, pi/2]^2 (sigma = 0.5)
    x, y, s = 0.3, -0.2, 0.5
    ref = (0.15 * (1 - x / s) ** 2 * math.exp(-((x / s) ** 2 + (y / s + 1) ** 2))
           - math.exp(-((y / s) ** 2 + (x / s + 1) ** 2)) / 60
           - s * (0.4 * x - (x / s) ** 3 - (y / s) ** 5) * math.exp(-(x * x + y * y) / s ** 2))
    assert abs(synth.paper_example(2)(x / (math.pi / 2), y / (math.pi / 2)) - ref) < 1e-15
    assert abs(synth.paper_example(1)(0.0, 0.0) + 1.5) < 1e-15


def test_noise_level():
    rng = np.random.default_rng(0)
    u = rng.standard_normal((6, 50)) + 1j * rng.standard_normal((6, 50))
    n = synth.add_noise(u, 0.05, seed=70)
    rel = np.linalg.norm(n - u, axis=1) / np.linalg.norm(u, axis=1)
    assert np.allclose(rel, 0.05, rtol=1e-12)
