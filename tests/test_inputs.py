"""The seeded input generators follow the recipes stated for the workloads: shapes,
ranges, value grids, sparsity, determinism per seed."""
import math

import numpy as np

import synth


def test_same_seed_same_bytes_other_seed_other_points():
    a, b = synth.as_f32(synth.s_curve(1000, seed=3)), synth.as_f32(synth.s_curve(1000, seed=3))
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] and a.shape == (1000, 3)
    assert a.tobytes() == b.tobytes()
    assert not np.array_equal(a, synth.as_f32(synth.s_curve(1000, seed=4)))


def test_s_curve_lies_on_the_surface_up_to_the_noise():
    X = synth.s_curve(20_000, seed=0, noise=0.0)
    x, h, z = X[:, 0], X[:, 1], X[:, 2]
    t = np.arcsin(np.clip(x, -1, 1))
    # (sin t, h, sign(t)(cos t - 1)): |z| = 1 - cos t for some t with sin t = x
    assert np.all((h >= 0) & (h <= 2))
    assert np.all(np.abs(x) <= 1) and np.all(np.abs(z) <= 2 + 1e-12)
    c = 1.0 - np.abs(z)  # cos t
    np.testing.assert_allclose(x ** 2 + c ** 2, 1.0, atol=1e-12)
    assert np.abs(np.mean(t)) < 0.05  # symmetric parameter range
    noisy = synth.s_curve(20_000, seed=0)
    assert 0.008 < np.std(noisy - X) < 0.012  # N(0, 0.01^2) per coordinate


def test_swiss_roll_radius_is_its_parameter():
    X = synth.swiss_roll(5000, seed=1, noise=0.0)
    r = np.hypot(X[:, 0], X[:, 2])
    assert r.min() >= 1.5 * math.pi - 1e-9 and r.max() <= 4.5 * math.pi + 1e-9
    assert X[:, 1].min() >= 0 and X[:, 1].max() <= 21


def test_mnist_like_grid_range_and_sparsity():
    X = synth.mnist_like(3000, seed=2)
    assert X.shape == (3000, 784)
    assert X.min() >= 0.0 and X.max() <= 1.0
    k = X * 255.0
    np.testing.assert_allclose(k, np.round(k), atol=1e-9)  # multiples of 1/255
    X32 = synth.as_f32(X)
    assert np.array_equal(np.rint(X32.astype(np.float64) * 255.0), np.round(k))  # 8-bit codes survive FP32
    zeros = float(np.mean(X == 0.0))
    assert 0.7 < zeros < 0.9  # about 80% zeros
    # rows come from a 10-dimensional subspace before the ReLU: most of the centred data's
    # energy stays in 10 directions
    sv = np.linalg.svd(X[:1000] - X[:1000].mean(0), compute_uv=False)
    assert (sv[:10] ** 2).sum() > 0.75 * (sv ** 2).sum()


def test_mixture_cloud_rhs_and_sizes():
    M = synth.gaussian_mixture(4000, d=64, seed=5)
    assert M.shape == (4000, 64)
    C = synth.gaussian_cloud(50_000, d=6, seed=6)
    assert abs(C.mean()) < 0.02 and abs(C.std() - 1.0) < 0.02
    R = synth.random_rhs(1000, 7, seed=8)
    assert R.shape == (1000, 7) and R.flags["F_CONTIGUOUS"]
    assert R.min() >= -1.0 and R.max() <= 1.0
    s = synth.log_uniform_sizes(5000, 1000, 32_000, seed=9)
    assert s.min() >= 1000 and s.max() <= 32_000
    # log-uniform: about a fifth of the sizes in each doubling of [1k, 32k]
    frac = np.mean((s >= 4000) & (s < 8000))
    assert 0.17 < frac < 0.23
