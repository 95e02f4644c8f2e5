"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds only input generation: point clouds shaped like the paper's
workloads (Section 4: s-curve, swiss roll, MNIST; Section 4.2: 6-D Gaussian
clouds) and random right-hand sides. It contains none of the diffusion-map
arithmetic (no kernel, no normalisation, no bandwidth choice), so that the
CUDA path and the FP64 oracle can both consume its output without sharing any
of the method's code.

Every generator draws in float64 with numpy's PCG64 from an explicit seed and
returns a C-contiguous float64 array; ``as_f32`` casts once, so both sides see
identical float32 bytes.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "s_curve",
    "swiss_roll",
    "circle",
    "mnist_like",
    "gaussian_mixture",
    "gaussian_cloud",
    "random_rhs",
    "as_f32",
    "log_uniform_sizes",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def as_f32(a: np.ndarray) -> np.ndarray:
    """Cast to a C-contiguous float32 array (the storage type of the points)."""
    return np.ascontiguousarray(a, dtype=np.float32)


def s_curve(n: int, seed: int = 0, noise: float = 0.01) -> np.ndarray:
    """3-D S-curve (the paper's first dataset, Section 4.1.1).

    Parameter t ~ U[-1.5 pi, 1.5 pi], height h ~ U[0, 2]; the point is
    (sin t, h, sign(t) (cos t - 1)) plus isotropic N(0, noise^2) noise.
    """
    g = _rng(seed)
    t = g.uniform(-1.5 * math.pi, 1.5 * math.pi, size=n)
    h = g.uniform(0.0, 2.0, size=n)
    x = np.stack([np.sin(t), h, np.sign(t) * (np.cos(t) - 1.0)], axis=1)
    x += g.normal(0.0, noise, size=x.shape)
    return np.ascontiguousarray(x)


def swiss_roll(n: int, seed: int = 0, noise: float = 0.01) -> np.ndarray:
    """3-D swiss roll (mentioned with the paper's datasets, Section 4).

    t = 1.5 pi (1 + 2u), u ~ U[0, 1]; y ~ U[0, 21]; point (t cos t, y, t sin t)
    plus N(0, noise^2) noise.
    """
    g = _rng(seed)
    t = 1.5 * math.pi * (1.0 + 2.0 * g.uniform(0.0, 1.0, size=n))
    y = g.uniform(0.0, 21.0, size=n)
    x = np.stack([t * np.cos(t), y, t * np.sin(t)], axis=1)
    x += g.normal(0.0, noise, size=x.shape)
    return np.ascontiguousarray(x)


def circle(n: int, radius: float = 1.0) -> np.ndarray:
    """n equally spaced points on a circle of the given radius in the z=0 plane.

    Deterministic: point j is radius (cos 2 pi j / n, sin 2 pi j / n, 0). The
    Gaussian kernel on these points is circulant, which gives closed-form
    eigenvalues for the tests.
    """
    a = 2.0 * math.pi * np.arange(n) / n
    return np.ascontiguousarray(np.stack([radius * np.cos(a), radius * np.sin(a), np.zeros(n)], axis=1))


def mnist_like(n: int, seed: int = 0, d: int = 784, n_classes: int = 10, subspace: int = 10,
               sparsity_quantile: float = 0.8, pilot: int = 1000) -> np.ndarray:
    """MNIST-shaped synthetic vectors (stand-in for the MNIST runs of Section 4.1.2).

    Class centres c_k ~ N(0, 9 I) in a random `subspace`-dimensional subspace of
    R^d (orthonormal basis from the QR of a Gaussian matrix); a sample is
    B (c_label + N(0, I)), shifted by the `sparsity_quantile` quantile of a
    seeded pilot batch and passed through ReLU (about 80% zeros), divided by
    the pilot maximum, clipped to [0, 1] and quantised to multiples of 1/255.
    No MNIST data is used or reproduced.
    """
    g = _rng(seed)
    basis, _ = np.linalg.qr(g.normal(size=(d, subspace)))
    centres = g.normal(0.0, 3.0, size=(n_classes, subspace))

    def draw(m: int) -> np.ndarray:
        lab = g.integers(0, n_classes, size=m)
        z = centres[lab] + g.normal(size=(m, subspace))
        return z @ basis.T

    u_pilot = draw(pilot)
    tau = float(np.quantile(u_pilot, sparsity_quantile))
    scale = float(np.max(np.maximum(u_pilot - tau, 0.0)))
    u = draw(n)
    v = np.clip(np.maximum(u - tau, 0.0) / scale, 0.0, 1.0)
    return np.ascontiguousarray(np.round(255.0 * v) / 255.0)


def gaussian_mixture(n: int, d: int = 64, seed: int = 0, components: int = 8) -> np.ndarray:
    """Mixture of `components` unit-covariance Gaussians in R^d, means ~ N(0, 4 I)."""
    g = _rng(seed)
    means = g.normal(0.0, 2.0, size=(components, d))
    lab = g.integers(0, components, size=n)
    return np.ascontiguousarray(means[lab] + g.normal(size=(n, d)))


def gaussian_cloud(n: int, d: int = 6, seed: int = 0) -> np.ndarray:
    """Standard normal points in R^d (the 6-D synthetic kernel of Section 4.2)."""
    return np.ascontiguousarray(_rng(seed).normal(size=(n, d)))


def random_rhs(n: int, nrhs: int = 1, seed: int = 1) -> np.ndarray:
    """Right-hand sides, uniform in [-1, 1], shape (n, nrhs) in column-major order."""
    x = _rng(seed).uniform(-1.0, 1.0, size=(nrhs, n))
    return np.asfortranarray(x.T)


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """`count` integers log-uniform in [lo, hi] (the batched and serving mixes)."""
    g = _rng(seed)
    return np.floor(np.exp(g.uniform(math.log(lo), math.log(hi + 1), size=count))).astype(np.int64)
