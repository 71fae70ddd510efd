"""Seeded synthetic inputs shaped like the paper's workloads.

Only input generation lives here -- random images and direction sets -- and none of
the transforms' arithmetic, so that the CPU oracle and the CUDA path can be fed the
same bytes.  Everything is numpy on the host, deterministic for a given seed.

Image arrays are C-ordered numpy arrays whose LAST axis is the paper's coordinate 0
(the fastest memory axis).

Workloads (Section 5 uses Fashion-MNIST and random images; the dataset is not
available, so these stand in for it):

* ``bernoulli``: i.i.d. Bernoulli(p) binary image.
* ``grf``: Gaussian random field -- white noise convolved (periodically, by FFT) with a
  Gaussian of standard deviation ell / sqrt(2), so that the field's covariance is
  exp(-r^2 / (2 ell^2)); standardised, then either quantised to 0..255 through the
  normal CDF (``floor(256 Phi(z))`` clipped) or thresholded at 0 (binary).
* ``blurred_noise``: uniform 0..255 noise blurred by a Gaussian (reflecting
  boundary), rounded and clipped -- Fashion-MNIST-like grey levels.
* ragged side lengths log-uniform in [lo, hi].
* direction sets: evenly spaced on S^1, Fibonacci points on S^2, random angles with
  log-uniform or uniform norms, Gaussian perturbations.
"""
from __future__ import annotations

import math

import numpy as np


def bernoulli(shape, p: float = 0.5, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.random(shape) < p).astype(np.uint8)


def uniform_u8(shape, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=shape, dtype=np.uint8)


def _std_normal_cdf(z: np.ndarray) -> np.ndarray:
    from scipy.special import ndtr
    return ndtr(z)


def grf_field(shape, ell: float, seed: int) -> np.ndarray:
    """Standardised Gaussian random field with covariance exp(-r^2 / (2 ell^2))."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    sigma = ell / math.sqrt(2.0)
    F = np.fft.rfftn(w)
    # Fourier transform of a unit-mass Gaussian kernel of std sigma
    freq2 = np.zeros(F.shape)
    for ax, m in enumerate(shape):
        if ax == len(shape) - 1:
            f = np.fft.rfftfreq(m)
        else:
            f = np.fft.fftfreq(m)
        sh = [1] * len(shape)
        sh[ax] = len(f)
        freq2 = freq2 + (f.reshape(sh) ** 2)
    F *= np.exp(-2.0 * (math.pi ** 2) * (sigma ** 2) * freq2)
    z = np.fft.irfftn(F, s=shape, axes=tuple(range(len(shape))))
    z -= z.mean()
    sd = z.std()
    return z / sd if sd > 0 else z


def grf(shape, ell: float, seed: int, binary: bool = False) -> np.ndarray:
    z = grf_field(shape, ell, seed)
    if binary:
        return (z >= 0.0).astype(np.uint8)
    q = np.floor(256.0 * _std_normal_cdf(z))
    return np.clip(q, 0, 255).astype(np.uint8)


def blurred_noise(shape, sigma: float, seed: int) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 256, size=shape).astype(np.float64)
    b = gaussian_filter(u, sigma=sigma, mode="reflect")
    return np.clip(np.rint(b), 0, 255).astype(np.uint8)


def ragged_shapes(count: int, lo: int, hi: int, seed: int) -> list:
    """(h, w) pairs, each side floor(exp(U[ln lo, ln (hi + 1)))), independent."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi + 1), size=(count, 2))
    sides = np.floor(np.exp(u)).astype(np.int64)
    sides = np.clip(sides, lo, hi)
    return [(int(h), int(w)) for h, w in sides]


def circle_dirs(D: int, radius: float = 1.0) -> np.ndarray:
    """xi_k = radius (cos 2 pi k / D, sin 2 pi k / D): [D, 2]."""
    th = 2.0 * math.pi * np.arange(D) / D
    return radius * np.stack([np.cos(th), np.sin(th)], axis=1)


def random_2d_dirs(D: int, seed: int, rmin: float, rmax: float, log_norm: bool = True) -> np.ndarray:
    """Uniform angle, norm log-uniform (or uniform) in [rmin, rmax]: [D, 2]."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 2.0 * math.pi, size=D)
    if log_norm:
        r = np.exp(rng.uniform(math.log(rmin), math.log(rmax), size=D))
    else:
        r = rng.uniform(rmin, rmax, size=D)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def fibonacci_dirs(D: int) -> np.ndarray:
    """Fibonacci lattice on S^2: z_k = 1 - (2k+1)/D, angle k pi (3 - sqrt 5): [D, 3]."""
    k = np.arange(D, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / D
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ang = k * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(ang), r * np.sin(ang), z], axis=1)


def sphere_dirs(D: int, seed: int, rmin: float, rmax: float) -> np.ndarray:
    """Uniform on S^2 times a norm uniform in [rmin, rmax]: [D, 3]."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((D, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = rng.uniform(rmin, rmax, size=(D, 1))
    return g * r


def scale_norms(dirs: np.ndarray, seed: int, rmin: float, rmax: float) -> np.ndarray:
    """Give unit directions norms uniform in [rmin, rmax]."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(rmin, rmax, size=(dirs.shape[0], 1))
    return dirs * r


def perturb(dirs: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return dirs + sigma * rng.standard_normal(dirs.shape)


def image_radius(n: int) -> float:
    """max_v |x(v)| for vertices in [-0.5, 0.5]^n: sqrt(n) / 2."""
    return math.sqrt(n) / 2.0
