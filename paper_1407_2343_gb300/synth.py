"""Seeded synthetic noisy scenes shaped like the paper's test images.

The paper's experiments (Sec. IV) use standard natural grey-scale images of
256x256 .. 1024x1024 corrupted by additive Gaussian noise (Eq. (15)). Those
images are not available here, so these scenes stand in for them:

  * a constant background with intensity U[0, 255];
  * 20 shapes painted in order, each an axis-aligned rectangle or a disc with
    probability 1/2, centre uniform in the image, half-size(s) uniform in
    [min(H,W)/32, min(H,W)/6], intensity U[0, 255];
  * a 2-D sinusoidal texture 10 sin(2 pi (a x / W + b y / H) + phi) with
    a, b ~ U[2, 12] and phi ~ U[0, 2 pi);
  * i.i.d. N(0, sigma^2) noise (Eq. (15)).

Storage variants: float32 as is, float16 by round-to-nearest-even, uint8 by
clipping to [0, 255] and rounding half to even.

This module is the single source of inputs for both the CUDA path and the
oracle; it contains none of the denoising arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Scene:
    clean: np.ndarray  # float64, the noise-free image f0
    noisy: np.ndarray  # float64, f = f0 + sigma * n (before storage rounding)
    sigma: float
    seed: int


def scene(H: int, W: int, sigma: float, seed: int = 0, n_shapes: int = 20) -> Scene:
    rng = np.random.Generator(np.random.PCG64(seed))
    img = np.full((H, W), rng.uniform(0.0, 255.0), dtype=np.float64)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    m = min(H, W)
    lo, hi = m / 32.0, m / 6.0
    for _ in range(n_shapes):
        is_rect = rng.uniform() < 0.5
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        val = rng.uniform(0.0, 255.0)
        if is_rect:
            hy, hx = rng.uniform(lo, hi), rng.uniform(lo, hi)
            mask = (np.abs(yy - cy) <= hy) & (np.abs(xx - cx) <= hx)
        else:
            r = rng.uniform(lo, hi)
            mask = (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
        img[mask] = val
    a, b = rng.uniform(2.0, 12.0), rng.uniform(2.0, 12.0)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    img = img + 10.0 * np.sin(2.0 * math.pi * (a * xx / W + b * yy / H) + phi)
    noisy = img + sigma * rng.standard_normal((H, W))
    return Scene(clean=img, noisy=noisy, sigma=float(sigma), seed=int(seed))


def store(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round an image to its storage type: 'u8', 'f16' or 'f32'."""
    if dtype == "u8":
        return np.clip(np.rint(x), 0, 255).astype(np.uint8)
    if dtype == "f16":
        return x.astype(np.float16)
    if dtype == "f32":
        return x.astype(np.float32)
    raise ValueError(f"unknown storage type {dtype!r}")


def noisy_image(H: int, W: int, sigma: float, seed: int = 0, dtype: str = "f32") -> np.ndarray:
    """The stored noisy image of `scene(H, W, sigma, seed)`."""
    return store(scene(H, W, sigma, seed).noisy, dtype)


def signals(n: int, N: int, sigma: float, seed: int = 0, dtype: str = "f32") -> np.ndarray:
    """n independent 1-D noisy signals of length N: piecewise-constant steps
    plus a sinusoid plus N(0, sigma^2) noise (the shape of the 1-D example of
    Sec. II, Fig. 2, on the [0, 255] scale)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    out = np.empty((n, N), np.float64)
    t = np.arange(N, dtype=np.float64)
    for k in range(n):
        nseg = int(rng.integers(1, 8))
        cuts = np.sort(rng.integers(0, max(N, 1), size=nseg))
        levels = rng.uniform(0, 255, size=nseg + 1)
        base = levels[np.searchsorted(cuts, t, side="right")]
        base = base + 10.0 * np.sin(2 * math.pi * rng.uniform(1, 6) * t / max(N, 1) + rng.uniform(0, 2 * math.pi))
        out[k] = base + sigma * rng.standard_normal(N)
    return store(out, dtype)


def batch_specs(n: int = 256, seed: int = 0):
    """Uneven batch: side log-uniform in [64, 1024], aspect in [1/2, 2] (also
    log-uniform), dtype u8 / f16 with p = 1/2, sigma ~ U[10, 50],
    S in {5, 10, 15}, K in {2, 3, 5}, box profile, order RC."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    specs = []
    for i in range(n):
        side = math.exp(rng.uniform(math.log(64), math.log(1024)))
        asp = math.exp(rng.uniform(math.log(0.5), math.log(2.0)))
        H = int(min(max(round(side * math.sqrt(asp)), 64), 1024))
        W = int(min(max(round(side / math.sqrt(asp)), 64), 1024))
        specs.append(dict(H=H, W=W, dtype="u8" if rng.uniform() < 0.5 else "f16",
                          sigma=float(rng.uniform(10, 50)), S=int(rng.choice([5, 10, 15])),
                          K=int(rng.choice([2, 3, 5])), profile="box", order="RC", seed=i))
    return specs
