"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module only draws random images and workload descriptions; it holds none
of the filter's arithmetic. Both the CUDA path and the FP64 oracle are fed
the identical arrays it returns.

Recipes (numpy PCG64, seeded):

* ``rectangles(H, W, seed)``: background U[0,1]; 16 axis-aligned rectangles
  painted in order, each with x-corners two sorted draws from U{0..W-1} (same
  for y) and level U[0,1]; then additive N(0, 0.05^2) noise, clipped to [0,1].
  A piecewise-constant image with edges, the workload a bilateral filter is
  meant for.
* ``sinusoids(H, W, seed)``: sum of 8 plane waves
  sin(2 pi (u_i x / W + v_i y / H) + phi_i), (u_i, v_i) ~ U[-16,16]^2,
  phi_i ~ U[0, 2 pi), min-max normalised to [0,1]. A smooth field.
* ``batch_specs(n, seed)``: n images with sides ~ U{64..2048} (independent),
  r ~ U{2..32}, sigma_r ~ U[0.08, 0.4]; image i is drawn with seed 1000+i.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def rectangles(H: int, W: int, seed: int = 0, n_rect: int = 16,
               noise: float = 0.05) -> np.ndarray:
    """Piecewise-constant image (16 rectangles, levels U[0,1]) plus Gaussian
    noise, clipped to [0, 1]. float32, shape (H, W)."""
    g = _rng(seed)
    img = np.full((H, W), g.uniform(0.0, 1.0), dtype=np.float64)
    for _ in range(n_rect):
        x0, x1 = np.sort(g.integers(0, W, size=2))
        y0, y1 = np.sort(g.integers(0, H, size=2))
        img[y0:y1 + 1, x0:x1 + 1] = g.uniform(0.0, 1.0)
    img += g.normal(0.0, noise, size=(H, W))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def sinusoids(H: int, W: int, seed: int = 0, n_waves: int = 8) -> np.ndarray:
    """Smooth field: sum of 8 random plane waves, min-max normalised to
    [0, 1]. float32, shape (H, W)."""
    g = _rng(seed)
    u = g.uniform(-16.0, 16.0, size=n_waves)
    v = g.uniform(-16.0, 16.0, size=n_waves)
    ph = g.uniform(0.0, 2.0 * np.pi, size=n_waves)
    ys = (np.arange(H, dtype=np.float64) / H)[:, None]
    xs = (np.arange(W, dtype=np.float64) / W)[None, :]
    acc = np.zeros((H, W), np.float64)
    for i in range(n_waves):
        acc += np.sin(2.0 * np.pi * (u[i] * xs + v[i] * ys) + ph[i])
    lo, hi = acc.min(), acc.max()
    acc = (acc - lo) / (hi - lo) if hi > lo else np.zeros_like(acc)
    return acc.astype(np.float32)


def noise(H: int, W: int, seed: int = 0) -> np.ndarray:
    """Independent U[0, 1] pixels: almost every neighbour differs from the
    centre by much more than sigma_r, so den stays near 1 (the hardest case
    for cancellation in the recombined sums)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((H, W)).astype(np.float32)


def image(kind: str, H: int, W: int, seed: int = 0) -> np.ndarray:
    if kind in ("rect", "rectangles"):
        return rectangles(H, W, seed)
    if kind in ("sin", "sinusoids"):
        return sinusoids(H, W, seed)
    if kind == "noise":
        return noise(H, W, seed)
    raise ValueError(f"unknown image kind {kind!r}")


def weights(shape, seed: int = 1) -> np.ndarray:
    """Loss weights w ~ N(0, 1) for L = sum(w * out). float32."""
    return _rng(seed).normal(0.0, 1.0, size=shape).astype(np.float32)


def batch_specs(n: int = 256, seed: int = 7, side_lo: int = 64, side_hi: int = 2048,
                r_lo: int = 2, r_hi: int = 32, s_lo: float = 0.08, s_hi: float = 0.4):
    """Descriptions of n uneven images: dicts with H, W, r, sigma_r, seed."""
    g = _rng(seed)
    out = []
    for i in range(n):
        out.append(dict(H=int(g.integers(side_lo, side_hi + 1)),
                        W=int(g.integers(side_lo, side_hi + 1)),
                        r=int(g.integers(r_lo, r_hi + 1)),
                        sigma_r=float(g.uniform(s_lo, s_hi)),
                        seed=1000 + i))
    return out
