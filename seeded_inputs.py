"""Seeded synthetic grey images for the FEM harmonic-inpainting data optimisation.

The paper's test images (trui, walter, peppers, the 16 Mpixel photograph of
Sec. 5) are not available, so every workload runs on images drawn from one
seeded family that has the ingredients those images exercise: smooth shading
(Gaussian blobs), sharp edges (constant polygons), fine noise and, for the
very large case, a periodic texture.

This module is shared by the CPU oracle's tests, the CUDA path's tests and the
benchmark.  It holds no part of the inpainting method: it only draws images.

Recipe (version 1), all in float64 then stored as float32, row-major, y down,
values clipped to [0, 1]:
  * background 0.5;
  * 8 Gaussian blobs: amplitude U[-0.4, 0.4], sigma U[0.02, 0.15]*n,
    centre uniform over the image;
  * 4 constant polygons painted over the blobs, each with 3..8 vertices at
    angles sorted around a uniform centre and radii U[0.05, 0.3]*n, filled
    with a value U[0, 1] (even-odd rule, a star-shaped polygon);
  * optional plane-wave texture 0.1*sin(2*pi*(x cos(th) + y sin(th))/lam + phi)
    with lam ~ U[16, 64] px, th ~ U[0, pi), phi ~ U[0, 2 pi);
  * additive N(0, 0.02^2) noise, then clipping to [0, 1].
"""
from __future__ import annotations

import numpy as np

GENERATOR_VERSION = 1


def _polygon_mask(xs: np.ndarray, ys: np.ndarray, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """Even-odd point-in-polygon test of pixel centres (xs, ys) against the
    closed polygon (px, py)."""
    inside = np.zeros(xs.shape, dtype=bool)
    nv = len(px)
    for i in range(nv):
        x0, y0 = px[i], py[i]
        x1, y1 = px[(i + 1) % nv], py[(i + 1) % nv]
        if y0 == y1:
            continue
        crosses = (ys >= min(y0, y1)) & (ys < max(y0, y1))
        xint = x0 + (ys - y0) * (x1 - x0) / (y1 - y0)
        inside ^= crosses & (xs < xint)
    return inside


def make_image(n: int, seed: int, texture: bool = False, rows_per_chunk: int = 512) -> np.ndarray:
    """Return an n x n float32 image of the seeded family (see module doc)."""
    if n < 2:
        raise ValueError("image side must be >= 2")
    rng = np.random.default_rng(seed)
    blobs = []
    for _ in range(8):
        amp = rng.uniform(-0.4, 0.4)
        sig = rng.uniform(0.02, 0.15) * n
        cx, cy = rng.uniform(0, n), rng.uniform(0, n)
        blobs.append((amp, sig, cx, cy))
    polys = []
    for _ in range(4):
        nv = int(rng.integers(3, 9))
        cx, cy = rng.uniform(0, n), rng.uniform(0, n)
        ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, nv))
        rad = rng.uniform(0.05, 0.3, nv) * n
        val = rng.uniform(0.0, 1.0)
        polys.append((cx + rad * np.cos(ang), cy + rad * np.sin(ang), val))
    if texture:
        lam = rng.uniform(16.0, 64.0)
        th = rng.uniform(0.0, np.pi)
        phi = rng.uniform(0.0, 2.0 * np.pi)
    noise_seed = int(rng.integers(0, 2**63 - 1))
    noise_rng = np.random.default_rng(noise_seed)

    out = np.empty((n, n), dtype=np.float32)
    xs1 = np.arange(n, dtype=np.float64)
    for r0 in range(0, n, rows_per_chunk):
        r1 = min(n, r0 + rows_per_chunk)
        ys, xs = np.meshgrid(np.arange(r0, r1, dtype=np.float64), xs1, indexing="ij")
        img = np.full(xs.shape, 0.5)
        for amp, sig, cx, cy in blobs:
            img += amp * np.exp(-((xs - cx) ** 2 + (ys - cy) ** 2) / (2.0 * sig * sig))
        for px, py, val in polys:
            img[_polygon_mask(xs, ys, px, py)] = val
        if texture:
            img += 0.1 * np.sin(2.0 * np.pi * (xs * np.cos(th) + ys * np.sin(th)) / lam + phi)
        img += noise_rng.normal(0.0, 0.02, size=img.shape)
        np.clip(img, 0.0, 1.0, out=img)
        out[r0:r1] = img.astype(np.float32)
    return out


def make_residual(n: int, seed: int) -> np.ndarray:
    """Return an n x n float32 field of N(0, 1) values (a seeded pixel-space
    co-vector, used to exercise adjoint operators)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n)).astype(np.float32)


def make_vector(m: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Return m float32 values U[lo, hi) (seeded; e.g. Dirichlet data g)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, m).astype(np.float32)
