"""Seeded synthetic test images: smooth background + sharp-edged shapes + Gaussian noise.

This module holds none of the WMC arithmetic.  It is the one piece both the CUDA path's tests
and the FP64 oracle's tests draw their inputs from.  The paper denoises photographs and a
synthetic image of circles at several scales and contrasts (Sec. V-B, V-C, V-D), all absent
here; these images stand in for them.  They have a smooth part (where WMC behaves like a
Laplacian), straight and curved edges (where the half-window selection keeps edges), and
i.i.d. Gaussian noise (the noise model under which Sec. III-B shows contrast invariance).

Recipe, all draws from ``numpy.random.Generator(PCG64(seed))`` in this order:
  1. background 0.5;
  2. ``n_bumps`` Gaussian bumps: amplitude U(-0.4, 0.4), centre uniform over the image,
     standard deviation U(0.03, 0.25) * min(H, W), built separably (outer product of 1-D
     Gaussians) and summed with one matrix product;
  3. ``n_shapes`` constant-intensity shapes painted over it, alternating axis-aligned
     rectangles (height, width each U(0.05, 0.3) * min(H, W)) and disks (diameter
     U(0.05, 0.3) * min(H, W)), centre uniform, intensity U(0, 1);
  4. clip the clean image to [0, 1];
  5. add N(0, sigma^2) noise (not clipped), drawn row-block by row-block in FP64.
Everything is FP64 until the final cast.
"""
from __future__ import annotations

import numpy as np


def make_image(h: int, w: int, seed: int, n_bumps: int = 8, n_shapes: int = 4, sigma: float = 0.05,
               dtype=np.float32, return_clean: bool = False, block_rows: int = 1024):
    """Return the noisy image (and optionally the clean one) as ``dtype`` arrays of shape (h, w)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = float(min(h, w))
    clean = np.full((h, w), 0.5, dtype=np.float64)
    if n_bumps > 0:
        amp = rng.uniform(-0.4, 0.4, n_bumps)
        cy = rng.uniform(0.0, h, n_bumps)
        cx = rng.uniform(0.0, w, n_bumps)
        sd = rng.uniform(0.03, 0.25, n_bumps) * m
        ys = np.arange(h, dtype=np.float64)[:, None]
        xs = np.arange(w, dtype=np.float64)[:, None]
        gy = np.exp(-0.5 * ((ys - cy[None, :]) / sd[None, :]) ** 2)  # h x n
        gx = np.exp(-0.5 * ((xs - cx[None, :]) / sd[None, :]) ** 2)  # w x n
        clean += (gy * amp[None, :]) @ gx.T
    for k in range(n_shapes):
        val = rng.uniform(0.0, 1.0)
        cy, cx = rng.uniform(0.0, h), rng.uniform(0.0, w)
        if k % 2 == 0:
            sh = rng.uniform(0.05, 0.3) * m
            sw = rng.uniform(0.05, 0.3) * m
            y0, y1 = int(round(cy - sh / 2)), int(round(cy + sh / 2))
            x0, x1 = int(round(cx - sw / 2)), int(round(cx + sw / 2))
            clean[max(y0, 0):max(min(y1, h), 0), max(x0, 0):max(min(x1, w), 0)] = val
        else:
            r = 0.5 * rng.uniform(0.05, 0.3) * m
            y0, y1 = max(int(np.floor(cy - r)), 0), min(int(np.ceil(cy + r)) + 1, h)
            x0, x1 = max(int(np.floor(cx - r)), 0), min(int(np.ceil(cx + r)) + 1, w)
            if y1 > y0 and x1 > x0:
                yy = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
                xx = np.arange(x0, x1, dtype=np.float64)[None, :] - cx
                mask = yy * yy + xx * xx <= r * r
                clean[y0:y1, x0:x1][mask] = val
    np.clip(clean, 0.0, 1.0, out=clean)
    noisy = np.empty((h, w), dtype=dtype)
    for r0 in range(0, h, block_rows):
        r1 = min(r0 + block_rows, h)
        noisy[r0:r1] = (clean[r0:r1] + sigma * rng.standard_normal((r1 - r0, w))).astype(dtype)
    if return_clean:
        return noisy, clean.astype(dtype)
    return noisy


# Named workloads (sizes, counts and noise levels of the configurations this library is
# measured on).
def pr1_image(return_clean: bool = False):
    """One 256 x 256 image, 8 bumps + 4 shapes, sigma 0.05, seed 0."""
    return make_image(256, 256, seed=0, n_bumps=8, n_shapes=4, sigma=0.05, return_clean=return_clean)


def scale_image(sigma: float = 0.02, return_clean: bool = False):
    """One 4096 x 4096 image, 64 bumps + 32 shapes; seed 1 for sigma 0.02, seed 2 for sigma 0.1."""
    seed = 1 if sigma == 0.02 else 2
    return make_image(4096, 4096, seed=seed, n_bumps=64, n_shapes=32, sigma=sigma,
                      return_clean=return_clean)


def batch_sizes(n: int = 512, seed: int = 999, lo: int = 64, hi: int = 1536):
    """Side lengths (H_i, W_i), each uniform on [lo, hi], for a batch of uneven images."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hs = rng.integers(lo, hi + 1, n)
    ws = rng.integers(lo, hi + 1, n)
    return [(int(a), int(b)) for a, b in zip(hs, ws)]


def batch_params(n: int = 512, seed: int = 998):
    """Per-image (sigma_i ~ U[0.01, 0.15], lambda_i ~ U[0.5, 2]) for the uneven batch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sig = rng.uniform(0.01, 0.15, n)
    lam = rng.uniform(0.5, 2.0, n)
    return [(float(s), float(l)) for s, l in zip(sig, lam)]
