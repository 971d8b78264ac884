"""Seeded synthetic 8-bit grayscale images that stand in for the paper's test images.

The paper's experiments (Section 4, Tables 2-4) use natural photographs at 256x256 and
512x512 that are not distributed with it. These generators produce images with the same
shape and value range and with the structure the classification cares about: regions of
different roughness (fractional Brownian motion with a different Hurst exponent per
quadrant, so local fractal dimensions spread over their range), smooth ramps, and
hard-edged flat rectangles (flat blocks and sharp edges).

This module holds no arithmetic of the compression method itself. It is shared by the
tests (which feed the same pixels to the CPU oracle and to the CUDA path) and by bench.py.

Recipe for ``fbm_image(seed, H, W)``:
  * numpy PCG64 generator seeded with ``seed``;
  * one diamond-square fBm field per quadrant on a (2^m+1)^2 grid at least the quadrant's
    size, cropped; Hurst exponents (top-left, top-right, bottom-left, bottom-right) default
    to 0.3, 0.3+0.5/3, 0.3+1.0/3, 0.8;
  * each field rescaled to mean 128 and standard deviation 40;
  * a linear ramp of +-32 across a random direction;
  * three axis-aligned rectangles of a random constant intensity in [0, 255], sides
    uniform in [side/8, side/4], written over the texture;
  * clipped to [0, 255] and rounded half-to-even to uint8.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "fbm_image",
    "pr1_image",
    "image_1024",
    "diff_image",
    "large_image",
    "batch_images",
    "BATCH_SIDES",
]

DEFAULT_HURST = (0.3, 0.3 + 0.5 / 3.0, 0.3 + 1.0 / 3.0, 0.8)
BATCH_SIDES = (256, 384, 512, 768, 1024, 1536, 2048)


def _diamond_square(rng: np.random.Generator, m: int, hurst: float) -> np.ndarray:
    """Midpoint-displacement fBm surface on a (2^m+1) x (2^m+1) grid."""
    n = (1 << m) + 1
    f = np.zeros((n, n), dtype=np.float64)
    f[0, 0], f[0, -1], f[-1, 0], f[-1, -1] = rng.standard_normal(4)
    step = n - 1
    scale = 1.0
    while step > 1:
        half = step // 2
        scale *= 2.0 ** (-hurst)
        # diamond step: square centres from the four corners
        c = (f[0:-1:step, 0:-1:step] + f[0:-1:step, step::step]
             + f[step::step, 0:-1:step] + f[step::step, step::step]) * 0.25
        f[half::step, half::step] = c + scale * rng.standard_normal(c.shape)
        # square step: edge midpoints from their (up to four) neighbours
        p = np.full((n + 2 * half, n + 2 * half), np.nan)
        p[half:half + n, half:half + n] = f
        for (y0, x0) in ((0, half), (half, 0)):
            ys = np.arange(y0, n, step)
            xs = np.arange(x0, n, step)
            yy, xx = np.meshgrid(ys + half, xs + half, indexing="ij")
            nb = np.stack([p[yy - half, xx], p[yy + half, xx], p[yy, xx - half], p[yy, xx + half]])
            cnt = np.sum(~np.isnan(nb), axis=0)
            avg = np.nansum(nb, axis=0) / cnt
            f[np.ix_(ys, xs)] = avg + scale * rng.standard_normal(avg.shape)
        step = half
    return f


def _field(rng: np.random.Generator, h: int, w: int, hurst: float) -> np.ndarray:
    side = max(h, w, 2)
    m = int(np.ceil(np.log2(side - 1))) if side > 2 else 1
    f = _diamond_square(rng, m, hurst)[:h, :w]
    sd = f.std()
    f = (f - f.mean()) / (sd if sd > 0 else 1.0)
    return 128.0 + 40.0 * f


def fbm_image(seed: int, H: int, W: int | None = None, hurst=DEFAULT_HURST,
              n_rects: int = 3) -> np.ndarray:
    """Seeded fBm + ramp + rectangles image, uint8, shape (H, W). H and W must be even."""
    W = H if W is None else W
    if H % 2 or W % 2 or H < 2 or W < 2:
        raise ValueError("image sides must be even and >= 2")
    rng = np.random.Generator(np.random.PCG64(seed))
    h2, w2 = H // 2, W // 2
    img = np.empty((H, W), dtype=np.float64)
    for q, (oy, ox) in enumerate(((0, 0), (0, w2), (h2, 0), (h2, w2))):
        img[oy:oy + h2, ox:ox + w2] = _field(rng, h2, w2, float(hurst[q]))
    theta = rng.random() * 2.0 * np.pi
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    proj = (xx - (W - 1) / 2.0) * np.cos(theta) + (yy - (H - 1) / 2.0) * np.sin(theta)
    img += 32.0 * proj / np.abs(proj).max()
    for _ in range(n_rects):
        rh = int(rng.integers(max(1, H // 8), max(1, H // 4) + 1))
        rw = int(rng.integers(max(1, W // 8), max(1, W // 4) + 1))
        y0 = int(rng.integers(0, H - rh + 1))
        x0 = int(rng.integers(0, W - rw + 1))
        img[y0:y0 + rh, x0:x0 + rw] = float(rng.integers(0, 256))
    return np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)


def pr1_image() -> np.ndarray:
    """256x256, seed 1000: the small case the oracle runs in full."""
    return fbm_image(1000, 256)


def image_1024() -> np.ndarray:
    """1024x1024, seed 2000: the encode throughput workload."""
    return fbm_image(2000, 1024)


def diff_image() -> np.ndarray:
    """512x512, seed 4000: the decode / adjoint workload."""
    return fbm_image(4000, 512)


def large_image() -> np.ndarray:
    """4096x4096, seed 5000."""
    return fbm_image(5000, 4096)


def batch_images(n: int = 64, base_seed: int = 3000, sides=BATCH_SIDES):
    """n images with sides drawn uniformly from ``sides`` and per-image Hurst exponents
    drawn uniformly from [0.3, 0.8] per quadrant; image i uses seed base_seed + i."""
    out = []
    for i in range(n):
        rng = np.random.Generator(np.random.PCG64(base_seed + i))
        side = int(sides[int(rng.integers(0, len(sides)))])
        hurst = tuple(float(h) for h in rng.uniform(0.3, 0.8, size=4))
        out.append(fbm_image(base_seed + i, side, side, hurst=hurst))
    return out
