"""Oracle: block geometry of the partitioned IFS encoder.

Test infrastructure only (see the package docstring).

* Ranges: the image is cut into non-overlapping B x B blocks (Section 1; Section 2 uses B = 8
  on a 1024 x 1024 image, giving 2^14 ranges).
* Domains: 2B x 2B blocks (twice the range side), allowed to overlap
  (Section 2). Their top-left corners lie on a grid of stride sigma; sigma = 1 gives the
  (n - 15)^2 domains per image of Table 1.
* Contraction ("resizing", Section 1): a domain is reduced to B x B by summing each 2 x 2 pixel
  cell. The real-valued contracted domain is that sum divided by 4 (2 x 2 averaging).
* Isometries ("rotation", Section 1): the 8 symmetries of the square, numbered
  0 identity, 1 rotation by 90 degrees clockwise, 2 rotation by 180, 3 rotation by 270
  clockwise, 4 left-right mirror, 5 up-down mirror, 6 transpose, 7 anti-transpose.
"""
from __future__ import annotations

import numpy as np

N_ISO = 8
# T_t^{-1} = T_{INVERSE[t]}
INVERSE = (0, 3, 2, 1, 4, 5, 6, 7)


def range_grid(H: int, W: int, B: int) -> tuple[int, int]:
    """Ranges per column and per row (Section 1: non-overlapping range blocks)."""
    return H // B, W // B


def n_ranges(H: int, W: int, B: int) -> int:
    ry, rx = range_grid(H, W, B)
    return ry * rx


def domain_grid(H: int, W: int, B: int, sigma: int) -> tuple[int, int]:
    """Domain corners per column and per row: dy in {0, sigma, ...} with dy + 2B <= H."""
    return (H - 2 * B) // sigma + 1, (W - 2 * B) // sigma + 1


def n_domains(H: int, W: int, B: int, sigma: int) -> int:
    dy, dx = domain_grid(H, W, B, sigma)
    return dy * dx


def range_origin(H: int, W: int, B: int, r: int) -> tuple[int, int]:
    """Top-left pixel of range r; ranges are numbered row-major."""
    _, rx = range_grid(H, W, B)
    return (r // rx) * B, (r % rx) * B


def domain_origin(H: int, W: int, B: int, sigma: int, d: int) -> tuple[int, int]:
    """Top-left pixel of domain d; domains are numbered row-major over the stride grid."""
    _, ndx = domain_grid(H, W, B, sigma)
    return (d // ndx) * sigma, (d % ndx) * sigma


def range_block(img: np.ndarray, B: int, r: int) -> np.ndarray:
    H, W = img.shape
    y, x = range_origin(H, W, B, r)
    return img[y:y + B, x:x + B].astype(np.int64)


def domain_sum_block(img: np.ndarray, B: int, sigma: int, d: int) -> np.ndarray:
    """Contracted domain as integer 2x2 sums: S[y][x] = sum_{a,b in {0,1}} I[dy+2y+a][dx+2x+b]."""
    H, W = img.shape
    dy, dx = domain_origin(H, W, B, sigma, d)
    blk = img[dy:dy + 2 * B, dx:dx + 2 * B].astype(np.int64)
    S = np.zeros((B, B), dtype=np.int64)
    for a in (0, 1):
        for b in (0, 1):
            S += blk[a::2, b::2]
    return S


def range_blocks(img: np.ndarray, B: int) -> np.ndarray:
    H, W = img.shape
    return np.stack([range_block(img, B, r) for r in range(n_ranges(H, W, B))])


def domain_sum_blocks(img: np.ndarray, B: int, sigma: int) -> np.ndarray:
    H, W = img.shape
    return np.stack([domain_sum_block(img, B, sigma, d) for d in range(n_domains(H, W, B, sigma))])


def iso_source(B: int, t: int, y: int, x: int) -> tuple[int, int]:
    """(T_t X)[y][x] = X[iso_source(B, t, y, x)]."""
    N = B - 1
    if t == 0:
        return y, x
    if t == 1:
        return N - x, y
    if t == 2:
        return N - y, N - x
    if t == 3:
        return x, N - y
    if t == 4:
        return y, N - x
    if t == 5:
        return N - y, x
    if t == 6:
        return x, y
    if t == 7:
        return N - x, N - y
    raise ValueError("isometry index must be 0..7")


def isometry(X: np.ndarray, t: int) -> np.ndarray:
    """Apply T_t to a square block by the index map above."""
    B = X.shape[0]
    out = np.empty_like(X)
    for y in range(B):
        for x in range(B):
            sy, sx = iso_source(B, t, y, x)
            out[y, x] = X[sy, sx]
    return out
