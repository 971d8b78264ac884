"""Oracle: local fractal dimension by differential box counting, and the LFD class of a block.

Test infrastructure only (see the package docstring).

Section 3.1 estimates the local fractal dimension (LFD) of every range and every overlapping
domain with the differential box-counting (DBC) method of Sarkar and Chaudhuri (ref. [9]); the
paper does not restate the estimator, so this module fixes one reading of it:

* An M x M block with G grey levels is covered by s x s cells for s = 2, 4, ..., M/2. Each
  cell carries a column of boxes of height h = s * G / M. A cell whose minimum and maximum
  fall in boxes floor(min / h) and floor(max / h) contributes
  n = floor(max / h) - floor(min / h) + 1 boxes; N_s is the sum over the cells.
* The dimension is the least-squares slope of log2 N_s against log2(M / s) (the box-counting
  definition, Section 3.1 Eq. 1, fitted over the available scales). For M = 8 the two points
  give FD = log2 N_2 - log2 N_4; for M = 16 the middle of three equally spaced points has zero
  weight and FD = (log2 N_2 - log2 N_8) / 2.
* log2 of an integer is the correctly rounded binary64 value, so every FD is one well-defined
  double.
* Ranges are measured on their pixels (G = 256). Domains are measured on their contracted
  block: the integer 2x2 sums (G = 1024), which is the 2x2 average with G = 256.

Classes (Section 3.1 Eq. 2 and 3): with F_l and F_m the least and largest domain FD of the
image, the FD axis [F_l, F_m] is cut into K equal classes, bin(f) = min(K-1, max(0,
floor(K * ((f - F_l) / (F_m - F_l))))) evaluated as separate IEEE binary64 operations, and
bin = 0 when F_m == F_l. A pool half-width of floor(K / 3) classes is the fractal distance
D_f = (F_m - F_l) / 3 of Eq. 2 measured in class units.
"""
from __future__ import annotations

import decimal
import functools

import numpy as np


@functools.lru_cache(maxsize=None)
def log2_cr(n: int) -> float:
    """Correctly rounded binary64 log2 of a positive integer (60 significant digits, then the
    nearest double; float(Decimal) rounds correctly)."""
    if n <= 0:
        raise ValueError("log2 of a non-positive integer")
    ctx = decimal.Context(prec=60)
    v = ctx.divide(ctx.ln(decimal.Decimal(n)), ctx.ln(decimal.Decimal(2)))
    return float(v)


def scales(M: int) -> list[int]:
    """Cell sizes s = 2, 4, ..., M/2."""
    out, s = [], 2
    while s <= M // 2:
        out.append(s)
        s *= 2
    return out


def box_counts(block: np.ndarray, G: int) -> list[int]:
    """N_s for s in scales(M), for an M x M block of integers in [0, G)."""
    M = block.shape[0]
    block = np.asarray(block, dtype=np.int64)
    counts = []
    for s in scales(M):
        h = s * G // M
        total = 0
        for cy in range(0, M, s):
            for cx in range(0, M, s):
                cell = block[cy:cy + s, cx:cx + s]
                total += int(cell.max()) // h - int(cell.min()) // h + 1
        counts.append(total)
    return counts


def fd_from_counts(counts: list[int], M: int) -> float:
    """Least-squares slope of log2 N_s against log2(M/s) (see the module docstring)."""
    L = [log2_cr(c) for c in counts]
    if M == 8:
        return L[0] - L[1]
    if M == 16:
        return (L[0] - L[2]) / 2.0
    raise ValueError("block side must be 8 or 16")


def range_fd(range_block: np.ndarray) -> tuple[list[int], float]:
    """Counts and FD of a range block of pixels (G = 256)."""
    c = box_counts(range_block, 256)
    return c, fd_from_counts(c, range_block.shape[0])


def domain_fd(sum_block: np.ndarray) -> tuple[list[int], float]:
    """Counts and FD of a contracted domain given as 2x2 sums (G = 1024)."""
    c = box_counts(sum_block, 1024)
    return c, fd_from_counts(c, sum_block.shape[0])


def fd_extent(fd_dom: np.ndarray) -> tuple[float, float]:
    """F_l and F_m of Eq. 2: least and largest FD over the image's domains."""
    return float(np.min(fd_dom)), float(np.max(fd_dom))


def classify(fd: np.ndarray, F_l: float, F_m: float, K: int) -> np.ndarray:
    """LFD class of each FD value (module docstring), as int64."""
    fd = np.asarray(fd, dtype=np.float64)
    if F_m == F_l:
        return np.zeros(fd.shape, dtype=np.int64)
    t = fd - F_l
    u = F_m - F_l
    v = t / u
    b = np.floor(v * float(K)).astype(np.int64)
    return np.clip(b, 0, K - 1)


def default_half_width(K: int) -> int:
    """Pool half-width in classes: D_f = (F_m - F_l)/3 (Eq. 2) is K/3 classes wide."""
    return K // 3
