"""Oracle: the dynamic domain pool of each range.

Test infrastructure only (see the package docstring).

Section 3 decides each range's domain pool at run time from the range's own local fractal
dimension; Section 3.1 Eq. 3 keeps the domains with d_r - D_f <= d_d <= d_r + D_f, where
D_f = (F_m - F_l)/3 (Eq. 2).

* class mode (the mode the GPU path computes): with the K classes of ``oracle.dbc``,
  Pool(r) = {d : |bin_d - bin_r| <= w}; w = floor(K/3) is Eq. 3's window in class units.
  K = 1 makes every pool the full domain set (exhaustive search, Section 2).
* literal mode: Pool(r) = {d : d_r - D_f <= FD_d <= d_r + D_f} on the FD values themselves.

The paper does not say what happens when no domain satisfies the window; this oracle (and the
GPU path) then searches every domain of the image, i.e. falls back to exhaustive search.
"""
from __future__ import annotations

import numpy as np


def class_pool(bin_r: int, bins_dom: np.ndarray, w: int) -> np.ndarray:
    """Ascending domain ids with |bin_d - bin_r| <= w (all domains if none)."""
    bins_dom = np.asarray(bins_dom)
    pool = np.nonzero(np.abs(bins_dom - int(bin_r)) <= w)[0]
    if pool.size == 0:
        pool = np.arange(bins_dom.size)
    return pool.astype(np.int64)


def literal_pool(fd_r: float, fd_dom: np.ndarray, D_f: float) -> np.ndarray:
    """Ascending domain ids with fd_r - D_f <= FD_d <= fd_r + D_f (all domains if none)."""
    fd_dom = np.asarray(fd_dom, dtype=np.float64)
    lo = fd_r - D_f
    hi = fd_r + D_f
    pool = np.nonzero((fd_dom >= lo) & (fd_dom <= hi))[0]
    if pool.size == 0:
        pool = np.arange(fd_dom.size)
    return pool.astype(np.int64)


def fractal_distance(F_l: float, F_m: float) -> float:
    """D_f = (F_m - F_l) / 3, Eq. 2."""
    return (F_m - F_l) / 3.0


def pools_csr(pools: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """Pack a list of pools into (ptr int64[n+1], idx int32[total])."""
    ptr = np.zeros(len(pools) + 1, dtype=np.int64)
    for i, p in enumerate(pools):
        ptr[i + 1] = ptr[i] + p.size
    idx = np.concatenate(pools).astype(np.int32) if pools else np.zeros(0, np.int32)
    return ptr, idx
