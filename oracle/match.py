"""Oracle: Python side of the exact matcher (oracle/match.c) and the whole encode pipeline.

Test infrastructure only (see the package docstring).

``encode`` follows the paper's order of operations (Section 3.1): FDs of the ranges into a
linear array, FDs of the overlapping domains, F_l / F_m and the fractal distance (Eq. 2), each
range's pool from its FD (Eq. 3, class mode or literal mode, ``oracle.pools``), then the
exhaustive least-squares search inside the pool (Section 1), done in C with exact integers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import dbc, geometry, pools

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/match.c with gcc (OpenMP, no floating-point contraction)."""
    src = os.path.join(_HERE, "match.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
           src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            ci = ctypes.c_int
            lib.oracle_match.argtypes = [p, i64, ci, ci, ci, ci, i64, p, p, p, p, p, p, p, p, ci]
            lib.oracle_match.restype = ci
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def match_pools(img: np.ndarray, B: int, sigma: int, range_ids, pool_list, n_threads: int = 1):
    """Exact best (domain, isometry, s, o, sse) for each listed range over its given pool."""
    lib = _load()
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    rid = np.ascontiguousarray(np.asarray(range_ids, dtype=np.int64))
    ptr, idx = pools.pools_csr([np.sort(np.asarray(p, dtype=np.int64)) for p in pool_list])
    n = rid.size
    out = {
        "dom": np.zeros(n, np.int32), "iso": np.zeros(n, np.int32),
        "s": np.zeros(n, np.float64), "o": np.zeros(n, np.float64), "sse": np.zeros(n, np.float64),
    }
    rc = lib.oracle_match(_ptr(img), W, H, W, B, sigma, n, _ptr(rid), _ptr(ptr), _ptr(idx),
                          _ptr(out["dom"]), _ptr(out["iso"]), _ptr(out["s"]), _ptr(out["o"]),
                          _ptr(out["sse"]), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_match rejected its arguments")
    return out


def range_blocks_all(img: np.ndarray, B: int) -> np.ndarray:
    """(R, B, B) int64 range blocks, row-major range order."""
    H, W = img.shape
    return img.reshape(H // B, B, W // B, B).transpose(0, 2, 1, 3).reshape(-1, B, B).astype(np.int64)


def domain_sums_all(img: np.ndarray, B: int, sigma: int) -> np.ndarray:
    """(Dn, B, B) int64 contracted domains: S[d][y][x] = sum of the 2x2 cell at
    (dy + 2y, dx + 2x)."""
    H, W = img.shape
    ndy, ndx = geometry.domain_grid(H, W, B, sigma)
    dy = (np.arange(ndy * ndx) // ndx) * sigma
    dx = (np.arange(ndy * ndx) % ndx) * sigma
    yy = dy[:, None, None] + 2 * np.arange(B)[None, :, None]
    xx = dx[:, None, None] + 2 * np.arange(B)[None, None, :]
    I = img.astype(np.int64)
    return I[yy, xx] + I[yy, xx + 1] + I[yy + 1, xx] + I[yy + 1, xx + 1]


def box_counts_all(blocks: np.ndarray, G: int) -> np.ndarray:
    """(N, n_scales) box counts of many M x M blocks: same formula as dbc.box_counts."""
    N, M, _ = blocks.shape
    out = []
    for s in dbc.scales(M):
        h = s * G // M
        cells = blocks.reshape(N, M // s, s, M // s, s)
        mx = cells.max(axis=(2, 4)) // h
        mn = cells.min(axis=(2, 4)) // h
        out.append((mx - mn + 1).sum(axis=(1, 2)))
    return np.stack(out, axis=1).astype(np.int64)


def fd_all(counts: np.ndarray, M: int) -> np.ndarray:
    """FD of each row of counts, with the same binary64 operations as dbc.fd_from_counts."""
    table = np.array([0.0] + [dbc.log2_cr(k) for k in range(1, int(counts.max()) + 1)])
    L = table[counts]
    if M == 8:
        return L[:, 0] - L[:, 1]
    if M == 16:
        return (L[:, 0] - L[:, 2]) / 2.0
    raise ValueError("block side must be 8 or 16")


def classify_image(img: np.ndarray, B: int, sigma: int, K: int) -> dict:
    """Block moments, DBC counts, FDs, F_l, F_m and classes of every range and domain."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    rb = range_blocks_all(img, B)
    ds = domain_sums_all(img, B, sigma)
    rc = box_counts_all(rb, 256)
    dc = box_counts_all(ds, 1024)
    rfd = fd_all(rc, B)
    dfd = fd_all(dc, B)
    F_l, F_m = dbc.fd_extent(dfd)
    return {
        "range_sum": rb.sum(axis=(1, 2)), "range_sumsq": (rb * rb).sum(axis=(1, 2)),
        "dom_sum": ds.sum(axis=(1, 2)), "dom_sumsq": (ds * ds).sum(axis=(1, 2)),
        "range_counts": rc, "dom_counts": dc, "range_fd": rfd, "dom_fd": dfd,
        "F_l": F_l, "F_m": F_m,
        "range_bin": dbc.classify(rfd, F_l, F_m, K), "dom_bin": dbc.classify(dfd, F_l, F_m, K),
    }


def encode(img: np.ndarray, B: int = 8, sigma: int = 8, K: int = 8, w: int | None = None,
           mode: str = "class", range_ids=None, n_threads: int = 1, cls: dict | None = None):
    """Oracle encode of the listed ranges (all by default). Returns codes plus the pools'
    sizes and the classification."""
    if cls is None:
        cls = classify_image(img, B, sigma, K)
    w = dbc.default_half_width(K) if w is None else w
    H, W = img.shape
    R = geometry.n_ranges(H, W, B)
    rid = np.arange(R) if range_ids is None else np.asarray(range_ids, dtype=np.int64)
    if mode == "class":
        plist = [pools.class_pool(cls["range_bin"][r], cls["dom_bin"], w) for r in rid]
    elif mode == "literal":
        Df = pools.fractal_distance(cls["F_l"], cls["F_m"])
        plist = [pools.literal_pool(cls["range_fd"][r], cls["dom_fd"], Df) for r in rid]
    else:
        raise ValueError("mode must be 'class' or 'literal'")
    codes = match_pools(img, B, sigma, rid, plist, n_threads=n_threads)
    codes["range_ids"] = rid
    codes["pool_size"] = np.array([p.size for p in plist], dtype=np.int64)
    codes["cls"] = cls
    return codes
