"""Pins of the oracle's dynamic pools (Section 3.1 Eq. 2-3) on hand-built fractal dimensions.

Eq. 2 fixes the fractal distance D_f = (F_m - F_l) / 3 and Eq. 3 keeps the domains whose FD lies
in the closed interval [d_r - D_f, d_r + D_f]. The FD values below are chosen so that every bound
is an exact binary64 number: a domain sitting exactly on a bound must be in the pool, one ulp
outside must not, and a window that holds no domain falls back to every domain. Each case runs
through ``oracle.match.encode`` (the path the GPU parity tests compare against) with the
classification replaced by the hand-built one, so a strict bound, a different divisor in D_f or a
missing fallback in that path fails here.
"""
import numpy as np

from oracle import match as omatch
from oracle import pools
from paper_1206_4880_gb300 import synth

F_L, F_M = 1.0, 2.5          # D_f = 1.5 / 3 = 0.5 exactly
BELOW_LO = np.nextafter(1.25, -np.inf)
ABOVE_HI = np.nextafter(2.25, np.inf)
# 9 domains of a 24 x 24 image (8x8 ranges, 16x16 domains at stride 4: a 3 x 3 grid)
DOM_FD = np.array([1.0, 1.25, BELOW_LO, 2.25, ABOVE_HI, 2.5, 1.75, 1.5, 2.0])


def _cls(range_fd):
    return {"F_l": F_L, "F_m": F_M, "dom_fd": DOM_FD.copy(),
            "range_fd": np.asarray(range_fd, dtype=np.float64)}


def _encode_literal(range_fd):
    img = synth.fbm_image(61, 24, 24)
    return omatch.encode(img, B=8, sigma=4, K=8, mode="literal", cls=_cls(range_fd))


def test_fractal_distance_is_a_third_of_the_fd_extent():
    assert pools.fractal_distance(F_L, F_M) == 0.5
    assert pools.fractal_distance(1.25, 2.75) == 0.5
    assert pools.fractal_distance(2.0, 2.0) == 0.0
    assert pools.fractal_distance(1.0, 1.75) == 0.25


def test_literal_window_bounds_are_inclusive_and_exact():
    # d_r = 1.75: window [1.25, 2.25]; the domains at 1.25 and 2.25 are in, their neighbours
    # one ulp outside are out
    pool = pools.literal_pool(1.75, DOM_FD, pools.fractal_distance(F_L, F_M))
    assert pool.tolist() == [1, 3, 6, 7, 8]
    # d_r = F_l: window [0.5, 1.5]
    assert pools.literal_pool(1.0, DOM_FD, 0.5).tolist() == [0, 1, 2, 7]
    # d_r = F_m: window [2.0, 3.0]
    assert pools.literal_pool(2.5, DOM_FD, 0.5).tolist() == [3, 4, 5, 8]


def test_literal_window_empty_falls_back_to_every_domain():
    # range FDs are not bounded by the domains' extent: d_r = 3.25 gives [2.75, 3.75], empty
    assert pools.literal_pool(3.25, DOM_FD, 0.5).tolist() == list(range(9))
    assert pools.literal_pool(0.25, DOM_FD, 0.5).tolist() == list(range(9))


def test_encode_literal_mode_uses_eq2_and_eq3():
    range_fd = [1.75, 1.0, 2.5, 3.25, 1.75, 2.0, 1.5, 2.25, 1.25]
    codes = _encode_literal(range_fd)
    # pool sizes from the hand-computed windows above; 2.0 -> [1.5, 2.5], 1.5 -> [1.0, 2.0],
    # 2.25 -> [1.75, 2.75], 1.25 -> [0.75, 1.75]
    assert codes["pool_size"].tolist() == [5, 4, 4, 9, 5, 6, 6, 5, 5]
    # every chosen domain lies in its range's window (or the range fell back to all domains)
    for r, f in enumerate(range_fd):
        d = codes["dom"][r]
        if codes["pool_size"][r] < 9:
            assert f - 0.5 <= DOM_FD[d] <= f + 0.5, (r, d)


def test_literal_window_edges_decide_the_code():
    """A domain that only the inclusive lower bound admits is chosen when it is the exact fit:
    range 8 (rows 16..23, columns 16..23) is set to the contraction of domain 1 (top-left (0, 4),
    which does not overlap it), built from constant 2x2 cells so the fit is exact (s = 1, o = 0,
    collage error 0). With d_r = 1.75 domain 1 sits on the bound 1.25 of the window."""
    rng = np.random.default_rng(63)
    img = synth.fbm_image(62, 24, 24)
    cells = rng.integers(0, 256, (8, 8), dtype=np.int64)
    img[0:16, 4:20] = np.kron(cells, np.ones((2, 2), np.int64)).astype(np.uint8)
    img[16:24, 16:24] = cells.astype(np.uint8)
    range_fd = [2.5, 2.5, 2.5, 2.5, 2.5, 2.5, 2.5, 2.5, 1.75]
    codes = omatch.encode(img, B=8, sigma=4, K=8, mode="literal", cls=_cls(range_fd))
    assert codes["pool_size"][8] == 5
    assert codes["dom"][8] == 1 and codes["iso"][8] == 0
    assert codes["sse"][8] == 0.0 and codes["s"][8] == 1.0
