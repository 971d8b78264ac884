"""Oracle: the intensity part of one range-domain map, in exact rational arithmetic.

Test infrastructure only (see the package docstring).

Section 1: each range is approximated by a contracted, isometrically transformed domain under
an affine map of the pixel intensities. Here that map is r ~ s * T_t(D) + o with D the
2x2-averaged domain (D = S / 4 for the integer 2x2 sums S), fitted by least squares, with the
contrast clamped to |s| <= s_max for contractivity; when the clamp is active the brightness is
re-solved for the clamped s. The paper prints none of these formulas; they are the textbook
least-squares solution written with the block moments

    n = B*B, A = sum r, Bs = sum r^2, C = sum S, E = sum S^2, X = sum r * T_t(S),
    P = n X - A C, Q = n E - C^2 (>= 0),

    s = 4 P / Q (Q > 0), s = 0 (Q = 0), then clamped to [-s_max, s_max];
    o = (A - s C / 4) / n.

``fit_candidate`` returns s, o and the collage error SSE = sum (r - s T_t(D) - o)^2 computed
from that definition, all as Fractions.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from .geometry import isometry


def moments(r: np.ndarray, S: np.ndarray) -> tuple[int, int, int, int]:
    r = np.asarray(r, dtype=np.int64)
    S = np.asarray(S, dtype=np.int64)
    return int(r.sum()), int((r * r).sum()), int(S.sum()), int((S * S).sum())


def fit_candidate(r: np.ndarray, S: np.ndarray, t: int, s_max: Fraction = Fraction(1)):
    """Exact (s, o, sse) for range block r against the sum block S under isometry t."""
    B = r.shape[0]
    n = B * B
    TS = isometry(np.asarray(S, dtype=np.int64), t)
    A, Bs, C, E = moments(r, TS)
    X = int((np.asarray(r, dtype=np.int64) * TS).sum())
    P = n * X - A * C
    Q = n * E - C * C
    if Q == 0:
        s = Fraction(0)
    else:
        s = Fraction(4 * P, Q)
        if s > s_max:
            s = Fraction(s_max)
        elif s < -s_max:
            s = -Fraction(s_max)
    o = (Fraction(A) - s * Fraction(C, 4)) / n
    sse = Fraction(0)
    for y in range(B):
        for x in range(B):
            e = Fraction(int(r[y, x])) - s * Fraction(int(TS[y, x]), 4) - o
            sse += e * e
    return s, o, sse
