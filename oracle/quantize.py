"""Oracle: a code format for the fractal codes (test infrastructure only, see the package
docstring).

Section 1 says the domain information and the map coefficients of every range are
stored in the compressed file, but the paper fixes no format, no bit allocation and no
quantiser. This module reads that as: the domain index and the isometry are stored as
integers; the contrast s in [-1, 1] is quantised uniformly to 2^bits_s levels including both
endpoints; the brightness o is quantised uniformly to 2^bits_o levels over the image's observed
range [min o, max o] (stored once per image). Quantisation rounds half to even; every step below
is one binary64 operation, in this order:

    L_s = 2^bits_s - 1;  q_s = clamp(rint(((s + 1) / 2) * L_s), 0, L_s);  s' = (q_s * 2) / L_s - 1
    L_o = 2^bits_o - 1;  q_o = clamp(rint(((o - o_lo) / (o_hi - o_lo)) * L_o), 0, L_o)
                          (q_o = 0 when o_hi == o_lo);  o' = o_lo + (q_o * (o_hi - o_lo)) / L_o
"""
from __future__ import annotations

import numpy as np


def quantize(s: np.ndarray, o: np.ndarray, bits_s: int = 5, bits_o: int = 7):
    """(q_s, q_o, s', o', o_lo, o_hi) for contrast and brightness arrays."""
    s = np.asarray(s, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    Ls = float((1 << bits_s) - 1)
    Lo = float((1 << bits_o) - 1)
    qs = np.clip(np.rint(((s + 1.0) / 2.0) * Ls), 0.0, Ls)
    s_hat = (qs * 2.0) / Ls - 1.0
    o_lo, o_hi = float(np.min(o)), float(np.max(o))
    if o_hi > o_lo:
        qo = np.clip(np.rint(((o - o_lo) / (o_hi - o_lo)) * Lo), 0.0, Lo)
    else:
        qo = np.zeros_like(o)
    o_hat = o_lo + (qo * (o_hi - o_lo)) / Lo
    return qs.astype(np.int64), qo.astype(np.int64), s_hat, o_hat, o_lo, o_hi


def bits_per_range(n_domains: int, bits_s: int = 5, bits_o: int = 7) -> int:
    """Bits one range's code takes: domain index, isometry (3 bits), s and o."""
    return int(np.ceil(np.log2(max(2, n_domains)))) + 3 + bits_s + bits_o
