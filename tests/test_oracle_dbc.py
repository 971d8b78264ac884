"""Pins for oracle.dbc: hand-computed box counts, invariants, log2 rounding, classes."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import dbc
from oracle import match as omatch


def test_log2_correctly_rounded_against_libm():
    for n in range(1, 1025):
        v = dbc.log2_cr(n)
        lib = math.log2(n)
        assert abs(v - lib) <= math.ulp(lib), n
        if n & (n - 1) == 0:
            assert v == float(n.bit_length() - 1)
    # additivity within rounding: log2(a*b) = log2 a + log2 b
    for a in (3, 5, 7, 9, 11):
        for b in (3, 6, 10, 13):
            assert abs(dbc.log2_cr(a * b) - (dbc.log2_cr(a) + dbc.log2_cr(b))) <= 4 * math.ulp(8.0)


def test_constant_block():
    blk = np.full((8, 8), 77)
    c, fd = dbc.range_fd(blk)
    assert c == [16, 4] and fd == 2.0


def test_checkerboard_block():
    blk = (np.indices((8, 8)).sum(axis=0) % 2) * 255
    c, fd = dbc.range_fd(blk)
    assert c == [64, 8] and fd == 3.0


def test_constant_quadrants():
    blk = np.zeros((8, 8), dtype=np.int64)
    blk[:4, 4:] = 255
    blk[4:, :4] = 100
    blk[4:, 4:] = 200
    c, fd = dbc.range_fd(blk)
    assert c == [16, 4] and fd == 2.0


def test_single_spike_by_hand():
    # 2x2 cell with 0 and 200: floor(200/64) - 0 + 1 = 4 boxes, the other 15 cells 1 box;
    # its 4x4 cell: floor(200/128) + 1 = 2, the other three 1.
    blk = np.zeros((8, 8), dtype=np.int64)
    blk[5, 2] = 200
    c, fd = dbc.range_fd(blk)
    assert c == [19, 5]
    assert fd == dbc.log2_cr(19) - dbc.log2_cr(5)


def test_sixteen_block_by_hand_and_polyfit():
    # B = 16: s = 2, 4, 8 with box heights 32, 64, 128 (pixels)
    blk = np.zeros((16, 16), dtype=np.int64)
    blk[0, 0] = 255
    c, fd = dbc.range_fd(blk)
    assert c == [64 + 7, 16 + 3, 4 + 1]
    x = np.log2(16 / np.array([2, 4, 8]))
    y = np.log2(np.array(c, dtype=np.float64))
    assert abs(fd - np.polyfit(x, y, 1)[0]) < 1e-12


@pytest.mark.parametrize("M", [8, 16])
def test_invariants_random(M):
    rng = np.random.default_rng(M)
    for _ in range(300):
        blk = rng.integers(0, 256, (M, M))
        c, fd = dbc.range_fd(blk)
        if M == 8:
            assert 16 <= c[0] <= 64 and 4 <= c[1] <= 8
            assert 2 * c[1] <= c[0] <= 8 * c[1]
        assert 1.0 <= fd <= 3.0 + 1e-12
        # on sums (G = 1024) the counts equal those of the 2x2 average with G = 256
        S = rng.integers(0, 1021, (M, M))
        cs = dbc.box_counts(S, 1024)
        avg = S / 4.0
        manual = []
        for s in dbc.scales(M):
            h = s * 256 / M
            tot = 0
            for cy in range(0, M, s):
                for cx in range(0, M, s):
                    cell = avg[cy:cy + s, cx:cx + s]
                    tot += int(math.floor(cell.max() / h)) - int(math.floor(cell.min() / h)) + 1
            manual.append(tot)
        assert cs == manual


@pytest.mark.parametrize("M", [8, 16])
def test_batch_counts_equal_loop(M):
    rng = np.random.default_rng(10 + M)
    blocks = rng.integers(0, 1021, (50, M, M))
    blocks[0] = 0
    blocks[1] = 1020
    bc = omatch.box_counts_all(blocks, 1024)
    fd = omatch.fd_all(bc, M)
    for i in range(50):
        c, f = dbc.domain_fd(blocks[i])
        assert list(bc[i]) == c
        assert fd[i] == f


def test_classes():
    K = 16
    F_l, F_m = 1.25, 2.75
    f = np.array([F_l, F_m, 0.5, 3.5, 2.0, 1.9, 2.6])
    b = dbc.classify(f, F_l, F_m, K)
    assert b[0] == 0 and b[1] == K - 1 and b[2] == 0 and b[3] == K - 1
    assert dbc.classify(f, 2.0, 2.0, K).tolist() == [0] * len(f)
    assert dbc.classify(f, F_l, F_m, 1).tolist() == [0] * len(f)
    # exact-rational floor agrees wherever K*v is not within 1e-9 of an integer
    rng = np.random.default_rng(3)
    vals = rng.uniform(F_l, F_m, 2000)
    bins = dbc.classify(vals, F_l, F_m, K)
    assert np.all(np.diff(bins[np.argsort(vals)]) >= 0)
    for v, bb in zip(vals, bins):
        q = (Fraction(float(v)) - Fraction(F_l)) / (Fraction(F_m) - Fraction(F_l)) * K
        if abs(q - round(q)) > Fraction(1, 10 ** 9):
            assert bb == min(K - 1, max(0, math.floor(q)))
    assert dbc.default_half_width(8) == 2 and dbc.default_half_width(16) == 5
    assert dbc.default_half_width(32) == 10 and dbc.default_half_width(1) == 0
