"""Pins for oracle.geometry: Table 1 counts, isometry group laws, contraction by 2x2 sums."""
import os

import numpy as np
import pytest

from oracle import geometry
from oracle import match as omatch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_counts.txt")


def _table1():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_table1_counts():
    """Section 2, Table 1: 8x8 ranges, 16x16 domains at every pixel (stride 1)."""
    rows = _table1()
    assert [r[0] for r in rows] == [64, 128, 256, 512, 1024]
    for n, ranges, domains, comps in rows:
        assert geometry.n_ranges(n, n, 8) == ranges
        assert geometry.n_domains(n, n, 8, 1) == domains
        prod = ranges * domains
        if comps > 0:
            assert prod == comps
        else:
            # the lower bound printed for n = 1024 (more than 3.5e10) is not met by the product;
            # Section 2's own estimate of the same case (about 2^34) is.
            assert prod == 16384 * 1009 * 1009 == 16_680_239_104
            assert prod < -comps
            assert 0.95 < prod / 2 ** 34 < 1.0


def test_section2_example():
    """Section 2: 1024x1024, 2^14 ranges, 1009 x 1009 domains."""
    assert geometry.n_ranges(1024, 1024, 8) == 2 ** 14
    assert geometry.domain_grid(1024, 1024, 8, 1) == (1009, 1009)


def _perm(B, t):
    """Isometry as a permutation of the B*B flat indices: out[i] = in[perm[i]]."""
    X = np.arange(B * B).reshape(B, B)
    return geometry.isometry(X, t).reshape(-1)


@pytest.mark.parametrize("B", [2, 8, 16])
def test_isometry_group_laws(B):
    perms = [_perm(B, t) for t in range(8)]
    ident = np.arange(B * B)
    # each map is a bijection, all 8 are distinct
    for p in perms:
        assert np.array_equal(np.sort(p), ident)
    assert len({tuple(p) for p in perms}) == 8
    # closure under composition
    keys = {tuple(p): t for t, p in enumerate(perms)}
    for a in range(8):
        for b in range(8):
            assert tuple(perms[b][perms[a]]) in keys
    r = perms[1]
    r2 = r[r]
    r3 = r2[r]
    r4 = r3[r]
    assert np.array_equal(r2, perms[2])
    assert np.array_equal(r3, perms[3])
    assert np.array_equal(r4, ident)
    for t in (2, 4, 5, 6, 7):
        assert np.array_equal(perms[t][perms[t]], ident)
    for t in range(8):
        X = np.random.default_rng(t).integers(0, 255, (B, B))
        assert np.array_equal(geometry.isometry(geometry.isometry(X, t), geometry.INVERSE[t]), X)


def test_isometry_library_and_hand_example():
    """Against numpy's rotations/flips, and a 2x2 block [[a,b],[c,d]] rotated clockwise."""
    X = np.random.default_rng(0).integers(0, 1000, (8, 8))
    lib = [X, np.rot90(X, -1), np.rot90(X, 2), np.rot90(X, 1), np.fliplr(X), np.flipud(X), X.T,
           np.rot90(X, 2).T]
    for t in range(8):
        assert np.array_equal(geometry.isometry(X, t), lib[t]), t
    a, b, c, d = 1, 2, 3, 4
    assert geometry.isometry(np.array([[a, b], [c, d]]), 1).tolist() == [[c, a], [d, b]]


@pytest.mark.parametrize("H,W,sigma", [(16, 16, 1), (24, 40, 2), (32, 24, 3), (48, 32, 8)])
def test_domain_sums_vectorised_equals_loop(H, W, sigma):
    img = np.random.default_rng(H * W + sigma).integers(0, 256, (H, W)).astype(np.uint8)
    ds = omatch.domain_sums_all(img, 8, sigma)
    assert ds.shape[0] == geometry.n_domains(H, W, 8, sigma)
    for d in range(ds.shape[0]):
        assert np.array_equal(ds[d], geometry.domain_sum_block(img, 8, sigma, d))
    rb = omatch.range_blocks_all(img, 8)
    for r in range(rb.shape[0]):
        assert np.array_equal(rb[r], geometry.range_block(img, 8, r))
    # a 2x2 sum is four times the 2x2 average (the "resizing" of Section 1)
    d = ds.shape[0] - 1
    dy, dx = geometry.domain_origin(H, W, 8, sigma, d)
    avg = img[dy:dy + 16, dx:dx + 16].astype(np.float64).reshape(8, 2, 8, 2).mean(axis=(1, 3))
    assert np.array_equal(ds[d], (4 * avg).astype(np.int64))
