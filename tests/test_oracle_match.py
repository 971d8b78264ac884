"""Pins for oracle.fit and the exact matcher: least squares against numpy, the clamp against a
1-D brute force, the whole search against an explicit FP64 loop on tiny images, and the pool
laws (one class = exhaustive search, wider pools never do worse)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fit, geometry, pools
from oracle import match as omatch
from paper_1206_4880_gb300 import synth


def _rand_pair(rng, B=8):
    r = rng.integers(0, 256, (B, B))
    S = rng.integers(0, 1021, (B, B))
    return r, S


def test_fit_unclamped_matches_lstsq():
    rng = np.random.default_rng(0)
    done = 0
    while done < 40:
        r, S = _rand_pair(rng)
        # make the range a noisy scaled copy so |s| < 1 and the fit is not clamped
        t = int(rng.integers(0, 8))
        D = geometry.isometry(S, t) / 4.0
        r = np.clip(np.rint(0.6 * D + 40 + rng.normal(0, 5, D.shape)), 0, 255).astype(np.int64)
        s, o, sse = fit.fit_candidate(r, S, t)
        if abs(s) >= 1:
            continue
        A = np.stack([D.reshape(-1), np.ones(64)], axis=1)
        (s_ls, o_ls), *_ = np.linalg.lstsq(A, r.reshape(-1).astype(np.float64), rcond=None)
        assert abs(float(s) - s_ls) < 1e-9 and abs(float(o) - o_ls) < 1e-7
        res = r.reshape(-1) - A @ np.array([s_ls, o_ls])
        assert abs(float(sse) - float(res @ res)) < 1e-6 * max(1.0, float(res @ res))
        done += 1


def test_fit_clamped_against_1d_bruteforce():
    rng = np.random.default_rng(1)
    done = 0
    while done < 20:
        r, S = _rand_pair(rng)
        S = (S // 8) + 300  # low-contrast domain: the optimal |s| exceeds 1
        t = int(rng.integers(0, 8))
        s, o, sse = fit.fit_candidate(r, S, t)
        if abs(s) != 1:
            continue
        D = geometry.isometry(S, t).reshape(-1) / 4.0
        rv = r.reshape(-1).astype(np.float64)
        grid = np.linspace(-1.0, 1.0, 4001)
        best = np.inf
        for sg in grid:
            og = np.mean(rv - sg * D)
            e = rv - sg * D - og
            best = min(best, float(e @ e))
        assert float(sse) <= best + 1e-9
        assert float(sse) >= best - 1e-3 * best
        done += 1


def test_flat_domain_and_flat_range():
    r = np.full((8, 8), 90)
    S = np.full((8, 8), 400)
    s, o, sse = fit.fit_candidate(r, S, 3)
    assert s == 0 and o == 90 and sse == 0
    r2 = np.random.default_rng(2).integers(0, 256, (8, 8))
    s, o, sse = fit.fit_candidate(r2, S, 0)
    assert s == 0 and o == Fraction(int(r2.sum()), 64)


def _bruteforce_fp64(img, B, sigma):
    """Exhaustive search written independently: FP64 normal equations, clamp, re-solve o."""
    H, W = img.shape
    R = geometry.n_ranges(H, W, B)
    Dn = geometry.n_domains(H, W, B, sigma)
    out = []
    for r in range(R):
        rv = geometry.range_block(img, B, r).astype(np.float64).reshape(-1)
        errs = np.empty((Dn, 8))
        for d in range(Dn):
            S = geometry.domain_sum_block(img, B, sigma, d).astype(np.float64) / 4.0
            for t in range(8):
                dv = geometry.isometry(S, t).reshape(-1)
                var = np.sum((dv - dv.mean()) ** 2)
                s = 0.0 if var == 0 else np.sum((dv - dv.mean()) * (rv - rv.mean())) / var
                s = min(1.0, max(-1.0, s))
                o = np.mean(rv - s * dv)
                e = rv - s * dv - o
                errs[d, t] = e @ e
        out.append(errs)
    return out


@pytest.mark.parametrize("H,W,sigma", [(16, 16, 1), (24, 24, 2), (32, 24, 3), (32, 32, 4)])
def test_full_search_equals_bruteforce(H, W, sigma):
    img = synth.fbm_image(100 + H + sigma, H, W)
    codes = omatch.encode(img, B=8, sigma=sigma, K=1)
    bf = _bruteforce_fp64(img, 8, sigma)
    for r, errs in enumerate(bf):
        emin = errs.min()
        tol = 1e-7 * max(1.0, emin)
        assert abs(codes["sse"][r] - emin) <= tol
        assert errs[codes["dom"][r], codes["iso"][r]] <= emin + tol
        # the chosen code is the first (domain, isometry) within tolerance of the minimum
        # unless FP64 rounding separates exact ties
        first = np.argwhere(errs <= emin + tol)[0]
        assert (codes["dom"][r], codes["iso"][r]) == (first[0], first[1]) or \
            abs(errs[first[0], first[1]] - errs[codes["dom"][r], codes["iso"][r]]) <= tol


def test_matcher_outputs_equal_exact_fit(pr1_img):
    img = pr1_img[:64, :64]
    codes = omatch.encode(img, B=8, sigma=4, K=4)
    for r in range(codes["dom"].size):
        rb = geometry.range_block(img, 8, r)
        S = geometry.domain_sum_block(img, 8, 4, int(codes["dom"][r]))
        s, o, sse = fit.fit_candidate(rb, S, int(codes["iso"][r]))
        assert codes["s"][r] == float(s)
        assert abs(codes["o"][r] - float(o)) <= 1e-12 * max(1.0, abs(float(o)))
        assert abs(codes["sse"][r] - float(sse)) <= 1e-9 * max(1.0, float(sse))


def test_one_class_and_wide_pools_are_full_search(pr1_img):
    img = pr1_img[:96, :128]
    full = omatch.encode(img, B=8, sigma=4, K=1)
    assert np.all(full["pool_size"] == geometry.n_domains(96, 128, 8, 4))
    for K in (2, 5, 9):
        wide = omatch.encode(img, B=8, sigma=4, K=K, w=K - 1)
        for key in ("dom", "iso", "s", "o", "sse"):
            assert np.array_equal(wide[key], full[key]), (K, key)
    lit = omatch.encode(img, B=8, sigma=4, K=8, mode="literal",
                        cls=None)  # D_f finite: a subset
    assert np.all(lit["sse"] >= full["sse"] - 1e-9)
    cls = omatch.classify_image(img, 8, 4, 8)
    allp = [pools.literal_pool(f, cls["dom_fd"], np.inf) for f in cls["range_fd"]]
    inf = omatch.match_pools(img, 8, 4, np.arange(len(allp)), allp)
    assert np.array_equal(inf["dom"], full["dom"]) and np.array_equal(inf["iso"], full["iso"])


def test_wider_pool_never_worse(pr1_img):
    img = pr1_img[64:160, 32:160]
    K = 12
    prev = None
    for w in range(0, K):
        c = omatch.encode(img, B=8, sigma=4, K=K, w=w)
        if prev is not None:
            assert np.all(c["sse"] <= prev["sse"] + 1e-9)
            assert np.all(c["pool_size"] >= prev["pool_size"])
        prev = c


def test_flat_range_takes_first_pool_domain():
    img = synth.fbm_image(5, 48, 48)
    img[8:16, 16:24] = 131  # range 1*6+2 = 8 is flat
    codes = omatch.encode(img, B=8, sigma=2, K=6)
    r = 8
    p = pools.class_pool(codes["cls"]["range_bin"][r], codes["cls"]["dom_bin"], 2)
    assert codes["dom"][r] == p[0] and codes["iso"][r] == 0 and codes["sse"][r] == 0.0


def test_empty_class_window_falls_back_to_all_domains():
    bins = np.array([0, 0, 3, 3])
    assert pools.class_pool(1, bins, 0).tolist() == [0, 1, 2, 3]
    assert pools.class_pool(3, bins, 0).tolist() == [2, 3]
    assert pools.class_pool(1, bins, 1).tolist() == [0, 1]


def test_sixteen_block_full_search_small():
    img = synth.fbm_image(9, 48, 48)
    codes = omatch.encode(img, B=16, sigma=8, K=1)
    for r in range(codes["dom"].size):
        rb = geometry.range_block(img, 16, r)
        best = None
        for d in range(geometry.n_domains(48, 48, 16, 8)):
            S = geometry.domain_sum_block(img, 16, 8, d)
            for t in range(8):
                sse = fit.fit_candidate(rb, S, t)[2]
                if best is None or sse < best[0]:
                    best = (sse, d, t)
        assert (codes["dom"][r], codes["iso"][r]) == (best[1], best[2])
        assert abs(codes["sse"][r] - float(best[0])) <= 1e-9 * max(1.0, float(best[0]))

