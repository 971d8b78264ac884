"""Pins for oracle.decode: contractivity, convergence, the collage bound, a dense-matrix
restatement on a tiny image, and the adjoint against central finite differences."""
import numpy as np
import pytest

from oracle import decode, geometry
from oracle import match as omatch
from paper_1206_4880_gb300 import synth


def _random_codes(rng, H, W, B, sigma, smax):
    R = geometry.n_ranges(H, W, B)
    Dn = geometry.n_domains(H, W, B, sigma)
    return {"dom": rng.integers(0, Dn, R), "iso": rng.integers(0, 8, R),
            "s": rng.uniform(-smax, smax, R), "o": rng.uniform(0, 128, R)}


def test_nonexpansive():
    rng = np.random.default_rng(0)
    H = W = 32
    c = _random_codes(rng, H, W, 8, 4, 0.9)
    for _ in range(5):
        x = rng.uniform(0, 255, (H, W))
        y = rng.uniform(0, 255, (H, W))
        a = decode.decode_step(x, c, 8, 4)
        b = decode.decode_step(y, c, 8, 4)
        assert np.max(np.abs(a - b)) <= np.max(np.abs(c["s"])) * np.max(np.abs(x - y)) + 1e-9


def test_geometric_convergence():
    rng = np.random.default_rng(1)
    H = W = 32
    c = _random_codes(rng, H, W, 8, 4, 0.9)
    x = np.full((H, W), 128.0)
    diffs = []
    for _ in range(30):
        y = decode.decode_step(x, c, 8, 4)
        diffs.append(np.max(np.abs(y - x)))
        x = y
    for k in range(1, len(diffs)):
        assert diffs[k] <= 0.9 * diffs[k - 1] + 1e-9


def test_constant_image_decodes_exactly_after_one_iteration():
    img = np.full((32, 48), 97, dtype=np.uint8)
    codes = omatch.encode(img, B=8, sigma=4, K=4)
    assert np.all(codes["s"] == 0) and np.all(codes["o"] == 97)
    x = decode.decode(codes, 32, 48, 8, 4, 1)
    assert np.array_equal(decode.to_u8(x), img)
    assert decode.psnr(decode.to_u8(x), img) == float("inf")


def test_collage_bound(pr1_img):
    img = pr1_img[:64, :64]
    codes = omatch.encode(img, B=8, sigma=4, K=1)
    smax = np.max(np.abs(codes["s"]))
    if smax >= 1.0:
        # the theorem needs a strict contraction; restrict to ranges fitted with |s| < 1
        codes["s"] = np.clip(codes["s"], -0.95, 0.95)
        smax = 0.95
    I = img.astype(np.float64)
    coll = np.max(np.abs(decode.decode_step(I, codes, 8, 4) - I))
    x = decode.decode(codes, 64, 64, 8, 4, 200, x0=I)
    assert np.max(np.abs(I - x)) <= coll / (1 - smax) + 1e-6


def _dense_step(H, W, B, sigma, codes):
    """x -> M x + b as an explicit matrix over the H*W pixels."""
    n = H * W
    M = np.zeros((n, n))
    b = np.zeros(n)
    for r in range(geometry.n_ranges(H, W, B)):
        ry, rx = geometry.range_origin(H, W, B, r)
        dy, dx = geometry.domain_origin(H, W, B, sigma, int(codes["dom"][r]))
        for y in range(B):
            for x in range(B):
                sy, sx = geometry.iso_source(B, int(codes["iso"][r]), y, x)
                row = (ry + y) * W + rx + x
                for a in (0, 1):
                    for c in (0, 1):
                        M[row, (dy + 2 * sy + a) * W + dx + 2 * sx + c] += codes["s"][r] / 4.0
                b[row] = codes["o"][r]
    return M, b


def test_decode_equals_dense_matrix_iteration():
    rng = np.random.default_rng(2)
    H, W = 16, 24
    c = _random_codes(rng, H, W, 8, 2, 1.0)
    M, b = _dense_step(H, W, 8, 2, c)
    x0 = rng.uniform(0, 255, H * W)
    x = x0.copy()
    for _ in range(6):
        x = M @ x + b
    got = decode.decode(c, H, W, 8, 2, 6, x0=x0.reshape(H, W))
    assert np.allclose(got.reshape(-1), x, rtol=0, atol=1e-9)
    # adjoint from the dense matrices: dL/dx_K = g
    g = rng.normal(size=(H, W))
    gs, go = decode.decode_adjoint(c, H, W, 8, 2, 6, g, x0=x0.reshape(H, W))
    R = geometry.n_ranges(H, W, 8)
    # derivative of x_K w.r.t. o_r: sum_{j<K} M^j e_r  (e_r = indicator of range r)
    for r in range(R):
        ry, rx = geometry.range_origin(H, W, 8, r)
        e = np.zeros((H, W))
        e[ry:ry + 8, rx:rx + 8] = 1
        e = e.reshape(-1)
        acc = np.zeros(H * W)
        v = e.copy()
        for _ in range(6):
            acc += v
            v = M @ v
        assert abs(go[r] - g.reshape(-1) @ acc) <= 1e-9 * max(1, abs(go[r]))


@pytest.mark.parametrize("iters", [1, 3, 8])
def test_adjoint_against_central_differences(iters):
    rng = np.random.default_rng(iters)
    H, W = 32, 32
    img = synth.fbm_image(40 + iters, H, W)
    codes = omatch.encode(img, B=8, sigma=4, K=4)
    codes = {k: np.array(codes[k], dtype=np.float64 if k in ("s", "o") else np.int64)
             for k in ("dom", "iso", "s", "o")}
    g = rng.normal(size=(H, W))
    gs, go = decode.decode_adjoint(codes, H, W, 8, 4, iters, g)
    h = 1e-4
    for r in rng.choice(geometry.n_ranges(H, W, 8), 6, replace=False):
        for key, grad in (("s", gs), ("o", go)):
            cp = {k: v.copy() for k, v in codes.items()}
            cm = {k: v.copy() for k, v in codes.items()}
            cp[key][r] += h
            cm[key][r] -= h
            fp = np.sum(g * decode.decode(cp, H, W, 8, 4, iters))
            fm = np.sum(g * decode.decode(cm, H, W, 8, 4, iters))
            fdv = (fp - fm) / (2 * h)
            assert abs(grad[r] - fdv) <= 1e-4 * max(1.0, abs(fdv)), (key, r, grad[r], fdv)


def test_scaled_decode_pins():
    """z = 1 is the ordinary decode; 2x2 averaging of the 2x decode is the 1x decode (the maps
    commute with block averaging: isometries move aligned 2x2 blocks to aligned 2x2 blocks and the
    brightness is constant over a block)."""
    rng = np.random.default_rng(5)
    H, W = 32, 48
    c = _random_codes(rng, H, W, 8, 4, 0.9)
    x1 = decode.decode(c, H, W, 8, 4, 5)
    assert np.allclose(decode.decode_scaled(c, H, W, 8, 4, 5, 1), x1, rtol=0, atol=1e-12)
    x2 = decode.decode_scaled(c, H, W, 8, 4, 5, 2)
    down = x2.reshape(H, 2, W, 2).mean(axis=(1, 3))
    assert np.allclose(down, x1, rtol=0, atol=1e-9)
    x3 = decode.decode_scaled(c, H, W, 8, 4, 3, 3)
    assert np.allclose(x3.reshape(H, 3, W, 3).mean(axis=(1, 3)), decode.decode(c, H, W, 8, 4, 3), atol=1e-9)


def _pool2(x):
    return (x[0::2, 0::2] + x[0::2, 1::2] + x[1::2, 0::2] + x[1::2, 1::2]) / 4.0


@pytest.mark.parametrize("B,sigma", [(8, 8), (8, 4), (8, 2), (8, 6), (16, 4), (16, 8), (16, 2)])
def test_plane_of_averages_iteration(B, sigma):
    """With an even stride the Jacobi iterates' 2x2 averages follow their own iteration on the
    half-size plane: P_{k+1}[cells of r] = s_r T_t(pool2(window of P_k at the domain's half
    position)) + o_r, and x_K = s_r T_t(window of P_{K-1}) + o_r. The decoder's plane form rests on
    this identity; here it is checked against the oracle's full-resolution iteration in binary64."""
    rng = np.random.default_rng(1000 * B + sigma)
    H, W = (48, 64) if B == 8 else (64, 96)
    codes = _random_codes(rng, H, W, B, sigma, 0.9)
    x0 = rng.uniform(0, 255, (H, W))
    iters = 4
    xs = [x0]
    for _ in range(iters):
        xs.append(decode.decode_step(xs[-1], codes, B, sigma))
    R = geometry.n_ranges(H, W, B)
    hb = B // 2
    P = _pool2(x0)
    for k in range(iters):
        assert np.max(np.abs(P - _pool2(xs[k]))) <= 1e-9, k
        nxt = np.empty_like(P)
        last = np.empty_like(x0)
        for r in range(R):
            dy, dx = geometry.domain_origin(H, W, B, sigma, int(codes["dom"][r]))
            ry, rx = geometry.range_origin(H, W, B, r)
            win = P[dy // 2:dy // 2 + B, dx // 2:dx // 2 + B]
            t, s, o = int(codes["iso"][r]), codes["s"][r], codes["o"][r]
            nxt[ry // 2:ry // 2 + hb, rx // 2:rx // 2 + hb] = s * geometry.isometry(_pool2(win), t) + o
            last[ry:ry + B, rx:rx + B] = s * geometry.isometry(win, t) + o
        # the full-resolution step from the plane alone
        assert np.max(np.abs(last - xs[k + 1])) <= 1e-9, k
        P = nxt


def _iso_scatter(out, q0y, q0x, vals, t):
    """out[q0 + src_t(p)] += vals[p] for the p of a square block (the transpose of
    geometry.isometry restricted to a window at q0)."""
    n = vals.shape[0]
    for y in range(n):
        for x in range(n):
            sy, sx = geometry.iso_source(n, t, y, x)
            out[q0y + sy, q0x + sx] += vals[y, x]


@pytest.mark.parametrize("B,sigma", [(8, 8), (8, 2), (16, 4)])
def test_plane_of_averages_adjoint(B, sigma):
    """The adjoint on the plane (nu_k = dL/dP_k: nu_{K-1} = M^T dL/dx_K, nu_k = H^T nu_{k+1}, the
    last step's gradient terms from dL/dx_K and the window of P_{K-1}, the others from nu_{k+1} and
    the 2x2 means of the windows of P_k) equals the oracle's full-resolution adjoint."""
    rng = np.random.default_rng(77 * B + sigma)
    H, W = (48, 64) if B == 8 else (64, 96)
    codes = _random_codes(rng, H, W, B, sigma, 0.9)
    x0 = rng.uniform(0, 255, (H, W))
    g = rng.normal(size=(H, W))
    iters = 4
    gs_ref, go_ref = decode.decode_adjoint(codes, H, W, B, sigma, iters, g, x0=x0)
    R = geometry.n_ranges(H, W, B)
    hb = B // 2
    geo = []
    for r in range(R):
        dy, dx = geometry.domain_origin(H, W, B, sigma, int(codes["dom"][r]))
        ry, rx = geometry.range_origin(H, W, B, r)
        geo.append((dy // 2, dx // 2, ry, rx, int(codes["iso"][r]), codes["s"][r], codes["o"][r]))
    # forward on the plane
    Ps = [_pool2(x0)]
    for _ in range(iters - 1):
        P, nxt = Ps[-1], np.empty_like(Ps[-1])
        for wy, wx, ry, rx, t, s, o in geo:
            nxt[ry // 2:ry // 2 + hb, rx // 2:rx // 2 + hb] = s * geometry.isometry(_pool2(P[wy:wy + B, wx:wx + B]), t) + o
        Ps.append(nxt)
    gs, go = np.zeros(R), np.zeros(R)
    # the last step: terms from dL/dx_K, then nu_{K-1} = M^T dL/dx_K
    P = Ps[-1]
    nu = np.zeros_like(P)
    for r, (wy, wx, ry, rx, t, s, o) in enumerate(geo):
        lr = g[ry:ry + B, rx:rx + B]
        gs[r] += np.sum(lr * geometry.isometry(P[wy:wy + B, wx:wx + B], t))
        go[r] += np.sum(lr)
        _iso_scatter(nu, wy, wx, s * lr, t)
    # the other steps, on the plane
    for k in range(iters - 2, -1, -1):
        P = Ps[k]
        prev = np.zeros_like(P)
        for r, (wy, wx, ry, rx, t, s, o) in enumerate(geo):
            nr = nu[ry // 2:ry // 2 + hb, rx // 2:rx // 2 + hb]
            gs[r] += np.sum(nr * geometry.isometry(_pool2(P[wy:wy + B, wx:wx + B]), t))
            go[r] += np.sum(nr)
            # H^T: each cell's value, times s / 4, to the four plane pixels of its 2x2 source block
            blk = np.zeros((hb, hb))
            _iso_scatter(blk, 0, 0, (s / 4.0) * nr, t)
            prev[wy:wy + B, wx:wx + B] += np.repeat(np.repeat(blk, 2, 0), 2, 1)
        nu = prev
    for a, b in ((gs, gs_ref), (go, go_ref)):
        assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b))
