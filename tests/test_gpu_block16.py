"""GPU parity of the 16x16-range pass (32x32 domains, n = 256 pixels per block) against the CPU
oracle, through the C ABI: classification with three box-count scales, pools, both matching
engines, batched encoding, decoding and the adjoint.

Bars as for 8x8 ranges: moments, box counts, FD bit patterns and classes bit-exact; chosen
(domain, isometry) identical; s and o within 1e-6; sse within 1e-9 relative; decoded iterates
within 2e-3 of the FP64 oracle; gradients within 1e-4 relative.
"""
import os

import numpy as np
import pytest
import torch

from oracle import dbc as odbc
from oracle import decode as odec
from oracle import match as omatch
from oracle import pools as opools
from paper_1206_4880_gb300 import fic, synth

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1  # oracle threads: every host core

ENGINES = ["simt", "tensor"]

# (H, W, sigma, K, w, seed): ragged cases spanning several 256-range tiles and odd strides
SMALL16 = [
    (32, 32, 1, 3, -1, 51),
    (48, 64, 2, 4, 0, 52),
    (96, 80, 3, 5, 1, 53),
    (160, 224, 4, 7, -1, 54),
    (128, 128, 8, 1, -1, 55),
    (272, 304, 4, 16, 2, 56),
    (256, 256, 8, 16, -1, 1000),
]


def _img(H, W, seed):
    return synth.pr1_image() if seed == 1000 else synth.fbm_image(seed, H, W)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _params(sigma, K, w, engine="simt"):
    return fic.EncodeParams(domain_stride=sigma, num_classes=K, half_width=w, engine=engine, block=16)


def _need_tensor(engine):
    if engine == "tensor":
        major, minor = torch.cuda.get_device_capability()
        if (major, minor) != (10, 3):
            pytest.skip("tensor engine needs sm_103")
        assert fic.engine_available("tensor"), "tensor engine missing on an sm_103 device"


def _compare_codes(gpu, ref, idx=None):
    idx = np.arange(gpu["dom"].numel()) if idx is None else np.asarray(idx)
    g = {k: v.cpu().numpy()[idx] for k, v in gpu.items()}
    bad = np.nonzero((g["dom"] != ref["dom"]) | (g["iso"] != ref["iso"]))[0]
    assert bad.size == 0, f"{bad.size} codes differ, first ranges {idx[bad[:8]]}: gpu " \
        f"{list(zip(g['dom'][bad[:4]], g['iso'][bad[:4]], g['sse'][bad[:4]]))} ref " \
        f"{list(zip(ref['dom'][bad[:4]], ref['iso'][bad[:4]], ref['sse'][bad[:4]]))}"
    assert np.max(np.abs(g["s"] - ref["s"])) <= 1e-6
    assert np.max(np.abs(g["o"] - ref["o"])) <= 1e-6
    assert np.all(np.abs(g["sse"] - ref["sse"]) <= 1e-9 * np.maximum(1.0, ref["sse"]))


@pytest.mark.parametrize("case", SMALL16)
def test_classify16_bit_exact(case):
    H, W, sigma, K, w, seed = case
    img = _img(H, W, seed)
    st = fic.classify(_t(img), _params(sigma, K, w))
    torch.cuda.synchronize()
    cls = omatch.classify_image(img, 16, sigma, K)
    g = {k: v.cpu().numpy() for k, v in st.items()}
    for k in ("range_sum", "range_sumsq", "dom_sum", "dom_sumsq", "range_counts", "dom_counts",
              "range_bin", "dom_bin"):
        assert np.array_equal(g[k], cls[k]), k
    assert g["range_counts"].shape[1] == 3
    assert np.array_equal(g["range_fd"].view(np.int64), cls["range_fd"].view(np.int64))
    assert np.array_equal(g["dom_fd"].view(np.int64), cls["dom_fd"].view(np.int64))
    assert g["fd_extent"][0] == cls["F_l"] and g["fd_extent"][1] == cls["F_m"]


@pytest.mark.parametrize("case", SMALL16[:4])
def test_pools16_exact(case):
    H, W, sigma, K, w, seed = case
    img = _img(H, W, seed)
    p = _params(sigma, K, w)
    st = fic.classify(_t(img), p)
    po = fic.build_pools(st, H, W, p)
    torch.cuda.synchronize()
    cls = omatch.classify_image(img, 16, sigma, K)
    dom_order = po["dom_order"].cpu().numpy()
    assert np.array_equal(dom_order, np.argsort(cls["dom_bin"], kind="stable"))
    ww = odbc.default_half_width(K) if w < 0 else w
    lo, hi = po["win_lo"].cpu().numpy(), po["win_hi"].cpu().numpy()
    for r in range(lo.size):
        pool = opools.class_pool(cls["range_bin"][r], cls["dom_bin"], ww)
        assert np.array_equal(np.sort(dom_order[lo[r]:hi[r]]), pool), r


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("case", SMALL16)
def test_encode16_parity_small(case, engine):
    _need_tensor(engine)
    H, W, sigma, K, w, seed = case
    img = _img(H, W, seed)
    info = fic.new_info("cuda")
    codes = fic.encode(_t(img), _params(sigma, K, w, engine), info=info)
    torch.cuda.synchronize()
    ref = omatch.encode(img, B=16, sigma=sigma, K=K, w=None if w < 0 else w, n_threads=NT)
    _compare_codes(codes, ref)
    rep = fic.read_info(info)
    assert rep["matches"] == int(ref["pool_size"].sum()) * 8
    assert rep["device_error"] == 0
    if engine == "tensor":
        assert rep["fallback_ranges"] <= max(4, codes["dom"].numel() // 20), rep


@pytest.mark.parametrize("engine", ENGINES)
def test_encode16_flat_and_extreme_images(engine):
    _need_tensor(engine)
    cases = [np.full((64, 64), 200, np.uint8), np.zeros((32, 48), np.uint8)]
    img = synth.fbm_image(78, 128, 128)
    img[16:112, 32:96] = 31  # flat ranges and flat (Q = 0) domains
    cases.append(img)
    # 0/255 checkerboard: the largest |X|, |P| and Q the 16x16 fit can meet
    cases.append(((np.indices((96, 96)).sum(axis=0) % 2) * 255).astype(np.uint8))
    # 0/255 stripes and a hard step: extreme centred operands for the Cauchy-Schwarz bound
    st = np.zeros((64, 96), np.uint8)
    st[:, ::2] = 255
    cases.append(st)
    step = np.zeros((64, 64), np.uint8)
    step[:, 32:] = 255
    cases.append(step)
    for im in cases:
        for K, sigma in ((4, 2), (1, 4), (255, 8)):
            codes = fic.encode(_t(im), _params(sigma, K, -1, engine))
            torch.cuda.synchronize()
            ref = omatch.encode(im, B=16, sigma=sigma, K=K, n_threads=NT)
            _compare_codes(codes, ref)


def test_full_search16_simt_equals_k1_tensor():
    _need_tensor("tensor")
    img = _t(synth.fbm_image(9, 192, 256))
    a = fic.encode(img, _params(4, 1, -1, "simt"))
    b = fic.encode(img, _params(4, 1, -1, "tensor"))
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("engine", ENGINES)
def test_encode16_batched_equals_oracle(engine):
    _need_tensor(engine)
    shapes = [(64, 48, 61), (160, 224, 62), (32, 32, 63), (256, 256, 64)]
    imgs = [synth.fbm_image(seed, H, W) for H, W, seed in shapes]
    p = _params(4, 7, -1, engine)
    info = fic.new_info("cuda")
    outs = fic.encode_batched([_t(im) for im in imgs], p, info=info)
    torch.cuda.synchronize()
    total = 0
    for im, out in zip(imgs, outs):
        ref = omatch.encode(im, B=16, sigma=4, K=7, n_threads=NT)
        _compare_codes(out, ref)
        total += int(ref["pool_size"].sum()) * 8
    rep = fic.read_info(info)
    assert rep["matches"] == total and rep["device_error"] == 0


@pytest.mark.parametrize("engine", ENGINES)
def test_encode16_1024_sampled(engine):
    """1024x1024, stride 4, K = 16 with 16x16 ranges: classification bit-exact, codes on 400
    seeded ranges plus every range the tensor engine re-searched exactly."""
    _need_tensor(engine)
    img = synth.image_1024()
    p = _params(4, 16, -1, engine)
    ws = torch.empty(fic.encode_workspace_size(1024, 1024, p), dtype=torch.uint8, device="cuda")
    info = fic.new_info("cuda")
    codes = fic.encode(_t(img), p, workspace=ws, info=info)
    fb = fic.fallback_ranges(1024, 1024, p, ws).cpu().numpy()
    st = fic.classify(_t(img), p)
    torch.cuda.synchronize()
    cls = omatch.classify_image(img, 16, 4, 16)
    assert np.array_equal(st["range_bin"].cpu().numpy(), cls["range_bin"])
    assert np.array_equal(st["dom_bin"].cpu().numpy(), cls["dom_bin"])
    R = 64 * 64
    rng = np.random.default_rng(2016)
    sample = np.unique(np.concatenate([[0, R - 1, 63, R - 64], rng.choice(R, 400, replace=False), fb]))
    ref = omatch.encode(img, B=16, sigma=4, K=16, range_ids=sample, n_threads=NT, cls=cls)
    _compare_codes(codes, ref, sample)
    rep = fic.read_info(info)
    ww = odbc.default_half_width(16)
    total = sum(opools.class_pool(b, cls["dom_bin"], ww).size for b in cls["range_bin"])
    assert rep["matches"] == total * 8 and rep["device_error"] == 0
    assert fb.size == rep["fallback_ranges"]
    if engine == "tensor":
        assert rep["fallback_ranges"] <= R // 20, rep


def _codes_gpu(c):
    return {"dom": torch.from_numpy(np.asarray(c["dom"], np.int32)).cuda(),
            "iso": torch.from_numpy(np.asarray(c["iso"], np.int32)).cuda(),
            "s": torch.from_numpy(np.asarray(c["s"], np.float64)).cuda(),
            "o": torch.from_numpy(np.asarray(c["o"], np.float64)).cuda()}


@pytest.mark.parametrize("sigma", [4, 8, 2, 6])
def test_decode16_parity_and_adjoint(sigma):
    """Decoding and its adjoint with 16x16 ranges. Even strides run on the plane of 2x2 averages:
    sigma = 4 and 8 with float2 window loads and 2x2-block transposes (sigma / 2 even), 2 and 6
    with single loads and per-pixel transposes (sigma / 2 odd)."""
    H, W, iters = 96, 128, 6
    img = synth.fbm_image(71, H, W)
    codes = omatch.encode(img, B=16, sigma=sigma, K=5, n_threads=NT)
    p = fic.EncodeParams(domain_stride=sigma, num_classes=5, block=16)
    for it in (1, iters):
        x = fic.decode(_codes_gpu(codes), H, W, p, it)
        torch.cuda.synchronize()
        assert np.max(np.abs(x.cpu().numpy() - odec.decode(codes, H, W, 16, sigma, it))) <= 2e-3
    z = 2
    xs = fic.decode_scaled(_codes_gpu(codes), H, W, p, z, 3)
    torch.cuda.synchronize()
    assert np.max(np.abs(xs.cpu().numpy() - odec.decode_scaled(codes, H, W, 16, sigma, 3, z))) <= 2e-3
    g = np.random.default_rng(16).normal(size=(H, W))
    gs_ref, go_ref = odec.decode_adjoint(codes, H, W, 16, sigma, iters, g)
    gs, go = fic.decode_backward(_codes_gpu(codes), H, W, p, iters, 2, torch.from_numpy(g.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    for a, b in ((gs.cpu().numpy(), gs_ref), (go.cpu().numpy(), go_ref)):
        assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(b))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("case", [c for c in SMALL16 if c[3] > 1])
def test_encode16_literal_window(case, engine):
    """Section 3.1 Eq. 3 on the FD values of 16x16 blocks: FD_r - D_f <= FD_d <= FD_r + D_f. The
    domains and ranges are ordered by FD value (stable), each range's window equals the oracle's
    literal pool, and the codes equal the oracle's literal-mode codes."""
    _need_tensor(engine)
    H, W, sigma, K, w, seed = case
    img = _img(H, W, seed)
    p = fic.EncodeParams(domain_stride=sigma, num_classes=K, half_width=w, engine=engine, block=16,
                         literal=True)
    info = fic.new_info("cuda")
    codes = fic.encode(_t(img), p, info=info)
    st = fic.classify(_t(img), p)
    po = fic.build_pools(st, H, W, p)
    torch.cuda.synchronize()
    ref = omatch.encode(img, B=16, sigma=sigma, K=K, mode="literal", n_threads=NT)
    _compare_codes(codes, ref)
    rep = fic.read_info(info)
    assert rep["matches"] == int(ref["pool_size"].sum()) * 8 and rep["device_error"] == 0
    cls = ref["cls"]
    Df = opools.fractal_distance(cls["F_l"], cls["F_m"])
    dom_order = po["dom_order"].cpu().numpy()
    assert np.array_equal(dom_order, np.argsort(cls["dom_fd"], kind="stable"))
    assert np.array_equal(po["range_order"].cpu().numpy(), np.argsort(cls["range_fd"], kind="stable"))
    lo, hi = po["win_lo"].cpu().numpy(), po["win_hi"].cpu().numpy()
    for r in range(lo.size):
        pool = opools.literal_pool(cls["range_fd"][r], cls["dom_fd"], Df)
        assert np.array_equal(np.sort(dom_order[lo[r]:hi[r]]), pool), r
    # bucket offsets: monotone, ending at the domain count, buckets of equal FD
    off = po["bin_off"].cpu().numpy()
    assert off.size == fic.LITERAL16_OFFSETS and off[0] == 0 and off[-1] == dom_order.size
    assert np.all(np.diff(off) >= 0)
    fd_sorted = cls["dom_fd"][dom_order]
    for k in np.nonzero(np.diff(off))[0]:
        run = fd_sorted[off[k]:off[k + 1]]
        assert np.all(run == run[0])
