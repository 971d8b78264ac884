"""GPU parity of classification, pools and encoding against the CPU oracle, through the C ABI.

Bars: block moments, box counts, FD bit patterns and classes bit-exact; pool orders and windows
exact; chosen (domain, isometry) identical; s and o within 1e-6 (they are formed from the same
exact integers, so in practice equal); sse within 1e-9 relative.
"""
import os

import numpy as np
import pytest
import torch

from oracle import dbc as odbc
from oracle import match as omatch
from oracle import pools as opools
from paper_1206_4880_gb300 import fic, synth

pytestmark = pytest.mark.gpu

ENGINES = ["simt", "tensor"]
NT = os.cpu_count() or 1  # oracle threads: every host core

# (H, W, sigma, K, w, seed): small ragged cases spanning several tensor tiles, odd strides
SMALL = [
    (32, 32, 1, 3, -1, 11),
    (24, 40, 2, 4, 0, 12),
    (64, 48, 3, 5, 1, 13),
    (136, 200, 4, 7, -1, 14),
    (96, 128, 8, 1, -1, 15),
    (128, 96, 5, 16, 2, 16),
    (256, 256, 8, 8, -1, 1000),
]


def _img(H, W, seed):
    return synth.pr1_image() if seed == 1000 else synth.fbm_image(seed, H, W)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _params(sigma, K, w, engine="simt"):
    return fic.EncodeParams(domain_stride=sigma, num_classes=K, half_width=w, engine=engine)


def _need_tensor(engine):
    if engine == "tensor":
        major, minor = torch.cuda.get_device_capability()
        if (major, minor) != (10, 3):
            pytest.skip("tensor engine needs sm_103")
        assert fic.engine_available("tensor"), "tensor engine missing on an sm_103 device"


@pytest.mark.parametrize("case", SMALL)
def test_classify_bit_exact(case):
    H, W, sigma, K, w, seed = case
    img = _img(H, W, seed)
    st = fic.classify(_t(img), _params(sigma, K, w))
    torch.cuda.synchronize()
    cls = omatch.classify_image(img, 8, sigma, K)
    g = {k: v.cpu().numpy() for k, v in st.items()}
    assert np.array_equal(g["range_sum"], cls["range_sum"])
    assert np.array_equal(g["range_sumsq"], cls["range_sumsq"])
    assert np.array_equal(g["dom_sum"], cls["dom_sum"])
    assert np.array_equal(g["dom_sumsq"], cls["dom_sumsq"])
    assert np.array_equal(g["range_counts"], cls["range_counts"])
    assert np.array_equal(g["dom_counts"], cls["dom_counts"])
    assert np.array_equal(g["range_fd"].view(np.int64), cls["range_fd"].view(np.int64))
    assert np.array_equal(g["dom_fd"].view(np.int64), cls["dom_fd"].view(np.int64))
    assert g["fd_extent"][0] == cls["F_l"] and g["fd_extent"][1] == cls["F_m"]
    assert np.array_equal(g["range_bin"], cls["range_bin"])
    assert np.array_equal(g["dom_bin"], cls["dom_bin"])


@pytest.mark.parametrize("case", SMALL)
def test_pools_exact(case):
    H, W, sigma, K, w, seed = case
    img = _img(H, W, seed)
    p = _params(sigma, K, w)
    st = fic.classify(_t(img), p)
    po = fic.build_pools(st, H, W, p)
    torch.cuda.synchronize()
    cls = omatch.classify_image(img, 8, sigma, K)
    dom_order = po["dom_order"].cpu().numpy()
    assert np.array_equal(dom_order, np.argsort(cls["dom_bin"], kind="stable"))
    assert np.array_equal(po["range_order"].cpu().numpy(), np.argsort(cls["range_bin"], kind="stable"))
    bo = np.concatenate([[0], np.cumsum(np.bincount(cls["dom_bin"], minlength=K))])
    assert np.array_equal(po["bin_off"].cpu().numpy()[:K + 1], bo)
    ww = odbc.default_half_width(K) if w < 0 else w
    lo, hi = po["win_lo"].cpu().numpy(), po["win_hi"].cpu().numpy()
    for r in range(lo.size):
        pool = opools.class_pool(cls["range_bin"][r], cls["dom_bin"], ww)
        assert np.array_equal(np.sort(dom_order[lo[r]:hi[r]]), pool), r


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


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("case", SMALL)
def test_encode_parity_small(case, engine):
    _need_tensor(engine)
    H, W, sigma, K, w, seed = case
    img = _img(H, W, seed)
    info = fic.new_info("cuda")
    codes = fic.encode(_t(img), _params(sigma, K, w, engine), info=info)
    torch.cuda.synchronize()
    ref = omatch.encode(img, B=8, sigma=sigma, K=K, w=None if w < 0 else w, n_threads=NT)
    _compare_codes(codes, ref)
    rep = fic.read_info(info)
    assert rep["matches"] == int(ref["pool_size"].sum()) * 8
    assert rep["device_error"] == 0
    if engine == "tensor":
        # the ranking must certify nearly every range by itself; a broken contraction would
        # push them all to the exact re-search and still pass the code comparison
        assert rep["fallback_ranges"] <= max(4, codes["dom"].numel() // 20), rep


@pytest.mark.parametrize("engine", ENGINES)
def test_encode_flat_and_edge_images(engine):
    _need_tensor(engine)
    cases = [np.full((48, 64), 200, np.uint8), np.zeros((32, 32), np.uint8)]
    img = synth.fbm_image(77, 96, 96)
    img[8:72, 16:64] = 31  # a large flat rectangle: flat ranges and flat (Q = 0) domains
    cases.append(img)
    chk = ((np.indices((64, 64)).sum(axis=0) % 2) * 255).astype(np.uint8)  # extreme values
    cases.append(chk)
    for im in cases:
        H, W = im.shape
        for K, sigma in ((4, 2), (1, 4), (255, 8)):
            codes = fic.encode(_t(im), _params(sigma, K, -1, engine))
            torch.cuda.synchronize()
            ref = omatch.encode(im, B=8, sigma=sigma, K=K, n_threads=NT)
            _compare_codes(codes, ref)


def test_encode_padded_pitch():
    img = synth.fbm_image(21, 64, 80)
    big = np.zeros((64, 96), np.uint8)
    big[:, :80] = img
    t = _t(big)[:, :80]
    assert t.stride(0) == 96
    codes = fic.encode(t, _params(4, 6, -1))
    torch.cuda.synchronize()
    ref = omatch.encode(img, B=8, sigma=4, K=6, n_threads=NT)
    _compare_codes(codes, ref)


@pytest.mark.parametrize("engine", ENGINES)
def test_encode_deterministic(engine):
    _need_tensor(engine)
    img = _t(synth.fbm_image(3, 256, 192))
    p = _params(4, 16, -1, engine)
    a = fic.encode(img, p)
    b = fic.encode(img, p)
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("block", [8, 16])
def test_encode_schedule_independent(block):
    """The persistent tensor matchers hand out work items from a global counter, so which CTA
    scores which item changes from run to run; items_per_sm and group_chunks change how the chunks
    are cut into items and groups, and pipeline_stages the depth of the operand ring: the codes must
    not change with any of them."""
    _need_tensor("tensor")
    img = _t(synth.fbm_image(41, 1024, 768))
    sigma, K = 4, (16 if block == 8 else 12)
    base, items = None, []
    stages = (3, 4) if block == 8 else (4, 5)
    variants = [(1, 0, 0), (5, 0, 0), (32, 0, 0), (64, 0, 0), (32, 0, 0),
                (24, 4, stages[0]), (24, 128, stages[1]), (8, 1, stages[0])]
    for ipsm, gch, stg in variants:
        p = fic.EncodeParams(domain_stride=sigma, num_classes=K, engine="tensor", block=block,
                             items_per_sm=ipsm, group_chunks=gch, pipeline_stages=stg)
        info = fic.new_info("cuda")
        codes = fic.encode(img, p, info=info)
        torch.cuda.synchronize()
        rep = fic.read_info(info)
        assert rep["device_error"] == 0
        items.append(rep["work_items"])
        if base is None:
            base = codes
            continue
        for k in base:
            assert torch.equal(base[k], codes[k]), (ipsm, gch, stg, k)
    assert items[0] < items[3], items  # the item counts really differ


@pytest.fixture(scope="module")
def oracle_1024():
    """The oracle's codes of every range of the 1024x1024, stride-4, K = 16 workload (about a
    minute on 16 host cores), computed once for both engines."""
    img = synth.image_1024()
    cls = omatch.classify_image(img, 8, 4, 16)
    ref = omatch.encode(img, B=8, sigma=4, K=16, n_threads=NT, cls=cls)
    return img, cls, ref


@pytest.mark.parametrize("engine", ENGINES)
def test_encode_1024_full(engine, oracle_1024):
    """The 1024x1024, stride-4, K=16 workload at full size, in the bench's launch configuration:
    classification bit-exact everywhere and all 16384 codes equal to the oracle's; the ranges the
    tensor engine had to re-search exactly are among them."""
    _need_tensor(engine)
    img, cls, ref = oracle_1024
    p = _params(4, 16, -1, engine)
    H, W = img.shape
    ws = torch.empty(fic.encode_workspace_size(H, W, p), dtype=torch.uint8, device="cuda")
    info = fic.new_info("cuda")
    codes = fic.encode(_t(img), p, workspace=ws, info=info)
    fb = fic.fallback_ranges(H, W, p, ws).cpu().numpy()
    st = fic.classify(_t(img), p)
    torch.cuda.synchronize()
    assert np.array_equal(st["range_bin"].cpu().numpy(), cls["range_bin"])
    assert np.array_equal(st["dom_bin"].cpu().numpy(), cls["dom_bin"])
    _compare_codes(codes, ref)
    rep = fic.read_info(info)
    assert rep["matches"] == int(ref["pool_size"].sum()) * 8
    assert rep["device_error"] == 0
    R = 128 * 128
    assert fb.size == rep["fallback_ranges"]
    if engine == "tensor":
        assert 0 < fb.size <= R // 20, rep
        assert np.unique(fb).size == fb.size and fb.min() >= 0 and fb.max() < R
    else:
        assert fb.size == 0


@pytest.mark.parametrize("engine", ENGINES)
def test_encode_batched_bench_subset(engine):
    """The first eight images of the benchmark's 64-image batch (sides 1536, 512, 768, 2048, 512,
    1024, 384, 2048; stride 8, K = 16) in one fic_encode_batched call: images up to 1024x1024
    compared with the oracle on every range, the larger ones on 400 seeded ranges (corners
    included) each."""
    _need_tensor(engine)
    imgs = synth.batch_images(64)[:8]
    p = _params(8, 16, -1, engine)
    info = fic.new_info("cuda")
    outs = fic.encode_batched([_t(im) for im in imgs], p, info=info)
    torch.cuda.synchronize()
    assert fic.read_info(info)["device_error"] == 0
    for k, (im, out) in enumerate(zip(imgs, outs)):
        H, W = im.shape
        R = (H // 8) * (W // 8)
        if H <= 1024:
            sample = None
        else:
            rng = np.random.default_rng(3100 + k)
            sample = np.unique(np.concatenate([[0, R - 1, W // 8 - 1, R - W // 8],
                                               rng.choice(R, 400, replace=False)]))
        ref = omatch.encode(im, B=8, sigma=8, K=16, range_ids=sample, n_threads=NT)
        _compare_codes(out, ref, sample)


def test_full_search_simt_equals_k1_tensor():
    _need_tensor("tensor")
    img = _t(synth.fbm_image(8, 192, 256))
    a = fic.encode(img, _params(4, 1, -1, "simt"))
    b = fic.encode(img, _params(4, 1, -1, "tensor"))
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("engine", ENGINES)
def test_encode_batched_equals_oracle(engine):
    """Several images of different sizes in one fic_encode_batched call (one tensor-engine launch
    for all of them): each image's codes equal the oracle's for that image alone."""
    _need_tensor(engine)
    shapes = [(64, 48, 31), (136, 200, 32), (96, 128, 33), (32, 32, 34), (256, 256, 35), (48, 64, 36)]
    imgs = [synth.fbm_image(seed, H, W) for H, W, seed in shapes]
    p = _params(4, 7, -1, engine)
    info = fic.new_info("cuda")
    outs = fic.encode_batched([_t(im) for im in imgs], p, info=info)
    torch.cuda.synchronize()
    total = 0
    for im, out in zip(imgs, outs):
        ref = omatch.encode(im, B=8, sigma=4, K=7, n_threads=NT)
        _compare_codes(out, ref)
        total += int(ref["pool_size"].sum()) * 8
    rep = fic.read_info(info)
    assert rep["matches"] == total and rep["device_error"] == 0
    # the same images one at a time give the same codes
    for im, out in zip(imgs, outs):
        single = fic.encode(_t(im), p)
        torch.cuda.synchronize()
        for k in ("dom", "iso", "s", "o", "sse"):
            assert torch.equal(single[k], out[k]), k


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("case", [c for c in SMALL if c[3] > 1])
def test_encode_literal_window(case, engine):
    """Section 3.1 Eq. 3 on FD values: FD_r - D_f <= FD_d <= FD_r + D_f, against the oracle's
    literal mode."""
    _need_tensor(engine)
    H, W, sigma, K, w, seed = case
    img = _img(H, W, seed)
    p = fic.EncodeParams(domain_stride=sigma, num_classes=K, half_width=w, engine=engine, literal=True)
    info = fic.new_info("cuda")
    codes = fic.encode(_t(img), p, info=info)
    st = fic.classify(_t(img), p)
    po = fic.build_pools(st, H, W, p)
    torch.cuda.synchronize()
    ref = omatch.encode(img, B=8, sigma=sigma, K=K, mode="literal", n_threads=NT)
    _compare_codes(codes, ref)
    assert fic.read_info(info)["matches"] == int(ref["pool_size"].sum()) * 8
    cls = ref["cls"]
    Df = opools.fractal_distance(cls["F_l"], cls["F_m"])
    dom_order = po["dom_order"].cpu().numpy()
    fd_sorted = cls["dom_fd"][dom_order]
    assert np.all(np.diff(fd_sorted) >= 0)  # ordered by FD value
    same = np.diff(fd_sorted) == 0
    assert np.all(np.diff(dom_order)[same] > 0)  # stable: equal FDs keep ascending ids
    lo, hi = po["win_lo"].cpu().numpy(), po["win_hi"].cpu().numpy()
    for r in range(lo.size):
        pool = opools.literal_pool(cls["range_fd"][r], cls["dom_fd"], Df)
        assert np.array_equal(np.sort(dom_order[lo[r]:hi[r]]), pool), r


@pytest.mark.parametrize("engine", ENGINES)
def test_conci_two_groups(engine):
    """Conci and Aquino's static classification (Section 2, ref. [8]) split the domains into two
    FD groups and searched the range's own group: K = 2 classes, half-width 0."""
    _need_tensor(engine)
    img = synth.fbm_image(88, 192, 160)
    p = fic.EncodeParams(domain_stride=4, num_classes=2, half_width=0, engine=engine)
    codes = fic.encode(_t(img), p)
    torch.cuda.synchronize()
    ref = omatch.encode(img, B=8, sigma=4, K=2, w=0, n_threads=NT)
    _compare_codes(codes, ref)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("prof", [False, True])
def test_encode_graph_replay(engine, prof):
    """One fic_encode call captured in a CUDA graph (internal streams, and with `prof` the stage
    events as graph nodes) replays to the same codes as a direct call, on a changed image too, and
    the stage times read back after a replay; profiling switched off and on again between capture
    and replay keeps the captured events valid."""
    _need_tensor(engine)
    a_np, b_np = synth.fbm_image(21, 200, 136), synth.fbm_image(22, 200, 136)
    img = _t(a_np)
    p = _params(4, 8, -1, engine)
    R, _ = fic.counts(200, 136, p)
    ws = torch.empty(fic.encode_workspace_size(200, 136, p), dtype=torch.uint8, device="cuda")
    out = fic.alloc_codes(R, img.device)
    fic.profile_enable(prof)
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fic.encode(img, p, out=out, workspace=ws)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            fic.encode(img, p, out=out, workspace=ws)
        fic.profile_enable(False)
        fic.profile_enable(prof)
        for src in (a_np, b_np):
            img.copy_(_t(src))
            for k in out:
                out[k].zero_()
            graph.replay()
            torch.cuda.synchronize()
            if prof:
                stages, _ = fic.profile_read()
                assert set(stages) == set(fic.STAGES) and all(v >= 0 for v in stages.values())
            ref = fic.encode(_t(src), p)
            torch.cuda.synchronize()
            for k in out:
                assert torch.equal(out[k], ref[k]), k
    finally:
        fic.profile_enable(False)


@pytest.mark.parametrize("engine", ENGINES)
def test_encode_repeated_calls_replay(engine):
    """Repeated fic_encode calls with the same arguments replay the library's cached graph of the
    call: codes follow the image content, different parameters on the same buffers give their own
    codes, and both equal the direct path (profiling on bypasses the cache)."""
    _need_tensor(engine)
    H, W = 152, 200
    img = torch.empty(H, W, dtype=torch.uint8, device="cuda")
    params = [_params(4, 8, -1, engine), _params(4, 5, 1, engine)]
    R, _ = fic.counts(H, W, params[0])
    ws = torch.empty(max(fic.encode_workspace_size(H, W, q) for q in params), dtype=torch.uint8, device="cuda")
    out = fic.alloc_codes(R, img.device)
    for rep in range(3):
        for q in params:
            src = synth.fbm_image(30 + rep, H, W)
            img.copy_(_t(src))
            fic.encode(img, q, out=out, workspace=ws)
            torch.cuda.synchronize()
            got = {k: v.clone() for k, v in out.items()}
            fic.profile_enable(True)
            try:
                ref = fic.encode(_t(src), q)
                torch.cuda.synchronize()
            finally:
                fic.profile_enable(False)
            for k in got:
                assert torch.equal(got[k], ref[k]), (rep, k)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("block,shape,sigma", [
    (8, (16, 16), 1),    # the smallest image: 4 ranges, one domain
    (8, (16, 48), 3),    # one domain row
    (8, (40, 16), 8),    # one domain column
    (16, (32, 32), 4),   # 16x16 ranges: 4 ranges, one domain
    (16, (32, 96), 16),  # one domain row, stride 16
])
def test_encode_smallest_images(engine, block, shape, sigma):
    """The degenerate geometries: a single domain, one row or one column of domains; every range's
    pool is then that set, so the codes are the exact full search (oracle parity), for K = 1 and
    for K > 1 (one class holds everything)."""
    _need_tensor(engine)
    H, W = shape
    img = synth.fbm_image(97 + H + W, H, W)
    for K in (1, 6):
        p = fic.EncodeParams(domain_stride=sigma, num_classes=K, engine=engine, block=block)
        info = fic.new_info("cuda")
        codes = fic.encode(_t(img), p, info=info)
        torch.cuda.synchronize()
        ref = omatch.encode(img, B=block, sigma=sigma, K=K, n_threads=NT)
        _compare_codes(codes, ref)
        rep = fic.read_info(info)
        assert rep["matches"] == int(ref["pool_size"].sum()) * 8 and rep["device_error"] == 0
