"""GPU parity of decoding and of its adjoint against the FP64 CPU oracle, through the C ABI.

Bars: decoded PSNR within 0.01 dB of the oracle's; iterates within 2e-3 absolute (FP32 against
FP64 over <= 8 contractive steps of values in [0, 255]); gradients within 1e-4 relative of the
oracle's FP64 adjoint and of FP64 central finite differences (h = 1e-4).
"""
import os

import numpy as np
import pytest
import torch

from oracle import decode as odec
from oracle import match as omatch
from paper_1206_4880_gb300 import fic, synth

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1  # oracle threads: every host core


def _codes_gpu(c):
    return {"dom": torch.from_numpy(np.asarray(c["dom"], np.int32)).cuda(),
            "iso": torch.from_numpy(np.asarray(c["iso"], np.int32)).cuda(),
            "s": torch.from_numpy(np.asarray(c["s"], np.float64)).cuda(),
            "o": torch.from_numpy(np.asarray(c["o"], np.float64)).cuda()}


@pytest.fixture(scope="module")
def pr1_codes():
    img = synth.pr1_image()
    return img, omatch.encode(img, B=8, sigma=8, K=8, n_threads=NT)


@pytest.mark.parametrize("iters", [0, 1, 2, 5, 8])
def test_decode_parity(pr1_codes, iters):
    img, codes = pr1_codes
    p = fic.EncodeParams(domain_stride=8, num_classes=8)
    x = fic.decode(_codes_gpu(codes), 256, 256, p, iters)
    torch.cuda.synchronize()
    ref = odec.decode(codes, 256, 256, 8, 8, iters)
    assert np.max(np.abs(x.cpu().numpy() - ref)) <= 2e-3
    if iters >= 5:
        pg = odec.psnr(odec.to_u8(x.cpu().numpy().astype(np.float64)), img)
        po = odec.psnr(odec.to_u8(ref), img)
        assert abs(pg - po) <= 0.01


def test_quality_matches_oracle_psnr(pr1_codes):
    img, codes = pr1_codes
    p = fic.EncodeParams(domain_stride=8, num_classes=8)
    x = fic.decode(_codes_gpu(codes), 256, 256, p, 8)
    mse, psnr = fic.quality(x, torch.from_numpy(img).cuda())
    xq = odec.to_u8(x.cpu().numpy().astype(np.float64))
    assert abs(psnr - odec.psnr(xq, img)) <= 1e-9
    assert abs(mse - np.mean((xq.astype(np.float64) - img) ** 2)) <= 1e-9
    m0, p0 = fic.quality(torch.from_numpy(img.astype(np.float32)).cuda(), torch.from_numpy(img).cuda())
    assert m0 == 0.0 and p0 == float("inf")


def test_decode_from_given_start(pr1_codes):
    img, codes = pr1_codes
    p = fic.EncodeParams(domain_stride=8, num_classes=8)
    x0 = np.random.default_rng(0).uniform(0, 255, (256, 256)).astype(np.float32)
    for iters in (1, 4):
        x = fic.decode(_codes_gpu(codes), 256, 256, p, iters, x0=torch.from_numpy(x0).cuda())
        torch.cuda.synchronize()
        ref = odec.decode(codes, 256, 256, 8, 8, iters, x0=x0.astype(np.float64))
        assert np.max(np.abs(x.cpu().numpy() - ref)) <= 2e-3


@pytest.mark.parametrize("sigma", [8, 4, 6, 3, 2, 1])
def test_adjoint_parity(sigma):
    H, W, iters = 64, 96, 6
    img = synth.fbm_image(90 + sigma, H, W)
    codes = omatch.encode(img, B=8, sigma=sigma, K=6, n_threads=NT)
    g = np.random.default_rng(sigma).normal(size=(H, W))
    gs_ref, go_ref = odec.decode_adjoint(codes, H, W, 8, sigma, iters, g)
    p = fic.EncodeParams(domain_stride=sigma, num_classes=6)
    outs = []
    for ck in (1, 2, 4, 6):
        gs, go = fic.decode_backward(_codes_gpu(codes), H, W, p, iters, ck,
                                     torch.from_numpy(g.astype(np.float32)).cuda())
        torch.cuda.synchronize()
        outs.append((gs.cpu().numpy(), go.cpu().numpy()))
    for gs, go in outs:
        assert np.array_equal(gs, outs[0][0]) and np.array_equal(go, outs[0][1])
    # deterministic: the same call again gives the same bits
    gs2, go2 = fic.decode_backward(_codes_gpu(codes), H, W, p, iters, 2,
                                   torch.from_numpy(g.astype(np.float32)).cuda())
    assert np.array_equal(gs2.cpu().numpy(), outs[0][0]) and np.array_equal(go2.cpu().numpy(), outs[0][1])
    gs, go = outs[0]
    for a, b in ((gs, gs_ref), (go, go_ref)):
        scale = np.max(np.abs(b))
        assert np.max(np.abs(a - b)) <= 1e-4 * scale


def test_adjoint_512_against_finite_differences():
    """The 512x512 differentiation workload: 8 iterations from mid-grey, checkpoints every 2."""
    img = synth.diff_image()
    H = W = 512
    iters = 8
    codes = omatch.encode(img, B=8, sigma=8, K=16, n_threads=NT)
    cg = _codes_gpu(codes)
    p = fic.EncodeParams(domain_stride=8, num_classes=16)
    base = {k: np.asarray(codes[k], np.float64 if k in ("s", "o") else np.int64)
            for k in ("dom", "iso", "s", "o")}
    I = img.astype(np.float64)
    # L = 0.5 * ||x_K - I||^2 ; dL/dx_K = x_K - I, with x_K the FP64 iterate the finite
    # differences below differentiate
    grad_out = torch.from_numpy((odec.decode(base, H, W, 8, 8, iters) - I).astype(np.float32)).cuda()
    gs, go = fic.decode_backward(cg, H, W, p, iters, 2, grad_out)
    torch.cuda.synchronize()
    gs, go = gs.cpu().numpy(), go.cpu().numpy()
    h = 1e-4

    def loss(c):
        x = odec.decode(c, H, W, 8, 8, iters)
        return 0.5 * np.sum((x - I) ** 2)

    rng = np.random.default_rng(4000)
    for r in rng.choice(gs.size, 3, replace=False):
        for key, grad in (("s", gs), ("o", go)):
            cp = {k: v.copy() for k, v in base.items()}
            cm = {k: v.copy() for k, v in base.items()}
            cp[key][r] += h
            cm[key][r] -= h
            fd = (loss(cp) - loss(cm)) / (2 * h)
            assert abs(grad[r] - fd) <= 1e-4 * max(abs(fd), 1.0), (key, r, grad[r], fd)


def test_autograd_function(pr1_codes):
    img, codes = pr1_codes
    cg = _codes_gpu(codes)
    p = fic.EncodeParams(domain_stride=8, num_classes=8)
    s = cg["s"].clone().requires_grad_(True)
    o = cg["o"].clone().requires_grad_(True)
    x = fic.Decode.apply(s, o, cg["dom"], cg["iso"], 256, 256, p, 4, 2)
    target = torch.from_numpy(img.astype(np.float32)).cuda()
    loss = 0.5 * torch.sum((x - target) ** 2)
    loss.backward()
    gs, go = fic.decode_backward(cg, 256, 256, p, 4, 2, (x - target).detach())
    torch.cuda.synchronize()
    assert torch.allclose(s.grad.float(), gs) and torch.allclose(o.grad.float(), go)


@pytest.mark.parametrize("scale", [1, 2, 3])
def test_decode_scaled(pr1_codes, scale):
    """Resolution-independent decode against the oracle, and 2x2 block averages of the 2x decode
    against the 1x decode."""
    img, codes = pr1_codes
    p = fic.EncodeParams(domain_stride=8, num_classes=8)
    cg = _codes_gpu(codes)
    x = fic.decode_scaled(cg, 256, 256, p, scale, 6)
    torch.cuda.synchronize()
    ref = odec.decode_scaled(codes, 256, 256, 8, 8, 6, scale)
    assert np.max(np.abs(x.cpu().numpy() - ref)) <= 2e-3
    if scale == 2:
        x1 = fic.decode(cg, 256, 256, p, 6).cpu().numpy()
        down = x.cpu().numpy().astype(np.float64).reshape(256, 2, 256, 2).mean(axis=(1, 3))
        assert np.max(np.abs(down - x1)) <= 2e-3


def test_quantize_bit_exact_against_oracle(pr1_codes):
    from oracle import quantize as oq
    img, codes = pr1_codes
    rng = np.random.default_rng(9)
    cases = [codes, {"dom": codes["dom"], "iso": codes["iso"], "s": rng.uniform(-1, 1, 1024),
                     "o": rng.uniform(-50, 300, 1024)}]
    for c in cases:
        for bs, bo in ((5, 7), (4, 6), (16, 16)):
            out, qs, qo, (lo, hi) = fic.quantize(_codes_gpu(c), bs, bo)
            torch.cuda.synchronize()
            rqs, rqo, rs, ro, rlo, rhi = oq.quantize(c["s"], c["o"], bs, bo)
            assert lo == rlo and hi == rhi
            assert np.array_equal(qs.cpu().numpy().view(np.uint16), rqs.astype(np.uint16))
            assert np.array_equal(qo.cpu().numpy().view(np.uint16), rqo.astype(np.uint16))
            assert np.array_equal(out["s"].cpu().numpy(), rs) and np.array_equal(out["o"].cpu().numpy(), ro)
            assert np.array_equal(out["dom"].cpu().numpy(), np.asarray(c["dom"], np.int32))


def test_refinement_improves_decoded_psnr(pr1_codes):
    from paper_1206_4880_gb300 import refine
    img, codes = pr1_codes
    p = fic.EncodeParams(domain_stride=8, num_classes=8)
    cg = _codes_gpu(codes)
    rep = refine.refine_and_quantize(cg, torch.from_numpy(img).cuda(), p, steps=15)
    assert rep["psnr_refined"] > rep["psnr_encoded"] + 0.05, rep
    assert rep["psnr_refined_quantized"] > rep["psnr_quantized"], rep
    r = refine.refine(cg, torch.from_numpy(img).cuda(), p, steps=3)
    assert float(r["s"].abs().max()) <= 1.0


def test_decode_repeated_calls_follow_contents(pr1_codes):
    """fic_decode replays a cached graph for repeated calls with the same buffers: the result
    must follow what the code and start buffers hold at each call."""
    img, codes_a = pr1_codes
    codes_b = omatch.encode(synth.fbm_image(44, 256, 256), B=8, sigma=8, K=8, n_threads=NT)
    p = fic.EncodeParams(domain_stride=8, num_classes=8)
    g = _codes_gpu(codes_a)
    out = torch.empty(256, 256, dtype=torch.float32, device="cuda")
    ws = torch.empty(fic.decode_workspace_size(256, 256, p, 6), dtype=torch.uint8, device="cuda")
    x0 = torch.full((256, 256), 128.0, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(9)
    for rep in range(3):
        for codes in (codes_a, codes_b):
            for k, v in _codes_gpu(codes).items():
                g[k].copy_(v)
            start = rng.uniform(0, 255, (256, 256))
            x0.copy_(torch.from_numpy(start.astype(np.float32)))
            fic.decode(g, 256, 256, p, 6, x0=x0, out=out, workspace=ws)
            torch.cuda.synchronize()
            ref = odec.decode(codes, 256, 256, 8, 8, 6, x0=start.astype(np.float32).astype(np.float64))
            assert np.max(np.abs(out.cpu().numpy() - ref)) <= 2e-3, rep


@pytest.mark.parametrize("block,sigma", [(8, 8), (8, 3), (16, 4)])
def test_adjoint_from_given_start(block, sigma):
    """The adjoint of decoding from a given start image (its 2x2 averages form the first plane when
    the stride is even) equals the FP64 oracle's."""
    H, W, iters = 64, 96, 4
    codes = omatch.encode(synth.fbm_image(80 + sigma, H, W), B=block, sigma=sigma, K=4, n_threads=NT)
    p = fic.EncodeParams(domain_stride=sigma, num_classes=4, block=block)
    rng = np.random.default_rng(21)
    start = rng.uniform(0, 255, (H, W)).astype(np.float32)
    up = rng.normal(size=(H, W))
    gs, go = fic.decode_backward(_codes_gpu(codes), H, W, p, iters, 2,
                                 torch.from_numpy(up.astype(np.float32)).cuda(),
                                 x0=torch.from_numpy(start).cuda())
    torch.cuda.synchronize()
    gs_ref, go_ref = odec.decode_adjoint(codes, H, W, block, sigma, iters, up.astype(np.float32).astype(np.float64),
                                         x0=start.astype(np.float64))
    for a, b in ((gs.cpu().numpy(), gs_ref), (go.cpu().numpy(), go_ref)):
        assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(b))


@pytest.mark.parametrize("sigma", [8, 3])
def test_backward_repeated_calls_follow_contents(pr1_codes, sigma):
    """fic_decode_backward replays a cached graph for repeated calls with the same buffers: the
    gradients must follow what the code and gradient buffers hold at each call."""
    H, W, iters, ck = 64, 96, 5, 2
    codes = [omatch.encode(synth.fbm_image(60 + k, H, W), B=8, sigma=sigma, K=4, n_threads=NT) for k in (0, 1)]
    p = fic.EncodeParams(domain_stride=sigma, num_classes=4)
    g = _codes_gpu(codes[0])
    R = g["dom"].numel()
    gout = torch.empty(H, W, dtype=torch.float32, device="cuda")
    gs = torch.empty(R, dtype=torch.float32, device="cuda")
    go = torch.empty_like(gs)
    ws = torch.empty(fic.decode_workspace_size(H, W, p, iters, ck), dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(13)
    for rep in range(2):
        for c in codes:
            for k, v in _codes_gpu(c).items():
                g[k].copy_(v)
            up = rng.normal(size=(H, W))
            gout.copy_(torch.from_numpy(up.astype(np.float32)))
            fic.decode_backward(g, H, W, p, iters, ck, gout, workspace=ws, grad_s=gs, grad_o=go)
            torch.cuda.synchronize()
            gs_ref, go_ref = odec.decode_adjoint(c, H, W, 8, sigma, iters, up.astype(np.float32).astype(np.float64))
            for a, b in ((gs.cpu().numpy(), gs_ref), (go.cpu().numpy(), go_ref)):
                assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(b)), rep


@pytest.mark.parametrize("block,sigma", [(8, 3), (8, 5), (16, 3), (16, 8), (8, 6), (8, 2)])
def test_decode_odd_strides_and_unaligned_start(block, sigma):
    """Odd strides, and a start image and an output that are only 4-byte aligned, take the kernels'
    scalar-load and scalar-store forms (odd strides: full-resolution steps; even strides: the plane
    of 2x2 averages, with single loads when sigma / 2 is odd); results equal the oracle's."""
    H, W = 96, 128
    img = synth.fbm_image(45 + sigma, H, W)
    codes = omatch.encode(img, B=block, sigma=sigma, K=4, n_threads=NT)
    p = fic.EncodeParams(domain_stride=sigma, num_classes=4, block=block)
    start = np.random.default_rng(sigma).uniform(0, 255, (H, W)).astype(np.float32)
    big = torch.empty(H * W + 1, dtype=torch.float32, device="cuda")
    x0 = big[1:].view(H, W)
    x0.copy_(torch.from_numpy(start))
    assert x0.data_ptr() % 8 == 4
    big_out = torch.empty(H * W + 1, dtype=torch.float32, device="cuda")
    for iters in (1, 4):
        for out in (None, big_out[1:].view(H, W)):
            x = fic.decode(_codes_gpu(codes), H, W, p, iters, x0=x0, out=out)
            torch.cuda.synchronize()
            ref = odec.decode(codes, H, W, block, sigma, iters, x0=start.astype(np.float64))
            assert np.max(np.abs(x.cpu().numpy() - ref)) <= 2e-3, iters


def test_decode_invalid_codes_give_nan_only_there(pr1_codes):
    """A code whose domain or isometry is out of range (as written by an encode whose matcher gave
    up) decodes to NaN over its own range and is never used to index the image."""
    img, codes = pr1_codes
    p = fic.EncodeParams(domain_stride=8, num_classes=8)
    g = _codes_gpu(codes)
    bad = [0, 77, 1023]
    g["dom"][bad[0]] = -1
    g["dom"][bad[1]] = 10 ** 6
    g["iso"][bad[2]] = 9
    x = fic.decode(g, 256, 256, p, 1).cpu().numpy()
    ref = odec.decode(codes, 256, 256, 8, 8, 1)
    mask = np.zeros((256, 256), bool)
    for r in bad:
        ry, rx = divmod(r, 32)
        mask[8 * ry:8 * ry + 8, 8 * rx:8 * rx + 8] = True
    assert np.all(np.isnan(x[mask]))
    assert np.max(np.abs(x[~mask] - ref[~mask])) <= 2e-3


@pytest.mark.parametrize("block", [8, 16])
def test_decode_load_and_store_forms_agree_bitwise(block):
    """The decode step's 16-byte, pair and single-float load forms and its vector and scalar store
    forms apply the same operations in the same order: one step from the same start image gives the
    same bits whichever form the alignment of the buffers selects."""
    H, W, sigma = 128, 160, 8
    img = synth.fbm_image(46, H, W)
    codes = _codes_gpu(omatch.encode(img, B=block, sigma=sigma, K=4, n_threads=NT))
    p = fic.EncodeParams(domain_stride=sigma, num_classes=4, block=block)
    start = torch.from_numpy(np.random.default_rng(3).uniform(0, 255, (H, W)).astype(np.float32)).cuda()
    outs = []
    for shift_in, shift_out in ((0, 0), (1, 0), (2, 1), (0, 3)):
        bi = torch.empty(H * W + 4, dtype=torch.float32, device="cuda")
        bo = torch.empty(H * W + 4, dtype=torch.float32, device="cuda")
        x0 = bi[shift_in:shift_in + H * W].view(H, W)
        x0.copy_(start)
        out = bo[shift_out:shift_out + H * W].view(H, W)
        fic.decode(codes, H, W, p, 1, x0=x0, out=out)
        torch.cuda.synchronize()
        outs.append(out.clone())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_adjoint_many_ranges_on_one_domain():
    """Ranges that share a domain are summed per domain in increasing range id: an image whose
    ranges mostly pick the same few domains (a smooth ramp with one textured patch) gives the
    oracle's gradients and the same bits on every call."""
    H, W, sigma, iters = 96, 128, 4, 4
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.clip(60 + yy + xx // 2, 0, 255).astype(np.uint8)
    img[32:64, 40:80] = synth.fbm_image(47, 32, 40)
    codes = omatch.encode(img, B=8, sigma=sigma, K=1, n_threads=NT)
    doms, counts = np.unique(codes["dom"][np.asarray(codes["s"]) != 0], return_counts=True)
    assert counts.max() >= 8, counts.max()  # some domain serves many ranges
    g = np.random.default_rng(11).normal(size=(H, W))
    gs_ref, go_ref = odec.decode_adjoint(codes, H, W, 8, sigma, iters, g)
    p = fic.EncodeParams(domain_stride=sigma, num_classes=1)
    res = []
    for _ in range(2):
        gs, go = fic.decode_backward(_codes_gpu(codes), H, W, p, iters, 2,
                                     torch.from_numpy(g.astype(np.float32)).cuda())
        torch.cuda.synchronize()
        res.append((gs.cpu().numpy(), go.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    for a, b in ((res[0][0], gs_ref), (res[0][1], go_ref)):
        assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(b))
