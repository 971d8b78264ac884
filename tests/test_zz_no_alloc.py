"""fic_decode_static, the decode entry point that allocates nothing, against fic_decode.

Callers that cannot call cudaMalloc (applications that reserve all device memory up front and
give libraries only the buffers they need, or latency-critical loops where an allocation could
block on or synchronise the device) cannot hand fic_decode its workspace. fic_decode_static
keeps that scratch image in a fixed array inside the library instead. These tests call it through
the C ABI twice in a row and compare each result with fic_decode given a workspace, at the decode
tolerance the other GPU tests use (2e-3 absolute), and check that an image larger than the fixed
scratch is refused.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1206_4880_gb300 import fic, synth

pytestmark = pytest.mark.gpu


def _call_static(codes, H, W, p, iters, x0, out):
    lib = fic.load()
    cs = fic.Codes(*(ctypes.c_void_p(codes[k].data_ptr()) for k in ("dom", "iso", "s", "o", "sse")))
    g = fic.geom(H, W)
    pc = p.c()
    x0p = ctypes.c_void_p(0) if x0 is None else ctypes.c_void_p(x0.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.fic_decode_static(ctypes.byref(cs), ctypes.byref(g), ctypes.byref(pc), iters, x0p,
                                 ctypes.c_void_p(out.data_ptr()), stream)


@pytest.fixture(scope="module", params=[8, 16])
def coded(request):
    """Codes of a 256 x 320 image for 8x8 or 16x16 ranges, and a random start image."""
    B = request.param
    H, W = 256, 320
    img = synth.fbm_image(321, H, W)
    p = fic.EncodeParams(domain_stride=8, num_classes=8, engine="simt", block=B)
    codes = fic.encode(torch.from_numpy(img).cuda(), p)
    x0 = torch.from_numpy(np.random.default_rng(5).uniform(0, 255, (H, W)).astype(np.float32)).cuda()
    return H, W, p, codes, x0


@pytest.mark.parametrize("iters", [0, 1, 2, 8])
@pytest.mark.parametrize("with_x0", [False, True])
def test_decode_static_matches_decode_on_two_calls(coded, iters, with_x0):
    """Two calls in a row (the second sees the scratch the first left behind) each equal
    fic_decode: iters = 0 copies or fills the start image, iters = 1 writes the output directly,
    even and odd counts end the ping-pong in the output buffer."""
    H, W, p, codes, x0 = coded
    start = x0 if with_x0 else None
    ref = fic.decode(codes, H, W, p, iters, x0=start)
    for _ in range(2):
        out = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        st = _call_static(codes, H, W, p, iters, start, out)
        assert st == fic.FIC_OK, fic.load().fic_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert torch.max(torch.abs(out - ref)).item() <= 2e-3
    if iters == 0:
        assert torch.equal(out, x0 if with_x0 else torch.full_like(out, 128.0))


def test_decode_static_refuses_images_beyond_its_scratch():
    H = W = 2048  # 4 Mi pixels > the 1 Mi-pixel fixed scratch
    p = fic.EncodeParams(domain_stride=8, num_classes=8, engine="simt")
    R, _ = fic.counts(H, W, p)
    codes = {"dom": torch.zeros(R, dtype=torch.int32, device="cuda"),
             "iso": torch.zeros(R, dtype=torch.int32, device="cuda"),
             "s": torch.zeros(R, dtype=torch.float64, device="cuda"),
             "o": torch.zeros(R, dtype=torch.float64, device="cuda"),
             "sse": torch.zeros(R, dtype=torch.float64, device="cuda")}
    out = torch.empty(H, W, dtype=torch.float32, device="cuda")
    st = _call_static(codes, H, W, p, 2, None, out)
    assert st == fic.FIC_ERR_INVALID_ARG
    assert b"fixed scratch" in fic.load().fic_last_error()
