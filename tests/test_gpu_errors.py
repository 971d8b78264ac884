"""The device-side error contract of the encoder, through the C ABI.

Every wait of the tensor matchers on another role of their CTA is bounded. The library's testing
hook (fic_debug_stall_matcher) makes each matcher CTA wait, before it issues any copy or MMA, on a
barrier that nothing completes, so the bounded wait runs out with no work in flight. The encode
must then report FIC_ERR_DEVICE_TIMEOUT in its info record and through fic_check, write every code
as invalid (dom = iso = -1, s = o = sse = NaN) instead of leaving stale values, and leave the CUDA
context usable: the next encode is correct and fic_check is clear again.
"""
import numpy as np
import pytest
import torch

from oracle import match as omatch
from paper_1206_4880_gb300 import fic, synth

pytestmark = pytest.mark.gpu


def _need_tensor():
    if torch.cuda.get_device_capability() != (10, 3):
        pytest.skip("tensor engine needs sm_103")


@pytest.mark.parametrize("block", [8, 16])
@pytest.mark.parametrize("batched", [False, True])
def test_matcher_timeout_is_reported_and_recovers(block, batched):
    _need_tensor()
    H, W = 96, 128
    img = synth.fbm_image(91, H, W)
    t = torch.from_numpy(img).cuda()
    p = fic.EncodeParams(domain_stride=4, num_classes=4, engine="tensor", block=block)
    fic.check()  # nothing pending from earlier tests
    info = fic.new_info("cuda")
    R, _ = fic.counts(H, W, p)
    out = fic.alloc_codes(R, t.device)
    for k in out:
        out[k].zero_()  # stale values that look like a valid code
    fic.debug_stall_matcher(10_000_000)  # 10 ms
    try:
        if batched:
            fic.encode_batched([t, t], p, outs=[out, fic.alloc_codes(R, t.device)], info=info)
        else:
            fic.encode(t, p, out=out, info=info)
    finally:
        fic.debug_stall_matcher(0)
    torch.cuda.synchronize()
    assert fic.read_info(info)["device_error"] == fic.FIC_ERR_DEVICE_TIMEOUT
    with pytest.raises(fic.FicError) as e:
        fic.check()
    assert e.value.status == fic.FIC_ERR_DEVICE_TIMEOUT
    assert bool((out["dom"] == -1).all()) and bool((out["iso"] == -1).all())
    for k in ("s", "o", "sse"):
        assert bool(torch.isnan(out[k]).all()), k
    fic.check()  # cleared by the previous check
    # the context is still usable: the same call without the hook gives the oracle's codes
    info2 = fic.new_info("cuda")
    codes = fic.encode(t, p, out=out, info=info2)
    fic.check()
    assert fic.read_info(info2)["device_error"] == 0
    ref = omatch.encode(img, B=block, sigma=4, K=4)
    assert np.array_equal(codes["dom"].cpu().numpy(), ref["dom"])
    assert np.array_equal(codes["iso"].cpu().numpy(), ref["iso"])

