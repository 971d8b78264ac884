"""The 4096x4096 workload at full size (stride-8 domains, K = 32, w = 10) in both range sizes, in
the launch configuration the benchmark times: classification bit-exact on every block, codes
equal to the oracle's on 1000 seeded ranges plus every range the tensor engine re-searched exactly
(each over its full pool), the match count equal to the oracle's pool sizes, and the ranking
certifying nearly every range by itself."""
import os

import numpy as np
import pytest
import torch

from oracle import dbc as odbc
from oracle import match as omatch
from oracle import pools as opools
from paper_1206_4880_gb300 import fic, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def img4096():
    return synth.large_image()


@pytest.mark.parametrize("B", [8, 16])
def test_encode_4096_sampled(img4096, B):
    major, minor = torch.cuda.get_device_capability()
    engine = "tensor" if (major, minor) == (10, 3) else "simt"
    img = img4096
    p = fic.EncodeParams(domain_stride=8, num_classes=32, half_width=-1, engine=engine, block=B)
    t = torch.from_numpy(img).cuda()
    ws = torch.empty(fic.encode_workspace_size(4096, 4096, p), dtype=torch.uint8, device="cuda")
    info = fic.new_info("cuda")
    codes = fic.encode(t, p, workspace=ws, info=info)
    fb = fic.fallback_ranges(4096, 4096, p, ws).cpu().numpy()
    st = fic.classify(t, p)
    torch.cuda.synchronize()
    cls = omatch.classify_image(img, B, 8, 32)
    for k in ("range_bin", "dom_bin", "range_counts", "dom_counts"):
        assert np.array_equal(st[k].cpu().numpy(), cls[k]), k
    assert np.array_equal(st["dom_fd"].cpu().numpy().view(np.int64), cls["dom_fd"].view(np.int64))
    R = (4096 // B) ** 2
    rng = np.random.default_rng(5000 + B)
    sample = np.unique(np.concatenate([[0, R - 1], rng.choice(R, 1000, replace=False), fb]))
    ref = omatch.encode(img, B=B, sigma=8, K=32, range_ids=sample, n_threads=os.cpu_count() or 1, cls=cls)
    g = {k: v.cpu().numpy()[sample] for k, v in codes.items()}
    assert np.array_equal(g["dom"], ref["dom"]) and np.array_equal(g["iso"], ref["iso"])
    assert np.max(np.abs(g["s"] - ref["s"])) <= 1e-6
    assert np.max(np.abs(g["o"] - ref["o"])) <= 1e-6
    assert np.all(np.abs(g["sse"] - ref["sse"]) <= 1e-9 * np.maximum(1.0, ref["sse"]))
    rep = fic.read_info(info)
    ww = odbc.default_half_width(32)
    bins, counts = np.unique(cls["range_bin"], return_counts=True)
    total = sum(int(c) * opools.class_pool(b, cls["dom_bin"], ww).size for b, c in zip(bins, counts))
    assert rep["matches"] == total * 8
    assert rep["device_error"] == 0
    assert fb.size == rep["fallback_ranges"]
    if engine == "tensor":
        assert rep["fallback_ranges"] <= R // 20, rep
