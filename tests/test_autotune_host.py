"""Host logic of the autotuner (no GPU): the candidate grid, the workload signature and the
timing cache."""
import json

from paper_1206_4880_gb300 import autotune, fic


def test_candidate_grid():
    for block in (8, 16):
        c = autotune.candidates(block)
        n = len(autotune.STAGES[block]) * len(autotune.GROUP_CHUNKS[block]) * len(autotune.ITEMS_PER_SM[block])
        assert len(c) == n
        labels = [autotune.label(x) for x in c]
        assert len(set(labels)) == n  # every combination once, with its own label
        for x in c:
            assert x["pipeline_stages"] in autotune.STAGES[block]
            assert x["group_chunks"] in autotune.GROUP_CHUNKS[block]
            assert x["items_per_sm"] in autotune.ITEMS_PER_SM[block]


def test_signature_depends_on_the_workload_not_on_the_image_order():
    p = fic.EncodeParams(domain_stride=8, num_classes=16)
    a = autotune.signature([(256, 256), (512, 384)], p)
    assert a == autotune.signature([(512, 384), (256, 256)], p)
    assert a != autotune.signature([(256, 256), (512, 512)], p)
    assert a != autotune.signature([(256, 256), (512, 384)], fic.EncodeParams(domain_stride=4, num_classes=16))
    assert a != autotune.signature([(256, 256), (512, 384)], fic.EncodeParams(domain_stride=8, num_classes=8))


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "autotune.json"
    monkeypatch.setenv("FIC_AUTOTUNE_CACHE", str(path))
    assert autotune._load_cache() == {}
    best = {"pipeline_stages": 3, "group_chunks": 64, "items_per_sm": 24}
    autotune._store("gpu|sig1", {"best": best, "ms": {"s3_g64_i24": 1.0}, "noise_ms": 0.1})
    autotune._store("gpu|sig2", {"best": best, "ms": {}, "noise_ms": 0.0})
    cache = autotune._load_cache()
    assert set(cache) == {"gpu|sig1", "gpu|sig2"} and cache["gpu|sig1"]["best"] == best
    assert json.loads(path.read_text()) == cache
    path.write_text("not json")  # a damaged cache reads as empty and is rewritten whole
    assert autotune._load_cache() == {}
    autotune._store("gpu|sig3", {"best": best, "ms": {}, "noise_ms": 0.0})
    assert set(autotune._load_cache()) == {"gpu|sig3"}
