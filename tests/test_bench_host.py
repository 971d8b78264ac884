"""Host logic of bench.py (no GPU): the DRAM traffic a roofline line reports comes from a capture
summary under profiles/ only while the kernel's sources hash to the value the summary records."""
import bench


def test_traffic_follows_the_recorded_source_hash(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    cur = bench.source_hash("k_match_tc")
    (tmp_path / "a.md").write_text(
        "# a capture\n\n"
        f"traffic: k_match_tc encode-1024 dram_bytes_per_launch=123456 source={cur}\n"
        "traffic: k_match_tc encode-4096 dram_bytes_per_launch=999 source=0000000000000000\n")
    assert bench.measured_traffic("k_match_tc", "encode-1024") == 123456.0
    assert bench.measured_traffic("k_match_tc", "encode-4096") is None  # sources changed since
    assert bench.measured_traffic("k_match_tc", "encode-2048-s4") is None  # never captured
    assert bench.measured_traffic("k_match_tc16", "encode-1024") is None  # another kernel


def test_source_hash_covers_each_kernels_files():
    for kernel, files in bench.KERNEL_SOURCES.items():
        h = bench.source_hash(kernel)
        assert len(h) == 16 and int(h, 16) >= 0
        assert files  # every reported kernel names the sources its capture depends on


def test_decode_figures():
    H = W = 4096
    R = (H // 8) * (W // 8)
    f = bench.decode_figures(H, W, R, 8, 0.1, 6780.0)
    assert f["decode_dram_bytes"] == 4 * H * W + 24 * R
    assert f["decode_full_res_bytes"] == 8 * H * W * 8
    assert abs(f["decode_full_res_roofline_ms"] - 8 * H * W * 8 / 6780e9 * 1e3) < 1e-12
    assert abs(f["decode_speedup_over_full_res_roofline"] - f["decode_full_res_roofline_ms"] / 0.1) < 1e-12
