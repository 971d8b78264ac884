"""The C ABI library builds, loads without a GPU, exports every entry point include/fic.h
declares, and rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

from oracle import dbc
from paper_1206_4880_gb300 import fic

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fic.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fic_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = fic.load()
    names = _declared()
    assert {"fic_classify", "fic_build_pools", "fic_encode", "fic_decode",
            "fic_decode_backward"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fic.SIGNATURES)


def test_log2_table_is_correctly_rounded():
    lib = fic.load()
    for n in range(1, 513):
        assert lib.fic_debug_log2(n) == dbc.log2_cr(n), n


def test_debug_stall_hook_validates_on_the_host():
    lib = fic.load()
    assert lib.fic_debug_stall_matcher(-1) == fic.FIC_ERR_INVALID_ARG
    assert lib.fic_debug_stall_matcher(2_000_000_000) == fic.FIC_ERR_INVALID_ARG
    assert lib.fic_debug_stall_matcher(0) == fic.FIC_OK


def _ws_size(H, W, **kw):
    p = fic.EncodeParams(**kw).c()
    g = fic.geom(H, W)
    return fic.load().fic_encode_workspace_size(ctypes.byref(g), ctypes.byref(p))


def test_workspace_size_and_validation():
    assert _ws_size(256, 256, domain_stride=8, num_classes=8) > 0
    assert _ws_size(1024, 1024, domain_stride=4, num_classes=16) > _ws_size(256, 256)
    for kw in ({"domain_stride": 0}, {"num_classes": 0}, {"num_classes": 256},
               {"block": 12}, {"s_max": 0.5}, {"half_width": -2},
               {"group_chunks": -1}, {"group_chunks": 1025},
               {"pipeline_stages": 2}, {"pipeline_stages": 5}, {"block": 16, "pipeline_stages": 3},
               {"block": 16, "pipeline_stages": 6}):
        assert _ws_size(64, 64, **kw) == 0, kw
    assert _ws_size(12, 64) == 0 and _ws_size(64, 60) == 0 and _ws_size(8, 64) == 0
    # 16x16 ranges: sides multiples of 16 and at least 32
    assert _ws_size(64, 64, block=16) > 0
    assert _ws_size(24, 64, block=16) == 0 and _ws_size(64, 48, block=16) > 0 and _ws_size(16, 64, block=16) == 0
    assert _ws_size(1024, 1024, block=16) > _ws_size(512, 512, block=16)
    # the literal FD window for both range sizes; the 16x16 one needs its key and sort scratch
    assert _ws_size(64, 64, literal=True) > 0
    assert _ws_size(64, 64, block=16, literal=True) > _ws_size(64, 64, block=16)
    assert fic.LITERAL16_OFFSETS == 2246
    for kw in ({"pipeline_stages": 3}, {"pipeline_stages": 4}, {"block": 16, "pipeline_stages": 4},
               {"block": 16, "pipeline_stages": 5}, {"group_chunks": 1}, {"group_chunks": 1024}):
        assert _ws_size(64, 64, **kw) > 0, kw
    # smaller domain groups need more work-item slots
    assert _ws_size(4096, 4096, domain_stride=8, group_chunks=4) > _ws_size(4096, 4096, domain_stride=8)


def test_encode_rejects_before_any_launch():
    lib = fic.load()
    p = fic.EncodeParams(domain_stride=4, num_classes=8).c()
    g = fic.geom(64, 64)
    codes = fic.Codes(*(ctypes.c_void_p(0x1000) for _ in range(5)))
    # null workspace
    st = lib.fic_encode(ctypes.c_void_p(0x1000), ctypes.byref(g), ctypes.byref(p),
                        ctypes.byref(codes), None, None, 0, None)
    assert st == fic.FIC_ERR_WORKSPACE and b"workspace" in lib.fic_last_error()
    # a workspace too small once aligned to 1024 bytes
    need = lib.fic_encode_workspace_size(ctypes.byref(g), ctypes.byref(p))
    st = lib.fic_encode(ctypes.c_void_p(0x1000), ctypes.byref(g), ctypes.byref(p),
                        ctypes.byref(codes), None, ctypes.c_void_p(0x1008), need - 1024, None)
    assert st == fic.FIC_ERR_WORKSPACE
    # batched: bad count
    assert lib.fic_encode_batched_workspace_size(ctypes.byref(g), 0, ctypes.byref(p)) == 0
    assert lib.fic_encode_batched_workspace_size(ctypes.byref(g), 1, ctypes.byref(p)) == need
    # too small
    st = lib.fic_encode(ctypes.c_void_p(0x1000), ctypes.byref(g), ctypes.byref(p),
                        ctypes.byref(codes), None, ctypes.c_void_p(0x1000), 1024, None)
    assert st == fic.FIC_ERR_WORKSPACE
    # bad geometry
    g2 = fic.geom(60, 64)
    st = lib.fic_encode(ctypes.c_void_p(0x1000), ctypes.byref(g2), ctypes.byref(p),
                        ctypes.byref(codes), None, ctypes.c_void_p(0x1000), 1 << 30, None)
    assert st == fic.FIC_ERR_INVALID_ARG
    # null code pointer
    codes_bad = fic.Codes(None, None, None, None, None)
    st = lib.fic_encode(ctypes.c_void_p(0x1000), ctypes.byref(g), ctypes.byref(p),
                        ctypes.byref(codes_bad), None, ctypes.c_void_p(0x1000), 1 << 30, None)
    assert st == fic.FIC_ERR_INVALID_ARG


def test_decode_rejects_bad_arguments():
    lib = fic.load()
    p = fic.EncodeParams(domain_stride=4).c()
    g = fic.geom(64, 64)
    codes = fic.Codes(*(ctypes.c_void_p(0x1000) for _ in range(5)))
    assert lib.fic_decode_workspace_size(ctypes.byref(g), ctypes.byref(p), -1, 1) == 0
    st = lib.fic_decode(ctypes.byref(codes), ctypes.byref(g), ctypes.byref(p), -1, None,
                        ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000), 1 << 20, None)
    assert st == fic.FIC_ERR_INVALID_ARG
    st = lib.fic_decode_backward(ctypes.byref(codes), ctypes.byref(g), ctypes.byref(p), 4, 0,
                                 None, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000),
                                 ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000), 1 << 20, None)
    assert st == fic.FIC_ERR_INVALID_ARG


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    img = torch.zeros(64, 64, dtype=torch.uint8)
    with pytest.raises(ValueError):
        fic.encode(img, fic.EncodeParams())


def test_fallback_ranges_and_check_validate_on_the_host():
    """fic_encode_fallback_ranges refuses bad arguments before any launch; fic_check reports a
    CUDA failure (no device here) or, on a GPU machine, nothing pending."""
    import torch

    lib = fic.load()
    p = fic.EncodeParams(domain_stride=4, num_classes=8).c()
    g = fic.geom(64, 64)
    n = ctypes.c_int32(0)
    assert lib.fic_encode_fallback_ranges(None, ctypes.byref(p), None, 0, None, 0, ctypes.byref(n), None) \
        == fic.FIC_ERR_INVALID_ARG
    assert lib.fic_encode_fallback_ranges(ctypes.byref(g), ctypes.byref(p), None, 0, None, 0, ctypes.byref(n),
                                          None) == fic.FIC_ERR_WORKSPACE
    buf = ctypes.create_string_buffer(64)
    assert lib.fic_encode_fallback_ranges(ctypes.byref(g), ctypes.byref(p), buf, 64, None, 0, ctypes.byref(n),
                                          None) == fic.FIC_ERR_WORKSPACE
    bad = fic.EncodeParams(domain_stride=4, num_classes=8, pipeline_stages=7).c()
    assert lib.fic_encode_fallback_ranges(ctypes.byref(g), ctypes.byref(bad), buf, 64, None, 0,
                                          ctypes.byref(n), None) == fic.FIC_ERR_INVALID_ARG
    expected = fic.FIC_OK if torch.cuda.is_available() else fic.FIC_ERR_CUDA
    assert lib.fic_check(None) == expected
