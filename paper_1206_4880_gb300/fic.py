"""Python binding of the fic C ABI (include/fic.h).

Argument marshalling only: every step of the encoder and decoder runs in the CUDA library
``_lib/libfic.so``. PyTorch supplies device memory and the current stream. There is no CPU
fallback: if the library is missing or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build

FIC_OK, FIC_ERR_INVALID_ARG, FIC_ERR_WORKSPACE, FIC_ERR_CUDA, FIC_ERR_DEVICE_TIMEOUT, \
    FIC_ERR_UNSUPPORTED = range(6)
ENGINES = {"tensor": 0, "simt": 1}
FLAG_LITERAL_WINDOW = 1
LITERAL16_OFFSETS = 2246  # FIC_LITERAL16_OFFSETS

c_i32, c_i64, c_dbl, c_vp, c_size = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t


class Geom(ctypes.Structure):
    _fields_ = [("H", c_i32), ("W", c_i32), ("pitch", c_i32)]


class Params(ctypes.Structure):
    _fields_ = [("block", c_i32), ("domain_stride", c_i32), ("num_classes", c_i32),
                ("half_width", c_i32), ("s_max", c_dbl), ("engine", c_i32), ("flags", c_i32),
                ("items_per_sm", c_i32), ("group_chunks", c_i32), ("pipeline_stages", c_i32)]


class BlockStats(ctypes.Structure):
    _fields_ = [(n, c_vp) for n in ("range_sum", "range_sumsq", "range_counts", "range_fd",
                                    "range_bin", "dom_sum", "dom_sumsq", "dom_counts", "dom_fd",
                                    "dom_bin", "fd_extent")]


class Pools(ctypes.Structure):
    _fields_ = [(n, c_vp) for n in ("dom_order", "bin_off", "range_order", "rbin_off", "win_lo",
                                    "win_hi")]


class Codes(ctypes.Structure):
    _fields_ = [(n, c_vp) for n in ("dom", "iso", "s", "o", "sse")]


class EncodeInfo(ctypes.Structure):
    _fields_ = [("matches", c_i64), ("fallback_ranges", c_i32), ("work_items", c_i32),
                ("device_error", c_i32), ("reserved", c_i32)]


# Every exported symbol of include/fic.h, with its ctypes signature.
SIGNATURES = {
    "fic_encode_workspace_size": (c_size, [c_vp, c_vp]),
    "fic_classify": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "fic_build_pools": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "fic_encode": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "fic_encode_fallback_ranges": (c_i32, [c_vp, c_vp, c_vp, c_size, c_vp, c_i32, c_vp, c_vp]),
    "fic_encode_batched_workspace_size": (c_size, [c_vp, c_i32, c_vp]),
    "fic_encode_batched": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "fic_decode_workspace_size": (c_size, [c_vp, c_vp, c_i32, c_i32]),
    "fic_decode": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_size, c_vp]),
    "fic_decode_backward": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp,
                                    c_size, c_vp]),
    "fic_profile_enable": (c_i32, [c_i32]),
    "fic_profile_read": (c_i32, [c_vp, c_i32, c_vp]),
    "fic_decode_static": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp]),
    "fic_quality": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "fic_quantize": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "fic_decode_scaled_workspace_size": (c_size, [c_vp, c_vp, c_i32]),
    "fic_decode_scaled": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_size, c_vp]),
    "fic_check": (c_i32, [c_vp]),
    "fic_debug_stall_matcher": (c_i32, [c_i64]),
    "fic_engine_available": (c_i32, [c_i32]),
    "fic_last_error": (ctypes.c_char_p, []),
    "fic_version": (c_i32, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfic.so (building it in-tree if it is absent and nvcc exists)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"fic CUDA library not built: {path}")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        lib.fic_debug_log2.restype = c_dbl
        lib.fic_debug_log2.argtypes = [c_i32]
        _lib = lib
    return _lib


class FicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fic status {status}: {msg}")
        self.status = status


def _check(status):
    if status != FIC_OK:
        raise FicError(status, load().fic_last_error().decode())


@dataclass
class EncodeParams:
    domain_stride: int = 8
    num_classes: int = 8
    half_width: int = -1
    engine: str = "tensor"
    block: int = 8
    s_max: float = 1.0
    items_per_sm: int = 0
    literal: bool = False   # Eq. 3's window on FD values instead of the class window
    group_chunks: int = 0   # tensor engine: chunk cap of a domain group (0: library default)
    pipeline_stages: int = 0  # tensor engine: domain-operand ring stages (0: library default)

    def c(self) -> Params:
        return Params(self.block, self.domain_stride, self.num_classes, self.half_width,
                      self.s_max, ENGINES[self.engine], FLAG_LITERAL_WINDOW if self.literal else 0,
                      self.items_per_sm, self.group_chunks, self.pipeline_stages)


def geom(H: int, W: int, pitch: int | None = None) -> Geom:
    return Geom(H, W, W if pitch is None else pitch)


def _p(t: torch.Tensor | None):
    return c_vp(0) if t is None else c_vp(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return c_vp(s.cuda_stream)


def _require_cuda(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


def n_scales(block: int) -> int:
    """Box-count scales per block: s = 2, 4 for 8x8 blocks; s = 2, 4, 8 for 16x16 blocks."""
    return 3 if block == 16 else 2


def counts(H: int, W: int, p: EncodeParams) -> tuple[int, int]:
    B = p.block
    R = (H // B) * (W // B)
    Dn = ((H - 2 * B) // p.domain_stride + 1) * ((W - 2 * B) // p.domain_stride + 1)
    return R, Dn


def encode_workspace_size(H: int, W: int, p: EncodeParams) -> int:
    g, pc = geom(H, W), p.c()
    n = load().fic_encode_workspace_size(ctypes.byref(g), ctypes.byref(pc))
    if n == 0:
        raise FicError(FIC_ERR_INVALID_ARG, load().fic_last_error().decode())
    return n


def alloc_codes(R: int, device) -> dict:
    return {"dom": torch.empty(R, dtype=torch.int32, device=device),
            "iso": torch.empty(R, dtype=torch.int32, device=device),
            "s": torch.empty(R, dtype=torch.float64, device=device),
            "o": torch.empty(R, dtype=torch.float64, device=device),
            "sse": torch.empty(R, dtype=torch.float64, device=device)}


def _codes_struct(c: dict) -> Codes:
    return Codes(_p(c["dom"]), _p(c["iso"]), _p(c["s"]), _p(c["o"]), _p(c.get("sse")))


def encode(img: torch.Tensor, p: EncodeParams, out: dict | None = None,
           workspace: torch.Tensor | None = None, info: torch.Tensor | None = None,
           stream=None) -> dict:
    """fic_encode on a uint8 CUDA image (H x W, rows may be padded: pitch = img.stride(0))."""
    _require_cuda(img, "img")
    if img.dtype != torch.uint8 or img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("img must be a 2-D uint8 tensor with unit column stride")
    H, W = img.shape
    g, pc = geom(H, W, img.stride(0)), p.c()
    R, _ = counts(H, W, p)
    if out is None:
        out = alloc_codes(R, img.device)
    if workspace is None:
        workspace = torch.empty(encode_workspace_size(H, W, p), dtype=torch.uint8, device=img.device)
    cs = _codes_struct(out)
    _check(load().fic_encode(_p(img), ctypes.byref(g), ctypes.byref(pc), ctypes.byref(cs),
                             _p(info), _p(workspace), workspace.numel(), _stream(stream)))
    return out


def check(stream=None):
    """fic_check: wait for `stream` and raise FicError (status FIC_ERR_DEVICE_TIMEOUT) if a bounded
    device-side wait of an encode on this device gave up since the last check."""
    _check(load().fic_check(_stream(stream)))


def debug_stall_matcher(ns: int):
    """fic_debug_stall_matcher: testing hook that makes this thread's tensor matchers time out
    (ns > 0) before they issue any work; 0 turns it off."""
    _check(load().fic_debug_stall_matcher(int(ns)))


def fallback_ranges(H: int, W: int, p: EncodeParams, workspace: torch.Tensor, stream=None) -> torch.Tensor:
    """fic_encode_fallback_ranges: ids of the ranges the last encode with `workspace` re-searched
    exactly because the tensor engine's ranking could not certify them (sorted)."""
    R, _ = counts(H, W, p)
    ids = torch.empty(R, dtype=torch.int32, device=workspace.device)
    n = torch.zeros(1, dtype=torch.int32, device=workspace.device)
    g, pc = geom(H, W), p.c()
    _check(load().fic_encode_fallback_ranges(ctypes.byref(g), ctypes.byref(pc), _p(workspace),
                                             workspace.numel(), _p(ids), R, _p(n), _stream(stream)))
    return torch.sort(ids[:int(n.item())]).values


def engine_available(engine: str) -> bool:
    """Whether the library can run `engine` on the current CUDA device."""
    return bool(load().fic_engine_available(ENGINES[engine]))


def encode_batched_workspace_size(shapes, p: EncodeParams) -> int:
    n = len(shapes)
    geoms = (Geom * n)(*[geom(H, W) for H, W in shapes])
    pc = p.c()
    size = load().fic_encode_batched_workspace_size(geoms, n, ctypes.byref(pc))
    if size == 0:
        raise FicError(FIC_ERR_INVALID_ARG, load().fic_last_error().decode())
    return size


def encode_batched(imgs, p: EncodeParams, outs=None, workspace=None, info=None, stream=None):
    """fic_encode_batched over a list of uint8 CUDA images (any sizes); returns one code dict per
    image. The tensor engine matches all images in one persistent launch."""
    n = len(imgs)
    for t in imgs:
        _require_cuda(t, "img")
        if t.dtype != torch.uint8 or t.dim() != 2 or t.stride(1) != 1:
            raise ValueError("images must be 2-D uint8 tensors with unit column stride")
    geoms = (Geom * n)(*[geom(t.shape[0], t.shape[1], t.stride(0)) for t in imgs])
    if outs is None:
        outs = [alloc_codes(counts(t.shape[0], t.shape[1], p)[0], t.device) for t in imgs]
    if workspace is None:
        workspace = torch.empty(encode_batched_workspace_size([tuple(t.shape) for t in imgs], p),
                                dtype=torch.uint8, device=imgs[0].device)
    ptrs = (c_vp * n)(*[t.data_ptr() for t in imgs])
    cs = (Codes * n)(*[_codes_struct(o) for o in outs])
    pc = p.c()
    _check(load().fic_encode_batched(ptrs, geoms, n, ctypes.byref(pc), cs, _p(info), _p(workspace),
                                     workspace.numel(), _stream(stream)))
    return outs


def new_info(device) -> torch.Tensor:
    return torch.zeros(ctypes.sizeof(EncodeInfo), dtype=torch.uint8, device=device)


def read_info(info: torch.Tensor) -> dict:
    raw = bytes(info.cpu().numpy().tobytes())
    s = EncodeInfo.from_buffer_copy(raw)
    return {"matches": s.matches, "fallback_ranges": s.fallback_ranges,
            "work_items": s.work_items, "device_error": s.device_error}


def classify(img: torch.Tensor, p: EncodeParams, workspace=None, stream=None) -> dict:
    _require_cuda(img, "img")
    H, W = img.shape
    R, Dn = counts(H, W, p)
    dev = img.device
    i32, f64, u8 = torch.int32, torch.float64, torch.uint8
    st = {"range_sum": torch.empty(R, dtype=i32, device=dev),
          "range_sumsq": torch.empty(R, dtype=i32, device=dev),
          "range_counts": torch.empty(R, n_scales(p.block), dtype=i32, device=dev),
          "range_fd": torch.empty(R, dtype=f64, device=dev),
          "range_bin": torch.empty(R, dtype=u8, device=dev),
          "dom_sum": torch.empty(Dn, dtype=i32, device=dev),
          "dom_sumsq": torch.empty(Dn, dtype=i32, device=dev),
          "dom_counts": torch.empty(Dn, n_scales(p.block), dtype=i32, device=dev),
          "dom_fd": torch.empty(Dn, dtype=f64, device=dev),
          "dom_bin": torch.empty(Dn, dtype=u8, device=dev),
          "fd_extent": torch.empty(2, dtype=f64, device=dev)}
    s = BlockStats(*[_p(st[n]) for n, _ in BlockStats._fields_])
    g, pc = geom(H, W, img.stride(0)), p.c()
    if workspace is None:
        workspace = torch.empty(encode_workspace_size(H, W, p), dtype=torch.uint8, device=dev)
    _check(load().fic_classify(_p(img), ctypes.byref(g), ctypes.byref(pc), ctypes.byref(s),
                               _p(workspace), workspace.numel(), _stream(stream)))
    return st


def build_pools(stats: dict, H: int, W: int, p: EncodeParams, workspace=None, stream=None) -> dict:
    R, Dn = counts(H, W, p)
    dev = stats["range_bin"].device
    i32 = torch.int32
    # bucket offsets: K + 1 entries, or one per FD key (+1) with the literal window (257 cover the
    # classes and the 8x8 literal window; the 16x16 literal window needs LITERAL16_OFFSETS)
    n_off = LITERAL16_OFFSETS if (p.literal and p.block == 16) else 257
    out = {"dom_order": torch.empty(Dn, dtype=i32, device=dev),
           "bin_off": torch.empty(n_off, dtype=i32, device=dev),
           "range_order": torch.empty(R, dtype=i32, device=dev),
           "rbin_off": torch.empty(n_off, dtype=i32, device=dev),
           "win_lo": torch.empty(R, dtype=i32, device=dev),
           "win_hi": torch.empty(R, dtype=i32, device=dev)}
    s = BlockStats(*[_p(stats[n]) for n, _ in BlockStats._fields_])
    po = Pools(*[_p(out[n]) for n, _ in Pools._fields_])
    g, pc = geom(H, W), p.c()
    if workspace is None:
        workspace = torch.empty(encode_workspace_size(H, W, p), dtype=torch.uint8, device=dev)
    _check(load().fic_build_pools(ctypes.byref(s), ctypes.byref(g), ctypes.byref(pc),
                                  ctypes.byref(po), _p(workspace), workspace.numel(),
                                  _stream(stream)))
    return out


def decode_workspace_size(H: int, W: int, p: EncodeParams, iters: int, ckpt_every: int = 1) -> int:
    g, pc = geom(H, W), p.c()
    n = load().fic_decode_workspace_size(ctypes.byref(g), ctypes.byref(pc), iters, ckpt_every)
    if n == 0:
        raise FicError(FIC_ERR_INVALID_ARG, load().fic_last_error().decode())
    return n


def decode(codes: dict, H: int, W: int, p: EncodeParams, iters: int, x0=None, out=None,
           workspace=None, stream=None) -> torch.Tensor:
    dev = codes["dom"].device
    if out is None:
        out = torch.empty(H, W, dtype=torch.float32, device=dev)
    if workspace is None:
        workspace = torch.empty(decode_workspace_size(H, W, p, iters), dtype=torch.uint8, device=dev)
    cs = _codes_struct(codes)
    g, pc = geom(H, W), p.c()
    _check(load().fic_decode(ctypes.byref(cs), ctypes.byref(g), ctypes.byref(pc), iters, _p(x0),
                             _p(out), _p(workspace), workspace.numel(), _stream(stream)))
    return out


def quality(x: torch.Tensor, ref: torch.Tensor, stream=None) -> tuple[float, float]:
    """(MSE, PSNR dB) of the decoded image clamp(round-half-even(x)) against the uint8 original,
    computed by the library on the GPU (Table 4's metric)."""
    _require_cuda(x, "x")
    _require_cuda(ref, "ref")
    H, W = ref.shape
    out = torch.empty(1026, dtype=torch.float64, device=x.device)
    g = geom(H, W, ref.stride(0))
    _check(load().fic_quality(_p(x.contiguous()), _p(ref), ctypes.byref(g), _p(out), _stream(stream)))
    mse, psnr = out[:2].tolist()
    return mse, psnr


def quantize(codes: dict, bits_s: int = 5, bits_o: int = 7, stream=None):
    """fic_quantize: (dequantised codes, q_s, q_o, (o_lo, o_hi)); the integer codes are uint16
    tensors stored as int16 bit patterns (torch has no uint16 arithmetic)."""
    dev = codes["s"].device
    n = codes["s"].numel()
    out = {"dom": torch.empty_like(codes["dom"]), "iso": torch.empty_like(codes["iso"]),
           "s": torch.empty_like(codes["s"]), "o": torch.empty_like(codes["o"])}
    if "sse" in codes:
        out["sse"] = codes["sse"].clone()
    q_s = torch.empty(n, dtype=torch.int16, device=dev)
    q_o = torch.empty(n, dtype=torch.int16, device=dev)
    header = torch.empty(514, dtype=torch.float64, device=dev)
    ci, co = _codes_struct(codes), _codes_struct(out)
    _check(load().fic_quantize(ctypes.byref(ci), n, bits_s, bits_o, _p(q_s), _p(q_o), _p(header),
                               ctypes.byref(co), _stream(stream)))
    lo, hi = header[:2].tolist()
    return out, q_s, q_o, (lo, hi)


DECODE_STATIC_MAX_PIXELS = 1 << 20


def decode_static(codes: dict, H: int, W: int, p: EncodeParams, iters: int, x0=None, out=None,
                  stream=None) -> torch.Tensor:
    """fic_decode_static: the same decode with no workspace (the library's fixed scratch image,
    at most DECODE_STATIC_MAX_PIXELS pixels)."""
    dev = codes["dom"].device
    if out is None:
        out = torch.empty(H, W, dtype=torch.float32, device=dev)
    cs = _codes_struct(codes)
    g, pc = geom(H, W), p.c()
    _check(load().fic_decode_static(ctypes.byref(cs), ctypes.byref(g), ctypes.byref(pc), iters,
                                    _p(x0), _p(out), _stream(stream)))
    return out


def decode_scaled(codes: dict, H: int, W: int, p: EncodeParams, scale: int, iters: int, x0=None,
                  out=None, stream=None) -> torch.Tensor:
    """fic_decode_scaled: the codes of an H x W encoding decoded on the (scale H) x (scale W) grid."""
    dev = codes["dom"].device
    if out is None:
        out = torch.empty(scale * H, scale * W, dtype=torch.float32, device=dev)
    g, pc = geom(H, W), p.c()
    n = load().fic_decode_scaled_workspace_size(ctypes.byref(g), ctypes.byref(pc), scale)
    if n == 0:
        raise FicError(FIC_ERR_INVALID_ARG, load().fic_last_error().decode())
    ws = torch.empty(n, dtype=torch.uint8, device=dev)
    cs = _codes_struct(codes)
    _check(load().fic_decode_scaled(ctypes.byref(cs), ctypes.byref(g), ctypes.byref(pc), scale, iters, _p(x0),
                                    _p(out), _p(ws), ws.numel(), _stream(stream)))
    return out


def decode_backward(codes: dict, H: int, W: int, p: EncodeParams, iters: int, ckpt_every: int,
                    grad_out: torch.Tensor, x0=None, workspace=None, stream=None, grad_s=None, grad_o=None):
    """dL/ds and dL/do of `iters` decoding steps given dL/dx (fic_decode_backward); grad_s and
    grad_o, when given, are R float32 device tensors that receive them (reused buffers let repeated
    calls replay the library's cached graph)."""
    dev = codes["dom"].device
    R, _ = counts(H, W, p)
    gs = torch.empty(R, dtype=torch.float32, device=dev) if grad_s is None else grad_s
    go = torch.empty(R, dtype=torch.float32, device=dev) if grad_o is None else grad_o
    for t in (gs, go):
        if t.dtype != torch.float32 or t.numel() != R or not t.is_contiguous() or t.device != dev:
            raise ValueError("grad_s and grad_o must be contiguous float32 tensors of R entries on the codes' device")
    if workspace is None:
        workspace = torch.empty(decode_workspace_size(H, W, p, iters, ckpt_every),
                                dtype=torch.uint8, device=dev)
    cs = _codes_struct(codes)
    g, pc = geom(H, W), p.c()
    grad_out = grad_out.contiguous().to(torch.float32)
    _check(load().fic_decode_backward(ctypes.byref(cs), ctypes.byref(g), ctypes.byref(pc), iters,
                                      ckpt_every, _p(x0), _p(grad_out), _p(gs), _p(go),
                                      _p(workspace), workspace.numel(), _stream(stream)))
    return gs, go


class Decode(torch.autograd.Function):
    """x_K = decode(codes with contrast s and brightness o) as a differentiable function of
    (s, o); the backward pass is the library's checkpointed adjoint."""

    @staticmethod
    def forward(ctx, s, o, dom, iso, H, W, p, iters, ckpt_every, x0=None):
        codes = {"dom": dom, "iso": iso, "s": s.detach().to(torch.float64).contiguous(),
                 "o": o.detach().to(torch.float64).contiguous()}
        ctx.save_for_backward(codes["s"], codes["o"], dom, iso)
        ctx.meta = (H, W, p, iters, ckpt_every, x0)
        return decode(codes, H, W, p, iters, x0=x0)

    @staticmethod
    def backward(ctx, grad_out):
        s, o, dom, iso = ctx.saved_tensors
        H, W, p, iters, ckpt_every, x0 = ctx.meta
        codes = {"dom": dom, "iso": iso, "s": s, "o": o}
        gs, go = decode_backward(codes, H, W, p, iters, ckpt_every, grad_out, x0=x0)
        return gs.to(s.dtype), go.to(o.dtype), None, None, None, None, None, None, None, None


STAGES = ("classify", "pools", "pack", "match", "reeval", "fallback")


def profile_enable(on: bool = True):
    _check(load().fic_profile_enable(1 if on else 0))


def profile_read() -> tuple[dict, int]:
    """Stage milliseconds of the last fic_encode on this thread and its kernel launch count."""
    ms = (ctypes.c_float * 6)()
    n = ctypes.c_int32(0)
    _check(load().fic_profile_read(ms, 6, ctypes.byref(n)))
    return {k: float(v) for k, v in zip(STAGES, ms)}, int(n.value)
