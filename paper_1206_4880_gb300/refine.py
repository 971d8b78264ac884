"""Refinement of the fractal codes against their decoded attractor, then re-quantisation.

The encoder fits each range by least squares against the *original* image's domains (the collage),
but the decoder reconstructs from its own iterates. With the domain and isometry of every range
fixed, the decoded image after K iterations is a smooth function x_K(s, o) of the contrasts and
brightnesses, so (s, o) can be refined by gradient descent on 0.5 ||x_K - I||^2, with |s| <= 1
kept by projection. The gradients come from `fic.Decode`, whose backward pass is the library's
checkpointed adjoint (fic_decode_backward); the optimiser (Adam, one step size for s and one for o)
only updates two vectors of R numbers. The refined codes are then quantised by fic_quantize.
"""
from __future__ import annotations

import torch

from . import fic


def refine(codes: dict, img: torch.Tensor, p: fic.EncodeParams, iters: int = 8, ckpt_every: int = 2,
           steps: int = 20, lr_s: float = 0.01, lr_o: float = 0.5) -> dict:
    """Codes with s, o refined against the decode of `img` (uint8 CUDA, H x W); dom, iso unchanged."""
    H, W = img.shape
    s = codes["s"].detach().to(torch.float64).clone().requires_grad_(True)
    o = codes["o"].detach().to(torch.float64).clone().requires_grad_(True)
    target = img.to(torch.float32)
    opt = torch.optim.Adam([{"params": [s], "lr": lr_s}, {"params": [o], "lr": lr_o}])
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        x = fic.Decode.apply(s, o, codes["dom"], codes["iso"], H, W, p, iters, ckpt_every)
        loss = 0.5 * torch.sum((x - target) ** 2)
        loss.backward()
        opt.step()
        with torch.no_grad():
            s.clamp_(-1.0, 1.0)
    out = {"dom": codes["dom"], "iso": codes["iso"], "s": s.detach().contiguous(), "o": o.detach().contiguous()}
    if "sse" in codes:
        out["sse"] = codes["sse"]
    return out


def refine_and_quantize(codes: dict, img: torch.Tensor, p: fic.EncodeParams, bits_s: int = 5, bits_o: int = 7,
                        iters: int = 8, **kw) -> dict:
    """Decoded PSNR of the codes as encoded, quantised, refined, and refined then quantised."""
    H, W = img.shape

    def psnr(c):
        return fic.quality(fic.decode(c, H, W, p, iters), img)[1]

    report = {"psnr_encoded": psnr(codes)}
    q, _, _, _ = fic.quantize(codes, bits_s, bits_o)
    report["psnr_quantized"] = psnr(q)
    r = refine(codes, img, p, iters=iters, **kw)
    report["psnr_refined"] = psnr(r)
    rq, _, _, _ = fic.quantize(r, bits_s, bits_o)
    report["psnr_refined_quantized"] = psnr(rq)
    return report
