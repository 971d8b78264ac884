"""Oracle: fractal decoding, its adjoint with respect to the codes, and PSNR.

Test infrastructure only (see the package docstring).

Section 1: decoding applies the stored maps to an initial image (typically a plain background)
repeatedly; the maps are contractive, so the iterates are attracted to a fixed point. The paper
gives no schedule; this oracle reads it as the Jacobi iteration

    x_{k+1}[range r] = s_r * T_{t_r}(D(x_k, d_r)) + o_r     for every range r,

with D(x, d) the 2x2 average of the 2B x 2B domain d of x_k, x_0 = 128 everywhere (a mid-grey
background) unless given, no clamping between iterations, and the decoded 8-bit image
clamp(round-half-even(x_K), 0, 255). PSNR (Table 4) is 10 log10(255^2 / MSE).

The adjoint: with W the linear part of one step (x -> s * T(D(x))), lambda_K = dL/dx_K and
lambda_k = W^T lambda_{k+1}, the gradients are
    dL/ds_r = sum_k sum_{p in r} lambda_{k+1}[p] * T_{t_r}(D(x_k, d_r))[p]
    dL/do_r = sum_k sum_{p in r} lambda_{k+1}[p].
Resolution independence (Section 1: the initial image may have any size, and decoding can
reconstruct at any size): decode_scaled applies the same codes on a z-times larger grid:
range r covers the (8z) x (8z) block at z times its position, domain d the (16z) x (16z) block at
z times its position, contracted by 2x2 averaging, with the isometries of the larger square.

Everything is binary64.
"""
from __future__ import annotations

import numpy as np

from . import geometry


def _contract(x: np.ndarray, B: int, dy: int, dx: int) -> np.ndarray:
    blk = x[dy:dy + 2 * B, dx:dx + 2 * B]
    return (blk[0::2, 0::2] + blk[0::2, 1::2] + blk[1::2, 0::2] + blk[1::2, 1::2]) / 4.0


def decode_step(x: np.ndarray, codes: dict, B: int, sigma: int) -> np.ndarray:
    H, W = x.shape
    y = np.empty_like(x)
    for r in range(geometry.n_ranges(H, W, B)):
        dy, dx = geometry.domain_origin(H, W, B, sigma, int(codes["dom"][r]))
        ry, rx = geometry.range_origin(H, W, B, r)
        D = _contract(x, B, dy, dx)
        y[ry:ry + B, rx:rx + B] = codes["s"][r] * geometry.isometry(D, int(codes["iso"][r])) + codes["o"][r]
    return y


def decode(codes: dict, H: int, W: int, B: int, sigma: int, iters: int, x0=None) -> np.ndarray:
    x = np.full((H, W), 128.0) if x0 is None else np.array(x0, dtype=np.float64)
    for _ in range(iters):
        x = decode_step(x, codes, B, sigma)
    return x


def to_u8(x: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2)
    return float("inf") if mse == 0 else float(10.0 * np.log10(255.0 ** 2 / mse))


def decode_adjoint(codes: dict, H: int, W: int, B: int, sigma: int, iters: int,
                   grad_out: np.ndarray, x0=None):
    """(dL/ds, dL/do) per range for L with dL/dx_K = grad_out."""
    xs = [np.full((H, W), 128.0) if x0 is None else np.array(x0, dtype=np.float64)]
    for _ in range(iters):
        xs.append(decode_step(xs[-1], codes, B, sigma))
    R = geometry.n_ranges(H, W, B)
    gs = np.zeros(R)
    go = np.zeros(R)
    lam = np.array(grad_out, dtype=np.float64)
    for k in range(iters - 1, -1, -1):
        x = xs[k]
        prev = np.zeros((H, W))
        for r in range(R):
            t = int(codes["iso"][r])
            dy, dx = geometry.domain_origin(H, W, B, sigma, int(codes["dom"][r]))
            ry, rx = geometry.range_origin(H, W, B, r)
            L = lam[ry:ry + B, rx:rx + B]
            gs[r] += float(np.sum(L * geometry.isometry(_contract(x, B, dy, dx), t)))
            go[r] += float(np.sum(L))
            # adjoint of D then T_t: T_t^T = T_t^{-1}, D^T spreads a quarter to each 2x2 cell
            G = geometry.isometry(L, geometry.INVERSE[t]) * (codes["s"][r] / 4.0)
            for a in (0, 1):
                for b in (0, 1):
                    prev[dy + a:dy + 2 * B:2, dx + b:dx + 2 * B:2] += G
        lam = prev
    return gs, go


def decode_scaled(codes: dict, H: int, W: int, B: int, sigma: int, iters: int, z: int, x0=None) -> np.ndarray:
    """Decode codes of an H x W encoding on the (zH) x (zW) grid (module docstring)."""
    Bz = B * z
    x = np.full((z * H, z * W), 128.0) if x0 is None else np.array(x0, dtype=np.float64)
    for _ in range(iters):
        y = np.empty_like(x)
        for r in range(geometry.n_ranges(H, W, B)):
            dy, dx = geometry.domain_origin(H, W, B, sigma, int(codes["dom"][r]))
            ry, rx = geometry.range_origin(H, W, B, r)
            D = _contract(x, Bz, z * dy, z * dx)
            y[z * ry:z * ry + Bz, z * rx:z * rx + Bz] = codes["s"][r] * geometry.isometry(D, int(codes["iso"][r])) + codes["o"][r]
        x = y
    return x
