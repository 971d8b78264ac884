"""Autotuner for the tensor engine's scheduling granularity.

The tensor engine splits every range tile's domain chunks into work items so that the whole batch
has about `items_per_sm` items per SM: fewer, longer items cost less per-item overhead (operand
reloads, key writes); more, shorter items balance uneven per-class pools better across SMs. The
best value depends on the image sizes and the class structure of the batch, so this module times
the candidates on the caller's own images and keeps the fastest. Results are cached in a JSON
file (``$FIC_AUTOTUNE_CACHE``, default ``~/.cache/fic/autotune.json``) keyed by the GPU name and
a signature of the workload (image shapes, domain stride, classes, half-width, engine).
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os
import statistics

import torch

from . import fic

CANDIDATES = (4, 8, 16, 24, 32)
# bumped when the matchers' scheduling changes, so that timings cached under another schedule are
# not reused (2: persistent CTAs fetch work items from a global counter)
SCHEDULE = 2


def cache_path() -> str:
    return os.environ.get("FIC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fic", "autotune.json"))


def signature(shapes, p: fic.EncodeParams) -> str:
    desc = {"shapes": sorted([list(s) for s in shapes]), "sigma": p.domain_stride,
            "K": p.num_classes, "w": p.half_width, "engine": p.engine, "block": p.block,
            "schedule": SCHEDULE}
    return hashlib.sha1(json.dumps(desc, sort_keys=True).encode()).hexdigest()[:16]


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    cache = _load_cache()
    cache[key] = value
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(imgs, p: fic.EncodeParams, candidates=CANDIDATES, reps: int = 3, use_cache: bool = True):
    """Best items_per_sm for encoding `imgs` (list of uint8 CUDA tensors) with parameters `p`.
    Returns (items_per_sm, {candidate: median ms})."""
    shapes = [tuple(t.shape) for t in imgs]
    key = f"{torch.cuda.get_device_name()}|{signature(shapes, p)}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return int(hit["items_per_sm"]), {int(k): v for k, v in hit["ms"].items()}
    ws = torch.empty(fic.encode_batched_workspace_size(shapes, p), dtype=torch.uint8, device=imgs[0].device)
    outs = None
    times = {}
    for c in candidates:
        pc = dataclasses.replace(p, items_per_sm=int(c))
        outs = fic.encode_batched(imgs, pc, outs=outs, workspace=ws)
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fic.encode_batched(imgs, pc, outs=outs, workspace=ws)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        times[int(c)] = statistics.median(ms)
    best = min(times, key=times.get)
    _store(key, {"items_per_sm": best, "ms": times})
    return best, times
