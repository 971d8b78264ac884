"""Autotuner for the tensor engine's tile pipeline and schedule.

Three shape parameters of the tensor matchers change their speed but never their results:

* ``pipeline_stages``: how many shared-memory stages the streamed domain operand (B) ring has
  (3 or 4 for 8x8 ranges, 4 or 5 for 16x16 ranges): deeper rings hide more TMA latency, shallower
  ones leave the CTA more shared memory headroom;
* ``group_chunks``: how many 512-domain chunks form one domain group, the band of B rows that the
  SMs running at the same time stream (the schedule is group-major so a group stays L2-resident):
  larger groups mean fewer, longer work items per range tile, smaller groups keep the band in L2
  when the batch's operands are much larger than it;
* ``items_per_sm``: how many work items per SM the work list aims for: fewer, longer items cost
  less per-item overhead (operand reloads, key writes), more, shorter items balance uneven
  per-class pools better.

The best combination depends on the image sizes and the class structure of the batch, so this
module times every candidate on the caller's own images and keeps the fastest. Results are cached
in a JSON file (``$FIC_AUTOTUNE_CACHE``, default ``~/.cache/fic/autotune.json``) keyed by the GPU
name and a signature of the workload (image shapes, domain stride, classes, half-width, engine).
"""
from __future__ import annotations

import dataclasses
import hashlib
import itertools
import json
import os
import statistics

import torch

from . import fic

STAGES = {8: (3, 4), 16: (4, 5)}
GROUP_CHUNKS = {8: (16, 32, 64, 128), 16: (4, 8, 16, 32)}
ITEMS_PER_SM = {8: (8, 24, 48), 16: (16, 48)}
# bumped when the matchers' scheduling changes, so that timings cached under another schedule are
# not reused (3: stages, domain-group size and items per SM are tuned together; 4: the 8x8
# matcher's epilogue warp sets drain whole tiles of alternate accumulators)
SCHEDULE = 4


def candidates(block: int):
    """Every (pipeline_stages, group_chunks, items_per_sm) combination tried for `block`."""
    return [dict(pipeline_stages=s, group_chunks=g, items_per_sm=i)
            for s, g, i in itertools.product(STAGES[block], GROUP_CHUNKS[block], ITEMS_PER_SM[block])]


def label(c: dict) -> str:
    return f"s{c['pipeline_stages']}_g{c['group_chunks']}_i{c['items_per_sm']}"


def cache_path() -> str:
    return os.environ.get("FIC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fic", "autotune.json"))


def signature(shapes, p: fic.EncodeParams) -> str:
    desc = {"shapes": sorted([list(s) for s in shapes]), "sigma": p.domain_stride,
            "K": p.num_classes, "w": p.half_width, "engine": p.engine, "block": p.block,
            "literal": p.literal, "schedule": SCHEDULE}
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


def tune(imgs, p: fic.EncodeParams, cands=None, reps: int = 3, use_cache: bool = True):
    """Best shape parameters for encoding `imgs` (list of uint8 CUDA tensors) with parameters `p`.

    Returns (best, times, noise): `best` a dict of the fields to set on `p`
    (pipeline_stages, group_chunks, items_per_sm), `times` the median milliseconds of one
    fic_encode_batched call per candidate label, `noise` the largest spread (max - min, ms) of a
    candidate's repetitions: differences below it are not significant."""
    shapes = [tuple(t.shape) for t in imgs]
    key = f"{torch.cuda.get_device_name()}|{signature(shapes, p)}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit["best"], hit["ms"], hit["noise_ms"]
    cands = candidates(p.block) if cands is None else cands
    # smaller domain groups need more work-item slots: one workspace sized for the smallest
    size = max(fic.encode_batched_workspace_size(shapes, dataclasses.replace(p, **c)) for c in cands)
    ws = torch.empty(size, dtype=torch.uint8, device=imgs[0].device)
    outs = None
    times, noise = {}, 0.0
    for c in cands:
        pc = dataclasses.replace(p, **c)
        outs = fic.encode_batched(imgs, pc, outs=outs, workspace=ws)
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fic.encode_batched(imgs, pc, outs=outs, workspace=ws)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        times[label(c)] = statistics.median(ms)
        noise = max(noise, max(ms) - min(ms))
    by_label = {label(c): c for c in cands}
    best = by_label[min(times, key=times.get)]
    _store(key, {"best": best, "ms": times, "noise_ms": noise})
    return best, times, noise
