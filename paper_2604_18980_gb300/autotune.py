"""Autotuner for the launch parameters of a rendering workload.

The knobs are the digit width of the radix sorts (7, 8 or 9 bits: fewer,
wider passes against more contention and larger look-back tables), whether
the Gaussians are depth-sorted before emission (the pair sort then runs only
the tile digits, on 32-bit keys), how the pair sort ranks a warp's equal
digits (warp match, or atomic-OR peer masks in shared memory) and whether the
tile-key emission runs as one fused pass or as two passes balanced by pairs.  Every candidate renders the same frames through
the same kernels -- results are identical -- and the fastest one (CUDA-event
time of a whole forward, after warm-up) is kept.  Results are cached in a JSON
file keyed by GPU name and workload shape.
"""
from __future__ import annotations

import json
import os

import torch

from . import binding as B
from . import render as R

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
CANDIDATES = ([dict(digit_bits=d, presort=True, pair_rank_or=o, emit_two_pass=t) for t in (True, False)
               for o in (True, False) for d in (9, 8, 7)]
              + [dict(digit_bits=d, presort=False, pair_rank_or=o) for o in (True, False) for d in (9, 8, 7)])


def workload_key(scene: dict, cams: list, scale_mode: int) -> str:
    n = int(scene["opacity_logit"].shape[0])
    return "%s|n=%d|views=%d|%dx%d|mode=%d" % (torch.cuda.get_device_name(), n, len(cams), cams[0]["width"],
                                                 cams[0]["height"], scale_mode)


def _time_forward(r: R.Renderer, warmup: int, reps: int) -> float:
    for _ in range(warmup):
        r.forward()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        r.forward()
    b.record()
    torch.cuda.synchronize()
    r.check()
    return a.elapsed_time(b) / reps


def tune(scene: dict, cams: list, scale_mode: int = B.AGS_SCALE_ADAGSCALE, K: float = 0.0, lut=None,
         warmup: int = 2, reps: int = 5, use_cache: bool = True, candidates=None) -> dict:
    """Fastest configuration for this workload: {"digit_bits", "presort", "pair_rank_or", "ms", "table"}."""
    key = workload_key(scene, cams, scale_mode)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]
    table = []
    capacity = None
    for cand in candidates or CANDIDATES:
        r = R.Renderer(scene, cams, scale_mode, K, lut, capacity=capacity, keep_state=False, **cand)
        capacity = r.capacity
        ms = _time_forward(r, warmup, reps)
        table.append(dict(cand, ms=ms))
        del r
    best = min(table, key=lambda t: t["ms"])
    out = dict(digit_bits=best["digit_bits"], presort=best["presort"], pair_rank_or=best["pair_rank_or"],
               emit_two_pass=best.get("emit_two_pass", True), ms=best["ms"], table=table)
    if use_cache:
        cache[key] = out
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".tmp%d" % os.getpid()
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, CACHE)
    return out
