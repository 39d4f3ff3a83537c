"""Autotuner for the launch parameters of a rendering workload.

The knobs of the sort and emission stages are the digit width of the radix
sorts (7, 8 or 9 bits: fewer, wider passes against more contention and larger
look-back tables), whether the Gaussians are depth-sorted before emission
(the pair sort then runs only the tile digits, on 32-bit keys), how the pair
sort ranks a warp's equal digits (warp match, or atomic-OR peer masks in
shared memory) and whether the tile-key emission runs as one fused pass or as
two passes balanced by pairs.  The block shapes come second, on the best of
those: the blend's warp block (8x16 pixels, two warps a tile and four rows a
lane, or 8x8, four warps and two rows), its tile batch (32 or 64 splats
staged per warp and round) and the partition shape of the 32-bit sort passes
(256 threads of 16 keys or 512 of 8).  A third round picks the depth
pre-sort's grid: resident blocks taking partitions of the visible count, or
one block per partition of every Gaussian-view.  The stages do not interact,
so the rounds find the best combination with 28 timings instead of 288.  Every
candidate renders the same frames through the same kernels -- results are
identical -- and the fastest one (CUDA-event time of a whole forward, after
warm-up) is kept.  Results are cached in a JSON file keyed by GPU name and
workload shape.
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
SHAPES = [dict(blend_flags=f, sort_wide=w) for w in (False, True)
          for f in (0, B.AGS_BLEND_ROWS2, B.AGS_BLEND_BATCH64, B.AGS_BLEND_ROWS2 | B.AGS_BLEND_BATCH64)]
DEPTH_PASSES = [dict(depth_persistent=p) for p in (True, False)]
KNOBS = ("digit_bits", "presort", "pair_rank_or", "emit_two_pass", "blend_flags", "sort_wide", "depth_persistent")
DEFAULTS = dict(emit_two_pass=True, blend_flags=0, sort_wide=False, depth_persistent=True)


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
         warmup: int = 2, reps: int = 5, use_cache: bool = True, candidates=None, shapes=None) -> dict:
    """Fastest configuration for this workload: the KNOBS, "ms" and "table"
    (every timed candidate with its ms: the stage knobs, then the shapes, then
    the depth pre-sort's grid)."""
    key = workload_key(scene, cams, scale_mode)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except (OSError, ValueError):
            cache = {}
        if key in cache and all(k in cache[key] for k in KNOBS):
            return cache[key]
    table = []
    capacity = None

    def timed(cand):
        nonlocal capacity
        r = R.Renderer(scene, cams, scale_mode, K, lut, capacity=capacity, keep_state=False, **cand)
        capacity = r.capacity
        ms = _time_forward(r, warmup, reps)
        del r
        table.append(dict(cand, ms=ms))
        return ms

    best = min((dict(DEFAULTS, **c) for c in (candidates or CANDIDATES)), key=timed)
    stage = {k: best[k] for k in KNOBS if k not in ("blend_flags", "sort_wide")}
    best = min((dict(stage, **sh) for sh in (shapes if shapes is not None else SHAPES)), key=timed)
    if best["presort"]:       # the depth pre-sort's grid: resident blocks or one per partition
        best = min((dict(best, **dp) for dp in DEPTH_PASSES), key=timed)
    ms = min(t["ms"] for t in table if all(t.get(k, DEFAULTS.get(k)) == best[k] for k in KNOBS))
    out = dict({k: best[k] for k in KNOBS}, ms=ms, table=table)
    if use_cache:
        cache[key] = out
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".tmp%d" % os.getpid()
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, CACHE)
    return out
