"""The autotuner's staged search on the host: a fake renderer whose forward
time is a known function of its launch knobs stands in for the GPU, so the
rounds, the choice and the cache can be checked without one."""
import json

import numpy as np
import pytest

from paper_2604_18980_gb300 import autotune
from paper_2604_18980_gb300 import binding as B


def _cost(knobs):
    """A separable cost with a unique minimum: digit 8, pre-sort on, OR
    ranking, two-pass emission, 8x8 warp blocks, narrow sort blocks, the
    persistent depth passes off."""
    c = {9: 0.3, 8: 0.0, 7: 0.5}[knobs["digit_bits"]]
    c += 0.0 if knobs["presort"] else 2.0
    c += 0.0 if knobs["pair_rank_or"] else 0.2
    c += 0.0 if knobs.get("emit_two_pass", True) else 0.1
    c += {0: 0.4, B.AGS_BLEND_ROWS2: 0.0, B.AGS_BLEND_BATCH64: 0.6,
          B.AGS_BLEND_ROWS2 | B.AGS_BLEND_BATCH64: 0.7}[knobs.get("blend_flags", 0)]
    c += 0.25 if knobs.get("sort_wide", False) else 0.0
    c += 0.05 if knobs.get("depth_persistent", True) else 0.0
    return 10.0 + c


class _FakeRenderer:
    def __init__(self, scene, cams, scale_mode, K, lut, capacity=None, keep_state=False, **knobs):
        self.knobs = knobs
        self.capacity = capacity or 1000


@pytest.fixture
def fake(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune.R, "Renderer", _FakeRenderer)
    monkeypatch.setattr(autotune, "_time_forward", lambda r, warmup, reps: _cost(r.knobs))
    monkeypatch.setattr(autotune, "workload_key", lambda scene, cams, mode: "fake|%d" % len(cams))
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    scene = dict(opacity_logit=np.zeros(10, dtype=np.float32))
    cams = [dict(width=64, height=48)]
    return scene, cams


def test_rounds_find_the_separable_minimum(fake):
    scene, cams = fake
    best = autotune.tune(scene, cams, use_cache=False)
    assert {k: best[k] for k in autotune.KNOBS} == dict(
        digit_bits=8, presort=True, pair_rank_or=True, emit_two_pass=True, blend_flags=B.AGS_BLEND_ROWS2,
        sort_wide=False, depth_persistent=False)
    # every candidate of the first round, then every shape, then the depth grids
    table = best["table"]
    assert len(table) == len(autotune.CANDIDATES) + len(autotune.SHAPES) + len(autotune.DEPTH_PASSES)
    assert best["ms"] == pytest.approx(min(t["ms"] for t in table))
    # the shape and depth rounds keep the first round's stage knobs
    for t in table[len(autotune.CANDIDATES):]:
        assert (t["digit_bits"], t["presort"], t["pair_rank_or"]) == (8, True, True)


def test_no_depth_round_without_the_presort(fake, monkeypatch):
    scene, cams = fake
    monkeypatch.setattr(autotune, "_time_forward",
                        lambda r, warmup, reps: _cost(r.knobs) - (3.0 if not r.knobs["presort"] else 0.0))
    best = autotune.tune(scene, cams, use_cache=False)
    assert best["presort"] is False
    assert len(best["table"]) == len(autotune.CANDIDATES) + len(autotune.SHAPES)


def test_cache_is_written_and_reused(fake, monkeypatch):
    scene, cams = fake
    first = autotune.tune(scene, cams)
    stored = json.load(open(autotune.CACHE))
    assert stored["fake|1"]["blend_flags"] == first["blend_flags"]
    monkeypatch.setattr(autotune, "_time_forward", lambda r, warmup, reps: pytest.fail("re-timed a cached workload"))
    again = autotune.tune(scene, cams)
    assert {k: again[k] for k in autotune.KNOBS} == {k: first[k] for k in autotune.KNOBS}


def test_an_entry_missing_a_knob_is_tuned_again(fake):
    scene, cams = fake
    json.dump({"fake|1": dict(digit_bits=9, presort=True, pair_rank_or=True, ms=1.0)}, open(autotune.CACHE, "w"))
    best = autotune.tune(scene, cams)
    assert all(k in best for k in autotune.KNOBS) and best["digit_bits"] == 8
