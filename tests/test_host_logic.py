"""Host-side planning logic (CPU only): key widths and digit plans of the
sorts, the choice of view-major tile keys, the skip thresholds of the
diagnostics and the view partition across ranks."""
import numpy as np
import pytest

from paper_2604_18980_gb300 import diagnostics as D
from paper_2604_18980_gb300 import render as R
from paper_2604_18980_gb300.multiview import shard_views


def test_key_widths():
    assert R.tile_key_bits(1, 1) == 1
    assert R.tile_key_bits(10, 8160) == 17            # 1080p, 10 views
    assert R.tile_key_bits(8, 62208) == 19            # 4608x3456, 8 views
    assert R.tile_key_bits(16, 45800) == 20           # 3660x3200, 16 views
    assert R.key_end_bit(10, 8160) == 49
    cam = dict(width=1920, height=1080)
    assert R.tiles_per_view(cam) == 120 * 68


@pytest.mark.parametrize("bits", range(1, 41))
@pytest.mark.parametrize("max_digit", [4, 7, 8, 9])
def test_digit_plan_covers_the_bits(bits, max_digit):
    passes, digit = R.digit_plan(bits, max_digit)
    assert passes * digit >= bits                     # every key bit is sorted
    assert (passes - 1) * digit < bits or passes == 1  # no empty pass
    assert 4 <= digit <= max(4, max_digit)
    assert passes == max(1, -(-bits // max_digit))    # the fewest passes


def test_view_major_rule_on_the_workloads():
    assert R.view_major_default(10, 8160, 9)              # C2: two 7/6-bit passes instead of 9/8
    assert R.view_major_default(8, 62208, 8)              # C3: two passes instead of three
    assert R.view_major_default(16, 45800, 9)             # C4: two passes instead of three
    assert not R.view_major_default(1, 256, 8)            # a single view has nothing to regroup
    for V in range(2, 33):
        for T in (1, 2, 17, 256, 8160, 45800, 62208):
            tb = max(1, (T - 1).bit_length())
            assert tb <= R.tile_key_bits(V, T)         # the tile bits never exceed the full key


def test_skip_thresholds_from_histogram():
    h = np.zeros(32768, dtype=np.int64)
    h[100] = 10
    h[200] = 30
    h[300] = 60
    assert D.Diagnostics.threshold_for(h, 0.0) == 0.0
    t = D.Diagnostics.threshold_for(h, 0.4)           # a bin edge with 40% of the blends below it
    b = int(np.float32(t).view(np.uint32) >> 16)
    assert h[:b].sum() == 40 and 200 < b <= 300
    assert D.bin_lower_edge(300) == float(np.array([300 << 16], dtype=np.uint32).view(np.float32)[0])
    assert D.Diagnostics.threshold_for(np.zeros(32768, dtype=np.int64), 0.5) == 0.0


def test_shard_views_balanced():
    for n in (1, 7, 10, 16):
        for world in (1, 2, 3, 8):
            parts = [shard_views(list(range(n)), r, world) for r in range(world)]
            assert sum(parts, []) == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
