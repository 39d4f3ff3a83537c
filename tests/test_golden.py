"""The oracle's defaults against the constants the paper prints."""
import os

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def _read():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, value = line.split()[:2]
        vals[name] = float(value)
    return vals


def test_paper_constants():
    g = _read()
    assert abs(oracle.TAU - g["tau"]) < 1e-17
    assert oracle.T_MIN == g["t_min"]
    assert oracle.LUT_BINS == g["lut_bins"]
    assert oracle.LUT_DEPTH_MAX == g["lut_depth_max"]
    p = oracle.params(None)
    assert p.tau == oracle.TAU and p.t_min == oracle.T_MIN and p.lut_bins == 20 and p.lut_depth_max == 100.0
