"""Comparison helpers between the CUDA path (through the C ABI) and the oracle."""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

import oracle
from paper_2604_18980_gb300 import binding as B
from paper_2604_18980_gb300 import render as R

IMG_TOL = 2e-3          # max-abs per channel outside edge-flagged pixels
PSNR_MIN = 60.0         # dB, over all pixels
EDGE_REL = 1e-5         # relative width of the oracle's edge classes

# Ceilings on what the edge classes exclude from the exact comparisons.
# Gaussians: each of the four ends of a footprint rectangle lies within
# +-1e-5 * scale of the pixel boundary that decides its tile with probability
# 2e-5 * scale / 16, the scale (|fx x/z| + |cx|) at most about the image
# extent, so rectangle edges flag about 0.5e-5 (W + H) of the live Gaussians;
# 0.2% on top covers the radius ceil, the opacity cull and the LUT bins.
# Pixels and tiles depend on the scene's density; each test states its own
# ceiling (default below), set at about 1.5x the fraction its configuration
# realises, so that a widened class fails the test.
FLAGGED_PX_MAX = 0.0075  # pixels with a near-threshold alpha decision
EDGE_TILES_MAX = 0.02    # compared tiles whose lists differ through edge Gaussians


def edge_gauss_ceiling(W, H):
    return 0.5 * EDGE_REL * (W + H) + 0.002


def report(kind, **kw):
    """Append one realised exclusion figure to $AGS_PARITY_REPORT (JSON lines), if set."""
    path = os.environ.get("AGS_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(kind=kind, test=os.environ.get("PYTEST_CURRENT_TEST", ""), **kw)) + "\n")


def gpu_render(scene_np, cams, scale_mode=0, K=0.0, lut=None, bg=(0.0, 0.0, 0.0), sh_degree=3, capacity=None,
               digit_bits=8, want_stats=False, tile_test=0, **knobs):
    scene = R.scene_to_device(scene_np)
    r = R.Renderer(scene, cams, scale_mode, K, lut, sh_degree, bg, capacity=capacity, digit_bits=digit_bits,
                   want_stats=want_stats, tile_test=tile_test, **knobs)
    r.forward()
    r.check()
    return r


def oracle_params(cam, scale_mode=0, K=0.0, lut=None, bg=(0.0, 0.0, 0.0), sh_degree=3, tile_test=0):
    lut32 = None if lut is None else np.asarray(lut, dtype=np.float32).astype(np.float64)
    return oracle.params(cam, scale_mode=scale_mode, K=float(np.float32(K)), lut=lut32, sh_degree=sh_degree,
                         bg=tuple(float(np.float32(b)) for b in bg), tau=float(np.float32(1.0 / 255.0)),
                         t_min=float(np.float32(1e-4)), alpha_max=float(np.float32(0.99)), tile_test=tile_test)


def gpu_features(r, view=0):
    n = r.n
    sp = r.proj["splat"].view(r.V, n, 12)[view].cpu().numpy()
    rect = r.proj["rect"].view(r.V, n, 4)[view].cpu().numpy().view(np.uint16).astype(np.int64)
    flags = r.proj["flags"].view(r.V, n)[view].cpu().numpy()
    depth = r.proj["depth"].view(r.V, n)[view].cpu().numpy()
    return sp, rect, flags, depth


def compare_features(r, orc_out, view=0, max_edge=None):
    """Per-Gaussian parity: survivors, rectangles and features.

    Discrete outcomes (survival, rectangle, tile count) are compared bit for
    bit outside the oracle's edge classes; an edge-class Gaussian live on both
    sides may differ by one tile at each end of its rectangle.  The continuous
    features are compared for every Gaussian live on both sides, edge classes
    included.  The edge Gaussians may be at most `max_edge` (default: the
    rectangle-edge estimate for this image size) of the live ones.  Returns counts."""
    sp, rect, flags, depth = gpu_features(r, view)
    dbl, irec = orc_out["dbl"], orc_out["irec"]
    edge = irec[:, oracle.I_EDGE] != 0
    o_live = irec[:, oracle.I_TOUCHED] > 0
    g_live = (flags & 0x80) == 0
    mism = (o_live != g_live) & ~edge
    assert not mism.any(), "survivor mismatch outside edge classes: %s" % np.nonzero(mism)[0][:10]
    live = o_live | g_live
    n_edge = int((edge & live).sum())
    ceiling = edge_gauss_ceiling(r.W, r.H) if max_edge is None else max_edge
    report("edge_gaussians", view=view, edge=n_edge, live=int(live.sum()), ceiling=ceiling,
           bits={b: int(((irec[live, oracle.I_EDGE] & v) != 0).sum()) for b, v in
                 (("near", 1), ("det", 2), ("th", 4), ("ceil", 8), ("rect", 16), ("lut", 32), ("ellipse", 64))})
    assert n_edge <= ceiling * max(int(live.sum()), 1) + 2, "edge classes hold %d of %d live Gaussians (ceiling %.4f)" % (
        n_edge, int(live.sum()), ceiling)
    both_all = o_live & g_live
    both = both_all & ~edge
    o_rect = irec[:, [oracle.I_X0, oracle.I_Y0, oracle.I_X1, oracle.I_Y1]].astype(np.int64)
    bad = both & np.any(o_rect != rect, axis=1)
    assert not bad.any(), "rect mismatch: %s" % np.nonzero(bad)[0][:10]
    bad = both_all & edge & np.any(np.abs(o_rect - rect) > 1, axis=1)
    assert not bad.any(), "edge-class rect off by more than one tile: %s" % np.nonzero(bad)[0][:10]
    touched = r.proj["tiles_touched"].view(r.V, r.n)[view].cpu().numpy().astype(np.int64)
    bad = both & (touched != irec[:, oracle.I_TOUCHED])
    assert not bad.any(), "tile count mismatch: %s" % np.nonzero(bad)[0][:10]
    both = both_all
    W = r.W
    du = np.abs(sp[both, 0] - dbl[both, oracle.F_U])
    dv = np.abs(sp[both, 1] - dbl[both, oracle.F_V])
    assert np.all(du <= 1e-5 * (np.abs(dbl[both, oracle.F_U]) + W)), du.max()
    assert np.all(dv <= 1e-5 * (np.abs(dbl[both, oracle.F_V]) + W)), dv.max()
    for gi, oi in ((2, oracle.F_A), (3, oracle.F_B), (4, oracle.F_C)):
        scale = np.abs(dbl[both, oracle.F_A]) + np.abs(dbl[both, oracle.F_C])
        err = np.abs(sp[both, gi] - dbl[both, oi])
        assert np.all(err <= 2e-5 * scale), (gi, (err / scale).max())
    np.testing.assert_allclose(sp[both, 5], dbl[both, oracle.F_OPAC], rtol=2e-6, atol=1e-7)
    for gi, oi in ((6, oracle.F_R), (7, oracle.F_G), (8, oracle.F_BL)):
        np.testing.assert_allclose(sp[both, gi], dbl[both, oi], rtol=1e-5, atol=2e-6)
    np.testing.assert_allclose(depth[both], dbl[both, oracle.F_DEPTH], rtol=1e-6)
    th = dbl[both, oracle.F_TH]
    np.testing.assert_allclose(sp[both, 9], th, rtol=1e-4)
    return dict(live=int(o_live.sum()), edge=n_edge, compared=int(both.sum()))


def gpu_pairs(r):
    """Sorted pairs as 64-bit (tile | depth) keys and values, rebuilt from the
    sorted values, the tile ranges and the per-splat depths (the renderer keeps
    no sorted keys), in the order of the range index view * T + tile (view-major
    keys group the array by tile, then view).  Checks on the way that the
    non-empty ranges partition [0, pairs)."""
    npairs = r.pairs()
    vals = r.sorted_vals[:npairs].cpu().numpy().view(np.uint32).astype(np.int64)
    rg = r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    length = rg[:, 1] - rg[:, 0]
    assert np.all(length >= 0)
    full = np.nonzero(length > 0)[0]
    starts, lens = rg[full, 0], length[full]
    by_start = np.argsort(starts, kind="stable")
    s_sorted, e_sorted = starts[by_start], starts[by_start] + lens[by_start]
    assert npairs == 0 or (s_sorted[0] == 0 and e_sorted[-1] == npairs), "ranges do not cover the pairs"
    assert np.array_equal(s_sorted[1:], e_sorted[:-1]), "ranges overlap or leave gaps"
    excl = np.cumsum(lens) - lens
    idx = np.arange(int(lens.sum()), dtype=np.int64) + np.repeat(starts - excl, lens)
    vals = vals[idx]
    tile = np.repeat(full, lens).astype(np.uint64)
    dbits = r.proj["depth"].cpu().numpy().view(np.uint32)[vals].astype(np.uint64)
    return (tile << np.uint64(32)) | dbits, vals


def compare_lists(r, orc_outs, tile_masks=None, max_edge_tiles=EDGE_TILES_MAX):
    """Per-tile sorted id lists: bit-exact outside edge-flagged Gaussians and depth near-ties.

    orc_outs: one oracle render dict per view (None to skip a view).
    tile_masks: optional per-view boolean masks of the tiles to compare (the
    oracle built lists for those tiles only).  Returns (number of tiles whose
    order differs only by near-ties, per-view edge tiles)."""
    keys, vals = gpu_pairs(r)
    n, T = r.n, r.T
    g_tile = (keys >> np.uint64(32)).astype(np.int64)
    assert np.all(keys[1:] >= keys[:-1]), "keys not sorted"
    assert np.all(vals // n == g_tile // T), "view of pair and of tile disagree"
    g_depth_bits = (keys & np.uint64(0xffffffff)).astype(np.uint32)
    tie_tiles = 0
    edge_tiles = []
    for v, oo in enumerate(orc_outs):
        if oo is None:
            edge_tiles.append([])
            continue
        edge = oo["irec"][:, oracle.I_EDGE] != 0
        ts, ids = oo["tile_start"], oo["ids"]
        o_tile = np.repeat(np.arange(T), np.diff(ts))
        sel = (g_tile // T) == v
        if tile_masks is not None:
            sel &= np.asarray(tile_masks[v], dtype=bool)[np.clip(g_tile - v * T, 0, T - 1)]
        gt, gi, gd = g_tile[sel] - v * T, vals[sel] - v * n, g_depth_bits[sel]
        # tiles whose lists differ only through edge-class Gaussians (excluded from image parity)
        eo = set(zip(o_tile[edge[ids]].tolist(), ids[edge[ids]].tolist()))
        eg = set(zip(gt[edge[gi]].tolist(), gi[edge[gi]].tolist()))
        edge_tiles.append(sorted({t for t, _ in eo ^ eg}))
        ncmp = int(np.asarray(tile_masks[v], dtype=bool).sum()) if tile_masks is not None else T
        report("edge_tiles", view=v, edge_tiles=len(edge_tiles[-1]), compared=ncmp, ceiling=max_edge_tiles)
        assert len(edge_tiles[-1]) <= max_edge_tiles * ncmp + 1, "%d of %d tiles differ through edge Gaussians" % (
            len(edge_tiles[-1]), ncmp)
        keep_o = ~edge[ids]
        o_tile, o_ids = o_tile[keep_o], ids[keep_o].astype(np.int64)
        keep_g = ~edge[gi]
        gt, gi, gd = gt[keep_g], gi[keep_g], gd[keep_g]
        assert len(gt) == len(o_tile), "pair count differs outside edge classes: gpu %d oracle %d" % (
            len(gt), len(o_tile))
        np.testing.assert_array_equal(gt, o_tile)
        # depth keys: exactly the fp32 depth (within 1 ulp of the oracle's rounding)
        od = oo["dbl"][gi, oracle.F_DEPTH].astype(np.float32).view(np.uint32).astype(np.int64)
        assert np.all(np.abs(gd.astype(np.int64) - od) <= 1), "depth key off by more than 1 ulp"
        if not np.array_equal(gi, o_ids):
            # allowed only between near-ties: same multiset per tile and oracle depths within 4 ulps
            diff_tiles = np.unique(gt[gi != o_ids])
            for t in diff_tiles:
                a = gi[gt == t]
                b = o_ids[o_tile == t]
                assert np.array_equal(np.sort(a), np.sort(b)), "tile %d holds different Gaussians" % t
                da = oo["dbl"][a, oracle.F_DEPTH].astype(np.float32).view(np.int32).astype(np.int64)
                bad = np.nonzero(a != b)[0]
                for k in bad:
                    j = np.nonzero(b == a[k])[0][0]
                    lo, hi = min(k, j), max(k, j)
                    span = da[lo:hi + 1]
                    assert span.max() - span.min() <= 4, "order differs beyond a depth near-tie in tile %d" % t
                tie_tiles += 1
    return tie_tiles, edge_tiles


def tile_pixel_mask(tile_mask, W, H):
    """Pixel mask [H][W] of the selected tiles."""
    gx = (W + 15) // 16
    m = np.zeros((H, W), dtype=bool)
    for t in np.nonzero(tile_mask)[0]:
        ty, tx = divmod(int(t), gx)
        m[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    return m


def compare_image(img_gpu, oo, tol=IMG_TOL, edge_tiles=(), pixel_mask=None, max_flagged=FLAGGED_PX_MAX):
    """Image parity: max-abs <= tol outside edge-flagged pixels; PSNR over all pixels.

    Edge pixels: a near-threshold alpha decision (oracle flip budget > 0; such
    a pixel must still be within tol + its budget, and they may be at most
    `max_flagged` of the compared pixels), or a tile whose pair list differs
    through an edge-class Gaussian (bounded by compare_lists)."""
    o = oo["image"]
    g = np.asarray(img_gpu, dtype=np.float64)
    H, W = o.shape[1:]
    flagged = oo["budget"] > 0
    tile_px = np.zeros((H, W), dtype=bool)
    gx = (W + 15) // 16
    for t in edge_tiles:
        ty, tx = divmod(int(t), gx)
        tile_px[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    flagged_budget = flagged & ~tile_px
    flagged = flagged | tile_px
    if pixel_mask is not None:
        o = o[:, pixel_mask]
        g = g[:, pixel_mask]
        flagged, flagged_budget = flagged[pixel_mask], flagged_budget[pixel_mask]
        budget = oo["budget"][pixel_mask]
    else:
        budget = oo["budget"]
    n_budget = int((budget > 0).sum())
    report("flagged_pixels", flagged=n_budget, compared=int(budget.size), edge_tile_px=int(tile_px.sum()),
           ceiling=max_flagged)
    assert n_budget <= max_flagged * budget.size + 2, "%d of %d pixels carry a flip budget" % (n_budget, budget.size)
    err = np.abs(g - o).max(axis=0)
    ok = err[~flagged]
    assert ok.size == 0 or ok.max() <= tol, "max abs error %.3g outside edge pixels" % ok.max()
    assert np.all(err[flagged_budget] <= tol + budget[flagged_budget]), "edge pixel beyond its flip bound"
    mse = float(np.mean((g - o) ** 2))
    psnr = math.inf if mse == 0 else 10 * math.log10(1.0 / mse)
    assert psnr >= PSNR_MIN, psnr
    return dict(max_err=float(ok.max()) if ok.size else 0.0, flagged=int(flagged.sum()),
                edge_tile_px=int(tile_px.sum()), psnr=psnr)


GRAD_KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def gradient_edge_gaussians(oo: dict, og: dict):
    """Gaussians whose derivative can jump under a one-rounding change of the
    inputs: an edge class of the preprocess (their pair lists may differ), a
    gradient-only clamp decision (frustum, colour) near its threshold, or a
    pixel decision of the blend (alpha vs tau, alpha vs its clamp, the stop)
    within its band."""
    return (oo["irec"][:, oracle.I_EDGE] != 0) | (oo["irec"][:, oracle.I_GEDGE] != 0) | (og["edge"] > 0)


GRAD_EDGE_MAX = 0.2      # ceiling on the Gaussians set aside by the elementwise check (C5 realises 12.8%)


def compare_gradients(g_gpu: dict, g_orc: dict, skip=None, rel_l2=1e-3, rel_elem=1e-3, big=1e-2,
                      max_skip=GRAD_EDGE_MAX):
    """Gradients: per-tensor relative L2 <= rel_l2, and elementwise
    |gpu - oracle| <= rel_elem |oracle| + budget on the entries with |g| >=
    big * max|g|, the budget being the oracle's bound on what near-threshold
    decisions of other Gaussians at shared pixels can change in that entry
    (zero where there are none).  `skip` (optional bool [n], see
    gradient_edge_gaussians) sets aside the Gaussians whose own derivative can
    jump under one rounding; they may be at most `max_skip` of the Gaussians
    with a gradient."""
    out = {}
    if skip is not None:
        has = np.abs(g_orc["opacity_logit"]) > 0
        n_skip = int((np.asarray(skip, bool) & has).sum())
        report("gradient_edges", skipped=n_skip, with_gradient=int(has.sum()), ceiling=max_skip)
        assert n_skip <= max_skip * max(int(has.sum()), 1) + 2, "%d of %d Gaussians set aside" % (
            n_skip, int(has.sum()))
    for k in GRAD_KEYS:
        a = g_gpu[k].cpu().numpy().astype(np.float64).reshape(g_orc[k].shape)
        b = g_orc[k]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        sel = np.abs(b) >= big * np.abs(b).max()
        if skip is not None:
            sel &= ~np.broadcast_to(np.asarray(skip, bool), b.shape)
        bud = g_orc["budget"][k] if "budget" in g_orc else np.zeros_like(b)
        # error over the allowance rel_elem |b| + budget (<= 1 passes)
        er = (np.abs(a[sel] - b[sel]) / (rel_elem * np.abs(b[sel]) + bud[sel])) if sel.any() else np.zeros(1)
        rr = np.abs(a[sel] - b[sel]) / np.abs(b[sel]) if sel.any() else np.zeros(1)
        bq = bud[sel] / np.abs(b[sel]) if sel.any() else np.zeros(1)
        report("gradients", key=k, rel_l2=float(rel), max_elem_rel=float(rr.max()), max_over_allowance=float(er.max()),
               entries=int(sel.sum()), over_rel=int((rr > rel_elem).sum()), with_budget=int((bud[sel] > 0).sum()),
               budget_rel_median=float(np.median(bq)), budget_rel_p99=float(np.percentile(bq, 99)))
        out[k] = (float(rel), float(er.max()), int(sel.sum()))
    for k, (rel, emax, cnt) in out.items():
        assert rel <= rel_l2, (k, rel)
        assert emax <= 1.0, ("elementwise", k, emax, cnt)
    return out
