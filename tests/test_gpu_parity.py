"""CUDA path (through the C ABI) against the FP64 oracle, element by element."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import (GRAD_KEYS, compare_features, compare_gradients, compare_image, compare_lists, gpu_pairs,
                         gpu_render, gradient_edge_gaussians, oracle_params)
from paper_2604_18980_gb300 import binding as B
from paper_2604_18980_gb300 import calibrate as C
from paper_2604_18980_gb300 import render as R
from paper_2604_18980_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_18980_gb300 import build
    build.build()
    B.lib()


def _c1(n=16384, W=256, H=256, views=1):
    scene, cams, calib = synth.workload("c1_cube16k_256", n=n, width=W, height=H, views=views)
    return scene, cams


def _full_check(scene, cams, mode, K, lut=None, bg=(0.0, 0.0, 0.0), tile_test=0, **knobs):
    r = gpu_render(scene, cams, mode, K, lut, bg, tile_test=tile_test, **knobs)
    outs, stats = [], []
    for v, cam in enumerate(cams):
        par = oracle_params(cam, mode, K, lut, bg, tile_test=tile_test)
        oo = oracle.render(scene, cam, par)
        outs.append(oo)
        stats.append(compare_features(r, oo, v))
    ties, edge_tiles = compare_lists(r, outs)
    for v, oo in enumerate(outs):
        stats.append(compare_image(r.image[v].cpu().numpy(), oo, edge_tiles=edge_tiles[v]))
    return r, outs, stats, ties


@pytest.mark.parametrize("mode,K", [(0, 0.0), (1, 0.0), (1, 0.3), (1, 3.0)])
def test_c1_parity(mode, K):
    scene, cams = _c1()
    lut = np.linspace(1.0, 0.4, 20).astype(np.float32)
    r, outs, stats, ties = _full_check(scene, cams, mode, K, lut)
    assert r.pairs() > 0


@pytest.mark.parametrize("mode,K,knobs", [(0, 0.0, {}), (1, 0.3, {}), (1, 0.3, dict(presort=False)),
                                          (1, 3.0, dict(emit_two_pass=False))])
def test_c1_parity_ellipse_tiles(mode, K, knobs):
    """The ellipse tile test: per-Gaussian kept-tile counts, per-tile lists and
    images against the oracle's exact per-tile minimum, on every emission path."""
    scene, cams = _c1(n=12000, W=256, H=200, views=2)
    lut = np.linspace(1.0, 0.4, 20).astype(np.float32)
    r, outs, stats, ties = _full_check(scene, cams, mode, K, lut, tile_test=B.AGS_TILE_ELLIPSE, **knobs)
    sq = gpu_render(scene, cams, mode, K, lut, tile_test=B.AGS_TILE_SQUARE, **knobs)
    assert 0 < r.pairs() < sq.pairs()


def test_plain_ellipse_tiles_render_the_square_image():
    """Plain mode: the ellipse test drops only tiles whose pixels all have
    alpha < tau, so the image is bit-identical with fewer pairs (ragged size,
    background)."""
    scene, cams = _c1(n=6000, W=173, H=94, views=2)
    a = gpu_render(scene, cams, 0, 0.0, bg=(0.1, 0.3, 0.7))
    b = gpu_render(scene, cams, 0, 0.0, bg=(0.1, 0.3, 0.7), tile_test=B.AGS_TILE_ELLIPSE)
    assert torch.equal(a.image, b.image)
    assert b.pairs() < a.pairs()
    ka, va = gpu_pairs(a)
    kb, vb = gpu_pairs(b)
    pa = set(zip((ka >> np.uint64(32)).tolist(), va.tolist()))
    pb = set(zip((kb >> np.uint64(32)).tolist(), vb.tolist()))
    assert pb <= pa


def test_ragged_sizes_and_background():
    # image not a multiple of the tile, n not a multiple of the block
    scene, cams = _c1(n=3001, W=173, H=94)
    _full_check(scene, cams, 1, 0.2, bg=(0.1, 0.3, 0.7))
    _full_check(scene, cams, 0, 0.0, bg=(0.1, 0.3, 0.7))


def test_batched_views_match_single_views():
    scene, cams = _c1(n=5000, W=128, H=96, views=3)
    rb = gpu_render(scene, cams, 1, 0.3)
    for v, cam in enumerate(cams):
        r1 = gpu_render(scene, [cam], 1, 0.3)
        np.testing.assert_array_equal(rb.image[v].cpu().numpy(), r1.image[0].cpu().numpy())
    _full_check(scene, cams, 1, 0.3)


def test_maximum_views_in_one_batch():
    """AGS_MAX_VIEWS views in one launch per stage (the most view bits in the
    keys) render each view exactly as it renders alone, with the default
    knobs and with 64-bit keys."""
    scene, cams = _c1(n=3000, W=72, H=40, views=B.AGS_MAX_VIEWS)
    for knobs in (dict(), dict(presort=False)):
        rb = gpu_render(scene, cams, 1, 0.3, **knobs)
        assert rb.V == B.AGS_MAX_VIEWS
        for v in (0, 1, 17, B.AGS_MAX_VIEWS - 1):
            r1 = gpu_render(scene, [cams[v]], 1, 0.3, **knobs)
            np.testing.assert_array_equal(rb.image[v].cpu().numpy(), r1.image[0].cpu().numpy())


@pytest.mark.parametrize("W,H", [(1, 1), (1, 40), (37, 1), (16, 16), (17, 17)])
def test_tiny_and_single_tile_images(W, H):
    """Images of one pixel, one column, one row, exactly one tile and one tile
    plus one pixel each way, against the oracle: features, pair lists and
    image exact outside the edge classes.  The ceilings on the edge classes'
    share are lifted: with a handful of pixels and live Gaussians a fraction
    says nothing."""
    scene, cams = _c1(n=2000, W=W, H=H, views=2)
    r = gpu_render(scene, cams, 1, 0.3)
    outs = [oracle.render(scene, cam, oracle_params(cam, 1, 0.3)) for cam in cams]
    for v, oo in enumerate(outs):
        compare_features(r, oo, v, max_edge=1.0)
    _, edge_tiles = compare_lists(r, outs, max_edge_tiles=1.0)
    for v, oo in enumerate(outs):
        compare_image(r.image[v].cpu().numpy(), oo, edge_tiles=edge_tiles[v], max_flagged=1.0)


def test_empty_and_all_culled():
    scene, cams = _c1(n=0, W=64, H=48)
    r = gpu_render(scene, cams, 0, 0.0, bg=(0.2, 0.4, 0.6), capacity=1024)
    img = r.image.cpu().numpy()
    np.testing.assert_array_equal(img[0, 0], np.full((48, 64), np.float32(0.2)))
    np.testing.assert_array_equal(img[0, 2], np.full((48, 64), np.float32(0.6)))
    scene, cams = _c1(n=500, W=64, H=48)
    scene["opacity_logit"][:] = -20.0           # opacity ~2e-9 < tau
    r = gpu_render(scene, cams, 1, 0.0, bg=(0.2, 0.4, 0.6), capacity=1024)
    assert r.pairs() == 0
    np.testing.assert_array_equal(r.image.cpu().numpy()[0, 1], np.full((48, 64), np.float32(0.4)))


def test_capacity_overflow_is_reported_and_bounded():
    scene, cams = _c1(n=4000, W=128, H=128)
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, 0, 0.0)
    need = r.pairs() if r.pairs() else r.count_pairs()
    cap = need // 2
    r.alloc_pairs(cap)
    guard = torch.full((4096,), -7, dtype=torch.int64, device="cuda")
    B.ags_status_reset(r.status)
    r.preprocess()
    # emit into a buffer followed by a guard region; nothing may land past capacity
    keys = torch.full((cap + 4096,), -7, dtype=torch.int64, device="cuda")
    vals = torch.full((cap + 4096,), -7, dtype=torch.int32, device="cuda")
    B.ags_emit_pairs(r.proj, r.n, r.cams, keys, vals, cap, r.num_pairs, r.status, r.ws_emit)
    code, detail = B.ags_check(r.status, raise_on_error=False)
    assert code == B.AGS_ERR_CAPACITY and detail == need
    assert int(r.num_pairs.item()) == need
    assert torch.all(keys[cap:] == -7) and torch.all(vals[cap:] == -7)
    del guard


@pytest.mark.parametrize("count,bits,digit,flags", [(1, 40, 8, 0), (4095, 40, 8, 4), (4097, 45, 8, 0),
                                                    (100003, 49, 8, 4), (250000, 52, 7, 0), (77777, 40, 5, 4),
                                                    (2049, 41, 9, 0), (300001, 49, 9, 4), (65536, 36, 9, 0)])
def test_sort_random_keys_stable(count, bits, digit, flags):
    rng = np.random.default_rng(count)
    tile_bits = bits - 32
    tiles = rng.integers(0, 1 << tile_bits, count, dtype=np.uint64)
    depth = rng.uniform(0.2, 30.0, count).astype(np.float32)
    depth[rng.random(count) < 0.2] = 1.5           # many exact ties: stability matters
    keys = (tiles << np.uint64(32)) | depth.view(np.uint32).astype(np.uint64)
    vals = np.arange(count, dtype=np.uint32)
    cap = count + 123
    k = torch.zeros(cap, dtype=torch.int64, device="cuda")
    v = torch.zeros(cap, dtype=torch.int32, device="cuda")
    k[:count] = torch.from_numpy(keys.view(np.int64)).cuda()
    v[:count] = torch.from_numpy(vals.view(np.int32)).cuda()
    ka, va = torch.zeros_like(k), torch.zeros_like(v)
    npairs = torch.tensor([count], dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    ws = torch.empty(B.ags_sort_workspace_bytes(cap), dtype=torch.uint8, device="cuda")
    nr = 1 << tile_bits
    ranges = torch.empty(2 * nr, dtype=torch.int32, device="cuda") if tile_bits <= 16 else None
    alt = B.ags_sort(k, v, ka, va, npairs, cap, 0, bits, digit, ranges, nr, st, ws, flags=flags)
    B.ags_check(st)
    ks = (ka if alt else k)[:count].cpu().numpy().view(np.uint64)
    vs = (va if alt else v)[:count].cpu().numpy().view(np.uint32)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(ks, keys[order])
    np.testing.assert_array_equal(vs, vals[order])
    if ranges is not None:
        rg = ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
        t = (keys[order] >> np.uint64(32)).astype(np.int64)
        starts = np.searchsorted(t, np.arange(nr), "left")
        ends = np.searchsorted(t, np.arange(nr), "right")
        empty = starts == ends
        np.testing.assert_array_equal(rg[~empty, 0], starts[~empty])
        np.testing.assert_array_equal(rg[~empty, 1], ends[~empty])
        assert np.all(rg[empty] == 0)


def test_calibration_lut_matches_oracle():
    scene, cams, calib = synth.workload("c1_cube16k_256", n=8000, width=128, height=128)
    sc = R.scene_to_device(scene)
    lut = C.calibrate_lut(sc, calib[:4], lut_bins=20, lut_depth_max=10.0)
    # oracle: max T per Gaussian per view, binned by its depth in that view
    exp = np.zeros(20)
    for cam in calib[:4]:
        par = oracle_params(cam)
        oo = oracle.render(scene, cam, par, want_max_T=True)
        mt = oo["max_T"]
        d = oo["dbl"][:, oracle.F_DEPTH]
        b = np.minimum(np.floor(d * 20 / 10.0), 19).astype(int)
        for i in np.nonzero(mt > 0)[0]:
            exp[b[i]] = max(exp[b[i]], mt[i])
    exp[exp == 0] = 1.0
    np.testing.assert_allclose(lut, exp, rtol=1e-4)


def test_backward_matches_oracle_gradients():
    scene, cam = synth.fd_subscene()
    scene["opacity_logit"][:4] = 5.5
    bg = (0.05, 0.1, 0.15)
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, [cam], 0, 0.0, bg=bg)
    r.forward()
    rng = np.random.default_rng(5)
    w = rng.normal(size=(3, cam["height"], cam["width"])).astype(np.float32)
    g = r.backward(torch.from_numpy(w).cuda()[None])
    r.check()
    par = oracle_params(cam, bg=bg)
    oo = oracle.render(scene, cam, par)
    og = oracle.backward(scene, cam, par, oo["tile_start"], oo["ids"], w.astype(np.float64))
    for k in ("mean", "log_scale", "quat", "opacity_logit", "sh"):
        a = g[k].cpu().numpy().astype(np.float64).reshape(og[k].shape)
        b = og[k]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel <= 1e-3, (k, rel)
        big = np.abs(b) >= 1e-2 * np.abs(b).max()
        np.testing.assert_allclose(a[big], b[big], rtol=1e-3, atol=0, err_msg=k)


def test_backward_c1_scale_and_views():
    scene, cams = _c1(n=4000, W=128, H=96, views=2)
    bg = (0.0, 0.0, 0.0)
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, 1, 0.2)
    r.forward()
    rng = np.random.default_rng(9)
    w = rng.normal(size=(2, 3, 96, 128)).astype(np.float32)
    g = r.backward(torch.from_numpy(w).cuda())
    r.check()
    tot, edge = None, None
    for v, cam in enumerate(cams):
        par = oracle_params(cam, 1, 0.2, bg=bg)
        oo = oracle.render(scene, cam, par)
        og = oracle.backward(scene, cam, par, oo["tile_start"], oo["ids"], w[v].astype(np.float64))
        if tot is None:
            tot = og
        else:     # gradients and their flip budgets add over views
            tot = dict({k: tot[k] + og[k] for k in GRAD_KEYS},
                       budget={k: tot["budget"][k] + og["budget"][k] for k in GRAD_KEYS})
        e = gradient_edge_gaussians(oo, og)
        edge = e if edge is None else edge | e
    compare_gradients(g, tot, skip=edge)


@pytest.mark.parametrize("knobs", [dict(view_major=False), dict(view_major=True),
                                   dict(view_major=True, emit_two_pass=False, digit_bits=5)])
def test_depth_presort_equals_full_key_sort(knobs):
    """Sorting the Gaussians by depth first and then only the tile digits of the
    pairs gives exactly the stable sort of the full (tile | depth) keys; so do
    view-major keys (the views one after the other in the emission order,
    sorted by the tile bits alone, the ranges indexed through the view bits)."""
    scene, cams = _c1(n=12000, W=200, H=150, views=3)
    sc = R.scene_to_device(scene)
    for mode, K in ((0, 0.0), (1, 0.5)):
        a = R.Renderer(sc, cams, mode, K, presort=True, **knobs)
        assert a.view_major == knobs["view_major"]
        b = R.Renderer(sc, cams, mode, K, presort=False)
        ia, ib = a.forward().clone(), b.forward().clone()
        a.check()
        b.check()
        assert a.pairs() == b.pairs()
        np_ = a.pairs()
        ka, va = gpu_pairs(a)
        kb, vb = gpu_pairs(b)
        np.testing.assert_array_equal(ka, kb)
        np.testing.assert_array_equal(va, vb)
        assert torch.equal(ia, ib)
        ra, rb = a.ranges.view(-1, 2), b.ranges.view(-1, 2)
        assert torch.equal(ra[:, 1] - ra[:, 0], rb[:, 1] - rb[:, 0])
        if not a.view_major:
            assert torch.equal(a.sorted_vals[:np_], b.sorted_vals[:np_])
            assert torch.equal(a.ranges, b.ranges)


def test_sort_identity_values_flag():
    rng = np.random.default_rng(3)
    count = 50000
    keys = rng.integers(0, 1 << 36, count, dtype=np.uint64)
    keys[::7] = keys[0]
    k = torch.from_numpy(keys.view(np.int64)).cuda()
    v = torch.full((count,), -1, dtype=torch.int32, device="cuda")
    ka, va = torch.zeros_like(k), torch.zeros_like(v)
    n = torch.tensor([count], dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    ws = torch.empty(B.ags_sort_workspace_bytes(count), dtype=torch.uint8, device="cuda")
    alt = B.ags_sort(k, v, ka, va, n, count, 0, 36, 6, None, 0, st, ws, flags=B.AGS_SORT_IDENTITY_VALUES)
    B.ags_check(st)
    vs = (va if alt else v).cpu().numpy()
    np.testing.assert_array_equal(vs, np.argsort(keys, kind="stable"))


@pytest.mark.parametrize("count,views,tiles,digit,flags", [(1, 2, 5, 4, 0), (50000, 3, 130, 8, 2),
                                                          (123457, 16, 45800, 8, 6), (70001, 10, 8160, 7, 6)])
def test_sort_tiles_view_shifted_keys(count, views, tiles, digit, flags):
    """ags_sort_tiles: stable by the tile bits alone, the view bits above them
    untouched; ranges indexed by view * tiles + tile.  ags_view_keys: order // n."""
    rng = np.random.default_rng(count + views)
    tb = max(1, (tiles - 1).bit_length())
    view = np.sort(rng.integers(0, views, count)).astype(np.uint64)   # emitted view by view
    tile = rng.integers(0, tiles, count).astype(np.uint64)
    tile[rng.random(count) < 0.3] = tile[0]
    keys = ((view << np.uint64(tb)) | tile).astype(np.uint32)
    vals = rng.permutation(count).astype(np.uint32)
    cap = count + 5
    k = torch.zeros(cap, dtype=torch.int32, device="cuda")
    k[:count] = torch.from_numpy(keys.view(np.int32))
    v = torch.zeros(cap, dtype=torch.int32, device="cuda")
    v[:count] = torch.from_numpy(vals.view(np.int32))
    ka, va = torch.zeros_like(k), torch.zeros_like(v)
    n = torch.tensor([count], dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    ws = torch.empty(B.ags_sort_workspace_bytes(cap), dtype=torch.uint8, device="cuda")
    rg = torch.full((views * tiles * 2,), -1, dtype=torch.int32, device="cuda")
    alt = B.ags_sort_tiles(k, v, ka, va, n, cap, tb, digit, rg, views, tiles, st, ws, flags=flags)
    B.ags_check(st)
    order = np.argsort(tile, kind="stable")
    got_v = (va if alt else v)[:count].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got_v, vals[order])
    if not (flags & B.AGS_SORT_DISCARD_KEYS):
        np.testing.assert_array_equal((ka if alt else k)[:count].cpu().numpy().view(np.uint32), keys[order])
    ranges = rg.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    r_idx = (view * np.uint64(tiles) + tile)[order].astype(np.int64)
    exp = np.zeros((views * tiles, 2), dtype=np.int64)
    first = np.ones(count, dtype=bool)
    first[1:] = r_idx[1:] != r_idx[:-1]
    last = np.ones(count, dtype=bool)
    last[:-1] = r_idx[1:] != r_idx[:-1]
    pos = np.arange(count)
    exp[r_idx[first], 0] = pos[first]
    exp[r_idx[last], 1] = pos[last] + 1
    np.testing.assert_array_equal(ranges, exp)
    # the view of each entry of an order over views * n entries
    nn = 1000
    order_e = torch.from_numpy(rng.permutation(views * nn).astype(np.int32)).cuda()
    vk = torch.full((views * nn,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.tensor([views * nn - 3], dtype=torch.int64, device="cuda")
    B.ags_view_keys(order_e, cnt, views * nn, nn, vk)
    got = vk.cpu().numpy()
    np.testing.assert_array_equal(got[:views * nn - 3], order_e.cpu().numpy()[:views * nn - 3] // nn)
    assert np.all(got[views * nn - 3:] == -1)


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("rank_or", [False, True])
@pytest.mark.parametrize("count,bits,digit,flags", [(1, 12, 8, 0), (4095, 13, 8, 2), (4097, 17, 9, 0),
                                                    (100003, 17, 9, 2), (250000, 20, 7, 1), (77777, 16, 5, 3),
                                                    (300001, 32, 8, 3), (65536, 32, 9, 0)])
def test_sort32_random_keys_stable(count, bits, digit, flags, rank_or, persistent):
    """32-bit keys: the stable order, the ranges of the whole key, the identity
    values flag, the discarded-keys flag, both ranking methods and the
    persistent passes (with a capacity six times the count, their use)."""
    if rank_or:
        flags |= B.AGS_SORT_RANK_OR
    if persistent:
        flags |= B.AGS_SORT_PERSISTENT
    rng = np.random.default_rng(count + bits)
    keys = rng.integers(0, 1 << bits, count, dtype=np.uint64).astype(np.uint32)
    keys[rng.random(count) < 0.3] = keys[0]          # long runs of equal keys: stability matters
    vals = rng.permutation(count).astype(np.uint32)
    cap = count * (6 if persistent else 1) + 77
    k = torch.zeros(cap, dtype=torch.int32, device="cuda")
    v = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    k[:count] = torch.from_numpy(keys.view(np.int32)).cuda()
    if not flags & B.AGS_SORT_IDENTITY_VALUES:
        v[:count] = torch.from_numpy(vals.view(np.int32)).cuda()
    else:
        vals = np.arange(count, dtype=np.uint32)
    ka, va = torch.zeros_like(k), torch.zeros_like(v)
    npairs = torch.tensor([count], dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    ws = torch.empty(B.ags_sort_workspace_bytes(cap), dtype=torch.uint8, device="cuda")
    nr = 1 << bits if bits <= 17 else 0
    ranges = torch.empty(2 * nr, dtype=torch.int32, device="cuda") if nr else None
    kout_before = (k.clone(), ka.clone())
    alt = B.ags_sort32(k, v, ka, va, npairs, cap, 0, bits, digit, ranges, nr, st, ws, flags=flags)
    B.ags_check(st)
    order = np.argsort(keys, kind="stable")
    vs = (va if alt else v)[:count].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(vs, vals[order])
    if not flags & B.AGS_SORT_DISCARD_KEYS:
        ks = (ka if alt else k)[:count].cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(ks, keys[order])
    else:
        # the last pass wrote no keys: the result's key buffer still holds what
        # the previous pass (or the caller) left there
        passes = -(-bits // digit)
        if passes == 1:
            assert torch.equal((ka if alt else k), kout_before[1 if alt else 0])
    # nothing written past the count
    assert torch.all(va[count:] == 0) and torch.all(v[count:] == -1)
    if ranges is not None:
        rg = ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
        t = keys[order].astype(np.int64)
        starts = np.searchsorted(t, np.arange(nr), "left")
        ends = np.searchsorted(t, np.arange(nr), "right")
        empty = starts == ends
        np.testing.assert_array_equal(rg[~empty, 0], starts[~empty])
        np.testing.assert_array_equal(rg[~empty, 1], ends[~empty])
        assert np.all(rg[empty] == 0)


def test_emit_tile_pairs_matches_emit_pairs():
    """32-bit tile keys in the depth order of the compacted visible views: the
    tile word of the 64-bit keys emitted in that order, same values, same count;
    the order holds every visible view once, each view by depth then index."""
    scene, cams = _c1(n=9000, W=176, H=144, views=3)
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, 1, 0.3, presort=True)
    r.preprocess()
    r.depth_sort()
    r.check()
    nvis = int(r.n_visible.item())
    flags = r.proj["flags"].cpu().numpy()
    visible = np.nonzero((flags & 0x80) == 0)[0]
    assert nvis == len(visible) and 0 < nvis < r.V * r.n
    o = r.emit_order[:nvis].cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(np.sort(o), visible)
    dk = r.proj["depth"].cpu().numpy().view(np.uint32)[o]
    v_of = o // r.n
    for v in range(len(cams)):
        sel = v_of == v
        ov, dv = o[sel], dk[sel].astype(np.int64)
        assert np.all(np.diff(dv) >= 0)
        ties = np.nonzero(np.diff(dv) == 0)[0]
        assert np.all(ov[ties + 1] > ov[ties])
    # pairs: 64-bit emission over the same order (a full-length copy whose tail
    # lists the culled views, which emit nothing) against the tile-key emission
    full = torch.from_numpy(np.concatenate([o, np.setdiff1d(np.arange(r.V * r.n), visible)]).astype(np.int32)).cuda()
    cap = r.capacity
    k64 = torch.empty(cap, dtype=torch.int64, device="cuda")
    v64 = torch.empty(cap, dtype=torch.int32, device="cuda")
    k32 = torch.empty(cap, dtype=torch.int32, device="cuda")
    v32 = torch.empty(cap, dtype=torch.int32, device="cuda")
    n64 = torch.zeros(1, dtype=torch.int64, device="cuda")
    n32 = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.ags_emit_pairs(r.proj, r.n, cams, k64, v64, cap, n64, r.status, r.ws_emit, order=full)
    B.ags_emit_tile_pairs(r.proj, r.n, cams, k32, v32, cap, n32, r.status, r.ws_emit, order=r.emit_order,
                          order_count=r.n_visible)
    r.check()
    P = int(n64.item())
    assert P == int(n32.item()) and P > 0
    hi = (k64[:P].cpu().numpy().view(np.uint64) >> np.uint64(32)).astype(np.uint32)
    np.testing.assert_array_equal(k32[:P].cpu().numpy().view(np.uint32), hi)
    assert torch.equal(v32[:P], v64[:P])


def test_emit_tile_pairs_balanced_blocks():
    """The two-pass tile-key emission over orders with culled entries (no pairs)
    and with Gaussians whose pairs span many 1024-pair blocks: identical to the
    64-bit emission's tile words and values."""
    scene, cams = _c1(n=6000, W=1280, H=960, views=2)
    scene["log_scale"][:, :40] = -0.3            # a few Gaussians covering thousands of tiles
    scene["mean"][:, -300:] = np.nan             # culled: entries without pairs
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, 0, 0.0, presort=True)
    r.preprocess()
    cap = r.capacity
    for order, flags in ((None, 0), (torch.randperm(r.V * r.n, device="cuda").to(torch.int32), 0),
                         (None, B.AGS_EMIT_SINGLE_PASS)):
        k64 = torch.empty(cap, dtype=torch.int64, device="cuda")
        v64 = torch.empty(cap, dtype=torch.int32, device="cuda")
        k32 = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        v32 = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        n64 = torch.zeros(1, dtype=torch.int64, device="cuda")
        n32 = torch.zeros(1, dtype=torch.int64, device="cuda")
        B.ags_emit_pairs(r.proj, r.n, cams, k64, v64, cap, n64, r.status, r.ws_emit, order=order)
        B.ags_emit_tile_pairs(r.proj, r.n, cams, k32, v32, cap, n32, r.status, r.ws_emit, order=order, flags=flags)
        r.check()
        P = int(n64.item())
        assert P == int(n32.item()) and P > 4096
        touched = r.proj["tiles_touched"].cpu().numpy()
        assert touched.max() > 2 * 2048 and (touched == 0).any()
        hi = (k64[:P].cpu().numpy().view(np.uint64) >> np.uint64(32)).astype(np.uint32)
        np.testing.assert_array_equal(k32[:P].cpu().numpy().view(np.uint32), hi)
        assert torch.equal(v32[:P], v64[:P])
        assert torch.all(k32[P:] == -1)


def test_emit_tile_pairs_long_runs_of_empty_entries():
    """An order with a run of thousands of entries without pairs in its middle:
    the pair block that straddles the run spans more records than one staged
    window, so the second pass must look the next window up.  Identical to the
    64-bit emission's tile words and values."""
    scene, cams = _c1(n=6000, W=640, H=480, views=2)
    scene["mean"][:, 1000:5000] = np.nan            # 4000 Gaussians culled in both views
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, 0, 0.0, presort=True)
    r.preprocess()
    touched = r.proj["tiles_touched"]
    e_all = torch.arange(r.V * r.n, device="cuda")
    vis, empty = e_all[touched > 0], e_all[touched == 0]
    assert len(empty) > 3 * 2049
    half = len(vis) // 2
    order = torch.cat([vis[:half], empty, vis[half:]]).to(torch.int32)
    cap = r.capacity
    for flags in (0, B.AGS_EMIT_SINGLE_PASS):
        k64 = torch.empty(cap, dtype=torch.int64, device="cuda")
        v64 = torch.empty(cap, dtype=torch.int32, device="cuda")
        k32 = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        v32 = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        n64 = torch.zeros(1, dtype=torch.int64, device="cuda")
        n32 = torch.zeros(1, dtype=torch.int64, device="cuda")
        B.ags_emit_pairs(r.proj, r.n, cams, k64, v64, cap, n64, r.status, r.ws_emit, order=order)
        B.ags_emit_tile_pairs(r.proj, r.n, cams, k32, v32, cap, n32, r.status, r.ws_emit, order=order, flags=flags)
        r.check()
        P = int(n64.item())
        assert P == int(n32.item()) and P > 2 * 2048
        hi = (k64[:P].cpu().numpy().view(np.uint64) >> np.uint64(32)).astype(np.uint32)
        np.testing.assert_array_equal(k32[:P].cpu().numpy().view(np.uint32), hi)
        assert torch.equal(v32[:P], v64[:P])
        assert torch.all(k32[P:] == -1)


def test_compact_visible_edges():
    """Compaction of ragged counts (not a multiple of the partition), all-culled
    and none-culled inputs, and more partitions than one chunk of the offset
    scan (16384), against numpy."""
    for total, p_cull in ((1, 0.0), (4095, 0.5), (4097, 0.3), (3 * 4096 + 17, 1.0), (70001, 0.0), (70001, 0.9),
                          ((1 << 26) + 3 * 4096 + 5, 0.85)):
        rng = np.random.default_rng(total + int(10 * p_cull))
        flags = np.where(rng.random(total) < p_cull, 0x80, rng.integers(0, 0x20, total)).astype(np.uint8)
        depth = rng.uniform(0.2, 50.0, total).astype(np.float32)
        proj = dict(splat=None, depth=torch.from_numpy(depth).cuda(), rect=None, flags=torch.from_numpy(flags).cuda())
        keys = torch.full((total,), -1, dtype=torch.int32, device="cuda")
        ids = torch.full((total,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(4, dtype=torch.int64, device="cuda")
        ws = torch.empty(B.ags_compact_workspace_bytes(total, 1), dtype=torch.uint8, device="cuda")
        B.ags_compact_visible(proj, total, 1, keys, ids, cnt, st, ws)
        B.ags_check(st)
        vis = np.nonzero((flags & 0x80) == 0)[0]
        assert int(cnt.item()) == len(vis)
        np.testing.assert_array_equal(ids[:len(vis)].cpu().numpy(), vis)
        np.testing.assert_array_equal(keys[:len(vis)].cpu().numpy().view(np.uint32), depth.view(np.uint32)[vis])
        assert torch.all(ids[len(vis):] == -1)


def test_cuda_graph_replay_matches_eager_and_follows_scene_updates():
    scene, cams = _c1(n=6000, W=160, H=120, views=2)
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, 1, 0.4)
    eager = r.forward().clone()
    r.check()
    g = r.capture()
    r.image.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(r.image, eager)
    # the graph reads the scene buffers: an in-place update is rendered on replay
    sc["opacity_logit"].add_(0.5)
    sc["mean"][0].add_(0.01)
    g.replay()
    torch.cuda.synchronize()
    replayed = r.image.clone()
    r2 = R.Renderer(sc, cams, 1, 0.4, capacity=r.capacity)
    assert torch.equal(replayed, r2.forward())
    r.check()


def test_autotuner_candidates_render_identically():
    from paper_2604_18980_gb300 import autotune
    scene, cams = _c1(n=8000, W=192, H=144, views=2)
    sc = R.scene_to_device(scene)
    imgs, lists = [], []
    for cand in autotune.CANDIDATES:
        r = R.Renderer(sc, cams, 1, 0.3, **cand)
        imgs.append(r.forward().clone())
        r.check()
        lists.append(gpu_pairs(r))                       # per-tile lists in range order
    for im, (k, v) in zip(imgs[1:], lists[1:]):
        assert torch.equal(im, imgs[0])
        np.testing.assert_array_equal(k, lists[0][0])
        np.testing.assert_array_equal(v, lists[0][1])
    best = autotune.tune(sc, cams, 1, 0.3, use_cache=False, warmup=1, reps=2)
    assert best["digit_bits"] in (7, 8, 9)
    assert len(best["table"]) == (len(autotune.CANDIDATES) + len(autotune.SHAPES)
                                  + (len(autotune.DEPTH_PASSES) if best["presort"] else 0))
    assert all(k in best for k in autotune.KNOBS)


@pytest.mark.parametrize("digit_bits", [8, 9])
def test_launch_shapes_give_identical_outputs(digit_bits):
    """The block shapes the autotuner sweeps -- the blend's 8x16 or 8x8 warp
    blocks and 32- or 64-splat batches, the 32-bit sort passes on 256 x 16 or
    512 x 8 partitions -- and the depth pre-sort's ranking method change no output: image, final T, last blended
    position, calibration max T, the evaluation and blend counts, and the
    sorted pair lists, bit for bit.  A ragged frame (tiles cut at the right and
    bottom edges), two views, and tiles long enough for several batches."""
    from paper_2604_18980_gb300 import autotune
    scene, cams = _c1(n=12000, W=200, H=150, views=2)
    sc = R.scene_to_device(scene)
    ref = None
    for sh in autotune.SHAPES + [dict(depth_rank_or=False), dict(depth_persistent=False)]:
        r = R.Renderer(sc, cams, 1, 0.3, want_stats=True, digit_bits=digit_bits, **sh)
        max_T = torch.zeros(r.V * r.n, dtype=torch.float32, device="cuda")
        img = r.forward(max_T=max_T).clone()
        r.check()
        out = dict(img=img, T=r.final_T.clone(), nc=r.n_contrib.clone(), maxT=max_T, st=r.stats[:2].clone(),
                   lists=gpu_pairs(r))
        if ref is None:
            ref = out
            rg = r.ranges.view(-1, 2).long()
            assert int(ref["st"][0]) > 0 and int((rg[:, 1] - rg[:, 0]).max()) > 2 * 64   # several batches a tile
            continue
        for k in ("img", "T", "nc", "maxT", "st"):
            assert torch.equal(out[k], ref[k]), (sh, k)
        np.testing.assert_array_equal(out["lists"][0], ref["lists"][0])
        np.testing.assert_array_equal(out["lists"][1], ref["lists"][1])


@pytest.mark.parametrize("mode,K", [(0, 0.0), (1, 0.3)])
def test_blend_counters_match_oracle(mode, K):
    """stats[0]: Eq. 1-2 evaluations (per pixel, its tile's pairs up to the one it
    stopped at); stats[1]: blends.  Both against the oracle's per-pixel counts;
    a pixel with a near-threshold decision (flip budget > 0) may move by its
    tile's list length (evaluations) or its blend count (blends)."""
    scene, cams = _c1(n=6000, W=173, H=94, views=1)
    lut = np.linspace(1.0, 0.4, 20).astype(np.float32)
    r = gpu_render(scene, cams, mode, K, lut, want_stats=True)
    ev, bl = int(r.stats[0].item()), int(r.stats[1].item())
    par = oracle_params(cams[0], mode, K, lut)
    oo = oracle.render(scene, cams[0], par, want_state=True)
    st = oo["state"]
    W, H = cams[0]["width"], cams[0]["height"]
    gx = (W + 15) // 16
    lens = np.diff(oo["tile_start"])
    yy, xx = np.mgrid[0:H, 0:W]
    px_len = lens[(yy // 16) * gx + (xx // 16)]
    flagged = oo["budget"] > 0
    ev_o, bl_o = int(st[..., 2].sum()), int(st[..., 0].sum())
    assert ev_o > bl_o > 0
    assert abs(ev - ev_o) <= int(px_len[flagged].sum()), (ev, ev_o)
    assert abs(bl - bl_o) <= int(px_len[flagged].sum()), (bl, bl_o)
    if not flagged.any():
        assert (ev, bl) == (ev_o, bl_o)


@pytest.mark.parametrize("knobs", [dict(), dict(emit_two_pass=False), dict(presort=False),
                                   dict(tile_test=B.AGS_TILE_ELLIPSE), dict(view_major=False)])
def test_launches_per_forward_counts_the_kernels(knobs):
    """Renderer.launches_per_forward(), the bench line's gpu_launches per step,
    equals the kernels one forward launches (counted by the profiler; memsets
    are not kernels)."""
    from torch.profiler import ProfilerActivity, profile
    scene, cams = _c1(n=6000, W=160, H=120, views=2)
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, 1, 0.3, keep_state=False, **knobs)
    r.forward()
    r.check()
    with profile(activities=[ProfilerActivity.CUDA]):     # the profiler's own first-use set-up
        r.forward()
        torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        r.forward()
        torch.cuda.synchronize()
    names = [e.name for e in prof.events() if e.device_type.name == "CUDA"]
    kernels = [nm for nm in names if not nm.lower().startswith(("memset", "memcpy"))]
    if not kernels:
        pytest.skip("the profiler recorded no kernels on this box")
    assert len(kernels) == r.launches_per_forward(), kernels
