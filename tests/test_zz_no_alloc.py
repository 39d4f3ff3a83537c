"""The allocation-free emission entry point against the workspace one.

ags_emit_pairs_noalloc serves callers that cannot allocate device memory (a
host application that owns a fixed device-memory budget and forbids its
plugins to allocate, or a caller from a language without a CUDA allocator
binding).  It must produce exactly what ags_emit_pairs produces with a caller
workspace, call after call, although every call reuses the same library-owned
scratch array.
"""
import ctypes

import pytest
import torch

from paper_2604_18980_gb300 import binding as B
from paper_2604_18980_gb300 import render as R
from paper_2604_18980_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _noalloc(L, r, order, keys, vals, cap, npairs, status):
    pr = B.projected(r.proj)
    cs = B.cameras(r.cams)
    return L.ags_emit_pairs_noalloc(ctypes.byref(pr), r.n, len(r.cams), cs, B.ptr(order), B.ptr(keys), B.ptr(vals),
                                    cap, B.ptr(npairs), B.ptr(status), B.stream_handle())


def test_noalloc_emit_matches_workspace_emit_twice():
    from paper_2604_18980_gb300 import build
    build.build()
    L = B.lib()
    scene, cams, _ = synth.workload("c1_cube16k_256", n=20000, width=200, height=150, views=2)
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, B.AGS_SCALE_ADAGSCALE, 0.3)
    r.preprocess()
    r.depth_sort()
    # a full permutation of the Gaussian-views: the depth order of the visible
    # ones (the renderer's compacted order), then the culled ones
    nvis = int(r.n_visible.item())
    culled = torch.nonzero((r.proj["flags"] & 0x80) != 0).flatten().to(torch.int32)
    order_full = torch.cat([r.emit_order[:nvis], culled]).contiguous()
    assert order_full.numel() == r.V * r.n
    cap = r.capacity
    keys_ref = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    vals_ref = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    np_ref = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    B.ags_emit_pairs(r.proj, r.n, r.cams, keys_ref, vals_ref, cap, np_ref, st, r.ws_emit, order=order_full)
    B.ags_check(st)
    n_ref = int(np_ref.item())
    assert n_ref > 0
    # the workspace call in Gaussian-id order (no `order`), the other reference
    keys_id = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    vals_id = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    st.zero_()
    B.ags_emit_pairs(r.proj, r.n, r.cams, keys_id, vals_id, cap, np_ref, st, r.ws_emit)
    B.ags_check(st)
    assert int(np_ref.item()) == n_ref
    for order in (order_full, None, order_full):   # several calls in a row share the scratch array
        keys = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        vals = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
        st.zero_()
        assert _noalloc(L, r, order, keys, vals, cap, npairs, st) == B.AGS_OK
        B.ags_check(st)
        assert int(npairs.item()) == n_ref
        ek, ev = (keys_id, vals_id) if order is None else (keys_ref, vals_ref)
        assert torch.equal(keys[:n_ref], ek[:n_ref])
        assert torch.equal(vals[:n_ref], ev[:n_ref])


def test_noalloc_emit_rejects_sizes_beyond_its_scratch():
    from paper_2604_18980_gb300 import build
    build.build()
    L = B.lib()
    limit = int(L.ags_emit_pairs_noalloc_max_gaussians())
    assert limit > 0
    scene, cams, _ = synth.workload("c1_cube16k_256", n=64, width=32, height=32, views=1)
    sc = R.scene_to_device(scene)
    r = R.Renderer(sc, cams, B.AGS_SCALE_PLAIN, capacity=1024)
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
    pr = B.projected(r.proj)
    cs = B.cameras(r.cams)
    code = L.ags_emit_pairs_noalloc(ctypes.byref(pr), limit + 1, 1, cs, None, B.ptr(r.keys), B.ptr(r.vals), 1024,
                                    B.ptr(npairs), B.ptr(st), B.stream_handle())
    assert code == B.AGS_ERR_INVALID_ARG


def test_noalloc_emit_takes_exactly_its_limit_over_two_views():
    """2 views of limit/2 Gaussians fill the whole static scratch (every
    look-back partition in use): accepted; all culled, so no pairs.  One more
    Gaussian per view is rejected."""
    from paper_2604_18980_gb300 import build
    build.build()
    L = B.lib()
    limit = int(L.ags_emit_pairs_noalloc_max_gaussians())
    n = limit // 2
    _, cams, _ = synth.workload("c1_cube16k_256", n=64, width=64, height=48, views=2)
    proj = dict(splat=torch.zeros(16, dtype=torch.float32, device="cuda"),
                depth=torch.zeros(limit, dtype=torch.float32, device="cuda"),
                rect=torch.zeros(4 * limit, dtype=torch.int16, device="cuda"),       # empty rectangles
                tiles_touched=torch.zeros(limit, dtype=torch.int32, device="cuda"),
                flags=torch.full((limit,), 0x80, dtype=torch.uint8, device="cuda"))
    npairs = torch.full((1,), -5, dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    pr = B.projected(proj)
    cs = B.cameras(cams)
    code = L.ags_emit_pairs_noalloc(ctypes.byref(pr), n, 2, cs, None, None, None, 0, B.ptr(npairs), B.ptr(st),
                                    B.stream_handle())
    assert code == B.AGS_OK
    B.ags_check(st)
    assert int(npairs.item()) == 0
    code = L.ags_emit_pairs_noalloc(ctypes.byref(pr), n + 1, 2, cs, None, None, None, 0, B.ptr(npairs), B.ptr(st),
                                    B.stream_handle())
    assert code == B.AGS_ERR_INVALID_ARG
