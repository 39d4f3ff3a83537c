"""The C-ABI library loads and exports every entry point include/ags.h declares,
and rejects invalid arguments on the host (no GPU needed: these paths return
before any CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_2604_18980_gb300 import binding as B
from paper_2604_18980_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ags.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return B.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ags_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_pipeline():
    names = declared_functions()
    for n in ("ags_preprocess", "ags_emit_pairs", "ags_emit_tile_pairs", "ags_sort", "ags_sort32",
              "ags_rasterize", "ags_rasterize_backward", "ags_calibrate_lut", "ags_check", "ags_status_reset",
              "ags_peripheral_scores", "ags_contribution_hist", "ags_render_skip"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in B.EXPORTS, "binding lacks %s" % name


def test_struct_layouts_match_header(lib):
    # sizes implied by the header's field lists (all 4- or 8-byte fields)
    assert ctypes.sizeof(B.AgsCamera) == 4 * (2 + 4 + 12 + 3 + 1)
    assert ctypes.sizeof(B.AgsParams) == 4 * (3 + 5 + 32 + 3 + 2)
    assert ctypes.sizeof(B.AgsGaussians) == 8 * 6
    assert ctypes.sizeof(B.AgsProjected) == 8 * 6


def test_status_strings_and_version(lib):
    assert B.ags_status_string(0) == "ok"
    assert "capacity" in B.ags_status_string(2)
    assert B.ags_status_string(B.AGS_ERR_BOUNDS) == B.STATUS_NAMES[B.AGS_ERR_BOUNDS]
    assert "sm_103a" in B.ags_version()


def test_workspace_sizes(lib):
    assert B.ags_emit_workspace_bytes(0, 1) == 256
    assert B.ags_emit_workspace_bytes(1024, 1) == 256 + 8
    assert B.ags_emit_workspace_bytes(1025, 1) == 256 + 16
    assert B.ags_sort_workspace_bytes(4096) == 256 + 16 * 512 * 4 + 1 * 512 * 4
    assert B.ags_sort_workspace_bytes(4097) == 256 + 16 * 512 * 4 + 2 * 512 * 4
    assert B.ags_backward_workspace_bytes(10, 2) == 10 * 2 * 9 * 4
    assert B.ags_compact_workspace_bytes(4096, 1) == 256 + (8 + 2 * 256) * 1       # header, count, masks per partition
    chunks = 4 * ((B.AGS_MAX_PAIRS + 2047) // 2048 + 1)
    assert B.ags_emit_tile_workspace_bytes(1024, 1) == 256 + 16 + 16 * 1024 + chunks
    assert B.ags_emit_tile_workspace_bytes(1025, 2) == 256 + 32 + 16 * 2050 + chunks
    assert B.ags_compact_workspace_bytes(4097, 2) == 256 + (8 + 2 * 256) * 3


def test_invalid_arguments_rejected_on_host(lib):
    L = lib
    cam = B.cameras([dict(width=64, height=48, fx=50.0, fy=50.0, cx=31.5, cy=23.5,
                          viewmat=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], campos=[0, 0, 0])])
    par = B.params()
    g = B.AgsGaussians()
    g.n = -1
    pr = B.AgsProjected()
    st = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    # negative n
    assert L.ags_preprocess(ctypes.byref(g), cam, 1, ctypes.byref(par), ctypes.byref(pr), st, None) == 1
    # zero / too many views
    g.n = 10
    assert L.ags_preprocess(ctypes.byref(g), cam, 0, ctypes.byref(par), ctypes.byref(pr), st, None) == 1
    assert L.ags_preprocess(ctypes.byref(g), cam, B.AGS_MAX_VIEWS + 1, ctypes.byref(par), ctypes.byref(pr), st,
                            None) == 1
    # bad parameters
    bad = B.params(sh_degree=4)
    assert L.ags_preprocess(ctypes.byref(g), cam, 1, ctypes.byref(bad), ctypes.byref(pr), st, None) == 1
    bad = B.params(K=-1.0)
    assert L.ags_preprocess(ctypes.byref(g), cam, 1, ctypes.byref(bad), ctypes.byref(pr), st, None) == 1
    bad = B.params(scale_mode=2)
    assert L.ags_preprocess(ctypes.byref(g), cam, 1, ctypes.byref(bad), ctypes.byref(pr), st, None) == 1
    bad = B.params(tile_test=2)
    assert L.ags_preprocess(ctypes.byref(g), cam, 1, ctypes.byref(bad), ctypes.byref(pr), st, None) == 1
    bad = B.params(blend_flags=4)      # a launch-shape bit the blend does not know
    assert L.ags_preprocess(ctypes.byref(g), cam, 1, ctypes.byref(bad), ctypes.byref(pr), st, None) == 1
    assert L.ags_rasterize(ctypes.byref(pr), 0, None, ctypes.c_void_p(256), cam, 1, ctypes.byref(bad),
                           ctypes.c_void_p(512), None, None, None, None, st, None) == 1
    # null outputs
    assert L.ags_preprocess(ctypes.byref(g), cam, 1, ctypes.byref(par), ctypes.byref(pr), st, None) == 1
    # sort: bad digit width, capacity beyond the limit, missing workspace
    npairs = ctypes.c_void_p(16)
    alt = ctypes.c_int32(0)
    assert L.ags_sort(None, None, None, None, npairs, 10, 0, 40, 10, 0, None, 0, ctypes.byref(alt), st, None, 0,
                      None) == 1
    assert L.ags_sort(None, None, None, None, npairs, B.AGS_MAX_PAIRS, 0, 40, 8, 0, None, 0, ctypes.byref(alt), st,
                      None, 0, None) == 1
    assert L.ags_sort(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), npairs,
                      10, 0, 40, 8, 0, None, 0, ctypes.byref(alt), st, None, 0, None) == 1
    assert L.ags_sort(None, None, None, None, npairs, 10, 0, 40, 8, 32, None, 0, ctypes.byref(alt), st, None, 0,
                      None) == 1
    # 32-bit sort: end bit beyond the key, unknown flag, unaligned keys
    assert L.ags_sort32(None, None, None, None, npairs, 10, 0, 33, 8, 0, None, 0, ctypes.byref(alt), st, None, 0,
                        None) == 1
    assert L.ags_sort32(None, None, None, None, npairs, 10, 0, 32, 8, 32, None, 0, ctypes.byref(alt), st, None, 0,
                        None) == 1
    assert L.ags_sort32(ctypes.c_void_p(20), ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), npairs,
                        10, 0, 32, 8, 0, None, 0, ctypes.byref(alt), st, ctypes.c_void_p(256), 1 << 20, None) == 1
    # ranges not 8-byte aligned
    assert L.ags_sort32(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), npairs,
                        10, 0, 32, 8, 0, ctypes.c_void_p(260), 4, ctypes.byref(alt), st, ctypes.c_void_p(256),
                        1 << 20, None) == 1
    assert L.ags_rasterize(ctypes.byref(pr), 0, None, ctypes.c_void_p(260), cam, 1, ctypes.byref(par),
                           ctypes.c_void_p(512), None, None, None, None, st, None) == 1
    # 64-bit sort: unaligned keys
    assert L.ags_sort(ctypes.c_void_p(24), ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), npairs,
                      10, 0, 40, 8, 0, None, 0, ctypes.byref(alt), st, ctypes.c_void_p(256), 1 << 20, None) == 1
    # emit: workspace too small
    assert L.ags_emit_pairs(ctypes.byref(pr), 10, 1, cam, None, None, None, 0, npairs, st, 0, None, 0, None) == 1
    # the ellipse flag needs the splat records and tile counts
    assert L.ags_emit_pairs(ctypes.byref(pr), 10, 1, cam, None, None, None, 0, npairs, st, 2, ctypes.c_void_p(256),
                            1 << 20, None) == 1
    assert L.ags_emit_pairs(ctypes.byref(pr), 10, 1, cam, None, None, None, 0, npairs, st, 4, ctypes.c_void_p(256),
                            1 << 20, None) == 1
    assert L.ags_emit_tile_pairs(ctypes.byref(pr), 10, 1, cam, None, None, None, None, 0, npairs, st, 0, None, 0,
                                 None) == 1
    # views * n beyond 32 bits (or wrapping int64) is rejected before the product is formed
    cam2 = B.cameras([dict(width=64, height=48, fx=50.0, fy=50.0, cx=31.5, cy=23.5,
                           viewmat=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], campos=[0, 0, 0])] * 2)
    for big in (1 << 31, (1 << 62) + 1):
        assert L.ags_emit_pairs(ctypes.byref(pr), big, 2, cam2, None, None, None, 0, npairs, st, 0,
                                ctypes.c_void_p(256), 1 << 40, None) == 1
        assert L.ags_emit_tile_pairs(ctypes.byref(pr), big, 2, cam2, None, None, None, None, 0, npairs, st, 0,
                                     ctypes.c_void_p(256), 1 << 40, None) == 1
        assert L.ags_emit_pairs_noalloc(ctypes.byref(pr), big, 2, cam2, None, None, None, 0, npairs, st, None) == 1
        assert B.ags_emit_workspace_bytes(big, 2) == 0
        assert B.ags_emit_tile_workspace_bytes(big, 2) == 0
    # the allocation-free emission: one more Gaussian-view than its scratch holds, over two views
    limit = int(L.ags_emit_pairs_noalloc_max_gaussians())
    assert L.ags_emit_pairs_noalloc(ctypes.byref(pr), limit // 2 + 1, 2, cam2, None, None, None, 0, npairs, st,
                                    None) == 1
    # unknown emission flag
    assert L.ags_emit_pairs(ctypes.byref(pr), 10, 1, cam, None, None, None, 0, npairs, st, 1 << 12,
                            ctypes.c_void_p(256), 1 << 20, None) == 1
    # compaction: zero views, missing workspace, unaligned flags
    assert L.ags_compact_visible(ctypes.byref(pr), 10, 0, None, None, npairs, st, None, 0, None) == 1
    pr2 = B.AgsProjected()
    pr2.flags, pr2.depth = ctypes.c_void_p(17), ctypes.c_void_p(32)
    assert L.ags_compact_visible(ctypes.byref(pr2), 10, 1, ctypes.c_void_p(16), ctypes.c_void_p(16), npairs, st,
                                 ctypes.c_void_p(256), 1 << 20, None) == 1
    assert L.ags_compact_visible(ctypes.byref(pr), 10, 1, ctypes.c_void_p(16), ctypes.c_void_p(16), npairs, st,
                                 None, 0, None) == 1
    # mismatched view sizes
    cams2 = B.cameras([dict(width=64, height=48, fx=50.0, fy=50.0, cx=31.5, cy=23.5,
                            viewmat=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], campos=[0, 0, 0]),
                       dict(width=65, height=48, fx=50.0, fy=50.0, cx=31.5, cy=23.5,
                            viewmat=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], campos=[0, 0, 0])])
    assert L.ags_rasterize(ctypes.byref(pr), 10, None, ctypes.c_void_p(16), cams2, 2, ctypes.byref(par),
                           ctypes.c_void_p(16), None, None, None, None, st, None) == 1
    # LUT: too many bins
    assert L.ags_calibrate_lut(None, None, 0, 33, 100.0, ctypes.c_void_p(16), None) == 1
    # view-major tile sort: no tile bits, more tiles than the bits hold, key overflow; view keys without n
    assert L.ags_sort_tiles(None, None, None, None, npairs, 0, 0, 8, 0, None, 2, 1, ctypes.byref(alt), st, None, 0,
                            None) == 1
    assert L.ags_sort_tiles(None, None, None, None, npairs, 0, 4, 8, 0, None, 2, 17, ctypes.byref(alt), st, None, 0,
                            None) == 1
    assert L.ags_sort_tiles(None, None, None, None, npairs, 0, 30, 8, 0, None, 5, 17, ctypes.byref(alt), st, None,
                            0, None) == 1
    assert L.ags_view_keys(ctypes.c_void_p(16), npairs, 10, 0, ctypes.c_void_p(16), None) == 1
    # diagnostics: missing outputs or inputs, unknown ranking, rule 1 without weights, negative threshold
    cam1 = B.cameras([dict(width=64, height=48, fx=50.0, fy=50.0, cx=31.5, cy=23.5,
                           viewmat=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], campos=[0, 0, 0])])
    full = B.AgsProjected()
    full.splat, full.depth, full.flags = ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.c_void_p(768)
    rg, sv = ctypes.c_void_p(1024), ctypes.c_void_p(2048)
    assert L.ags_peripheral_scores(ctypes.byref(full), 10, sv, rg, cam1, 1, ctypes.byref(par), None, None) == 1
    assert L.ags_peripheral_scores(ctypes.byref(pr), 10, sv, rg, cam1, 1, ctypes.byref(par),
                                   ctypes.c_void_p(4096), None) == 1
    assert L.ags_contribution_hist(ctypes.byref(full), 10, sv, rg, cam1, 1, ctypes.byref(par), 3, None,
                                   ctypes.c_void_p(4096), None) == 1
    assert L.ags_contribution_hist(ctypes.byref(full), 10, sv, rg, cam1, 1, ctypes.byref(par), 1, None,
                                   ctypes.c_void_p(4096), None) == 1
    assert L.ags_render_skip(ctypes.byref(full), 10, sv, rg, cam1, 1, ctypes.byref(par), 0, None, -1.0,
                             ctypes.c_void_p(4096), ctypes.c_void_p(8192), None) == 1
    assert L.ags_render_skip(ctypes.byref(full), 10, sv, rg, cam1, 1, ctypes.byref(par), 0, None, 0.5,
                             None, ctypes.c_void_p(8192), None) == 1


def test_debug_library_builds_and_exports_every_symbol():
    """libags_debug.so (-DAGS_DEBUG): the same C ABI, and a version string that says so."""
    from paper_2604_18980_gb300 import build as cuda_build
    path = cuda_build.build(debug=True, quiet=True)
    assert path != cuda_build.LIB
    L = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name), name
    L.ags_version.restype = ctypes.c_char_p
    assert b"AGS_DEBUG" in L.ags_version()
    assert "AGS_DEBUG" not in B.ags_version()
