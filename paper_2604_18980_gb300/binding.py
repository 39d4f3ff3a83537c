"""ctypes binding of libags (include/ags.h): the same entry points, argument
marshalling only.  Every computation happens in the CUDA library; this module
converts torch tensors and Python camera/parameter descriptions into the C
structures and raises ``AgsError`` on a non-zero status.

The library must have been built (``paper_2604_18980_gb300.build.build()`` or
``__graft_entry__.build()``); nothing here falls back to another
implementation when it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

AGS_TILE = 16
AGS_MAX_VIEWS = 32
AGS_MAX_LUT_BINS = 32
AGS_MAX_PAIRS = 1 << 30
AGS_SCALE_PLAIN, AGS_SCALE_ADAGSCALE = 0, 1
AGS_TILE_SQUARE, AGS_TILE_ELLIPSE = 0, 1
AGS_BLEND_ROWS2, AGS_BLEND_BATCH64 = 1, 2     # ags_params.blend_flags (launch shape of the blend)
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "pair capacity exceeded", 3: "bounded device wait timed out",
                4: "CUDA error", 5: "non-finite Gaussian parameters culled",
                6: "index out of range (debug build check)"}
AGS_OK, AGS_ERR_INVALID_ARG, AGS_ERR_CAPACITY, AGS_ERR_TIMEOUT, AGS_ERR_CUDA, AGS_ERR_NUMERIC, AGS_ERR_BOUNDS = range(7)
# check ids of AGS_ERR_BOUNDS (debug builds)
AGS_CHECK_BLEND_RANGE, AGS_CHECK_BLEND_VALUE, AGS_CHECK_BACKWARD_RANGE, AGS_CHECK_BACKWARD_VALUE, \
    AGS_CHECK_EMIT_ORDER = 1, 2, 3, 4, 5

_P = ctypes.c_void_p
_F = ctypes.c_float
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


class AgsError(RuntimeError):
    def __init__(self, code: int, where: str, detail: int | None = None):
        self.code = int(code)
        self.detail = detail
        msg = "%s: %s" % (where, STATUS_NAMES.get(self.code, "status %d" % self.code))
        if detail is not None:
            msg += " (detail %d)" % detail
        super().__init__(msg)


class AgsCamera(ctypes.Structure):
    _fields_ = [("width", _I32), ("height", _I32), ("fx", _F), ("fy", _F), ("cx", _F), ("cy", _F),
                ("viewmat", _F * 12), ("campos", _F * 3), ("near_z", _F)]


class AgsParams(ctypes.Structure):
    _fields_ = [("scale_mode", _I32), ("sh_degree", _I32), ("lut_bins", _I32), ("K", _F), ("tau", _F),
                ("t_min", _F), ("alpha_max", _F), ("lut_depth_max", _F), ("lut", _F * AGS_MAX_LUT_BINS),
                ("bg", _F * 3), ("tile_test", _I32), ("blend_flags", _I32)]


class AgsGaussians(ctypes.Structure):
    _fields_ = [("mean", _P), ("log_scale", _P), ("quat", _P), ("opacity_logit", _P), ("sh", _P), ("n", _I64)]


class AgsProjected(ctypes.Structure):
    _fields_ = [("splat", _P), ("depth", _P), ("rect", _P), ("tiles_touched", _P), ("flags", _P),
                ("depth_key", _P)]


EXPORTS = {
    "ags_status_reset": ([_P, _P], _I32),
    "ags_check": ([_P, _P, _P], _I32),
    "ags_status_string": ([_I32], ctypes.c_char_p),
    "ags_preprocess": ([_P, _P, _I32, _P, _P, _P, _P], _I32),
    "ags_emit_workspace_bytes": ([_I64, _I32], ctypes.c_size_t),
    "ags_emit_pairs": ([_P, _I64, _I32, _P, _P, _P, _P, _I64, _P, _P, _I32, _P, ctypes.c_size_t, _P], _I32),
    "ags_emit_tile_pairs": ([_P, _I64, _I32, _P, _P, _P, _P, _P, _I64, _P, _P, _I32, _P, ctypes.c_size_t, _P],
                            _I32),
    "ags_compact_workspace_bytes": ([_I64, _I32], ctypes.c_size_t),
    "ags_emit_tile_workspace_bytes": ([_I64, _I32], ctypes.c_size_t),
    "ags_compact_visible": ([_P, _I64, _I32, _P, _P, _P, _P, _P, ctypes.c_size_t, _P], _I32),
    "ags_emit_pairs_noalloc_max_gaussians": ([], _I64),
    "ags_emit_pairs_noalloc": ([_P, _I64, _I32, _P, _P, _P, _P, _I64, _P, _P, _P], _I32),
    "ags_sort_workspace_bytes": ([_I64], ctypes.c_size_t),
    "ags_sort": ([_P, _P, _P, _P, _P, _I64, _I32, _I32, _I32, _I32, _P, _I64, _P, _P, _P, ctypes.c_size_t, _P],
                 _I32),
    "ags_sort32": ([_P, _P, _P, _P, _P, _I64, _I32, _I32, _I32, _I32, _P, _I64, _P, _P, _P, ctypes.c_size_t, _P],
                   _I32),
    "ags_sort_tiles": ([_P, _P, _P, _P, _P, _I64, _I32, _I32, _I32, _P, _I32, _I32, _P, _P, _P, ctypes.c_size_t,
                        _P], _I32),
    "ags_view_keys": ([_P, _P, _I64, _I64, _P, _P], _I32),
    "ags_rasterize": ([_P, _I64, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _P], _I32),
    "ags_calibrate_lut": ([_P, _P, _I64, _I32, _F, _P, _P], _I32),
    "ags_morton_workspace_bytes": ([], ctypes.c_size_t),
    "ags_morton_codes": ([_P, _P, _P, ctypes.c_size_t, _P], _I32),
    "ags_gather_gaussians": ([_P, _P, _I32, _P, _P, _P, _P, _P, _P], _I32),
    "ags_peripheral_scores": ([_P, _I64, _P, _P, _P, _I32, _P, _P, _P], _I32),
    "ags_contribution_hist": ([_P, _I64, _P, _P, _P, _I32, _P, _I32, _P, _P, _P], _I32),
    "ags_render_skip": ([_P, _I64, _P, _P, _P, _I32, _P, _I32, _P, _F, _P, _P, _P], _I32),
    "ags_backward_workspace_bytes": ([_I64, _I32], ctypes.c_size_t),
    "ags_rasterize_backward": ([_P, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                ctypes.c_size_t, _P], _I32),
    "ags_version": ([], ctypes.c_char_p),
}

_lib = None


def library_path() -> str:
    """libags.so, or the index-checking libags_debug.so when AGS_DEBUG=1."""
    return _build.DEBUG_LIB if os.environ.get("AGS_DEBUG") == "1" else _build.LIB


def lib():
    """The loaded libags.so.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libags.so is not built (%s); run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, (args, res) in EXPORTS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def ptr(t):
    """Device (or host) address of a tensor / None."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def camera(cam: dict) -> AgsCamera:
    c = AgsCamera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    vm = np.asarray(cam["viewmat"], dtype=np.float32).reshape(-1)
    for k in range(12):
        c.viewmat[k] = float(vm[k])
    cp = np.asarray(cam["campos"], dtype=np.float32)
    for k in range(3):
        c.campos[k] = float(cp[k])
    c.near_z = float(cam.get("near", 0.2))
    return c


def cameras(cams) -> ctypes.Array:
    arr = (AgsCamera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera(c)
    return arr


def params(scale_mode: int = AGS_SCALE_PLAIN, K: float = 0.0, lut=None, sh_degree: int = 3, bg=(0.0, 0.0, 0.0),
           tau: float = 1.0 / 255.0, t_min: float = 1e-4, alpha_max: float = 0.99, lut_bins: int = 20,
           lut_depth_max: float = 100.0, tile_test: int = AGS_TILE_SQUARE, blend_flags: int = 0) -> AgsParams:
    p = AgsParams()
    p.scale_mode, p.sh_degree, p.lut_bins = int(scale_mode), int(sh_degree), int(lut_bins)
    p.tile_test, p.blend_flags = int(tile_test), int(blend_flags)
    p.K, p.tau, p.t_min, p.alpha_max, p.lut_depth_max = float(K), float(tau), float(t_min), float(alpha_max), \
        float(lut_depth_max)
    lut = np.ones(lut_bins, dtype=np.float32) if lut is None else np.asarray(lut, dtype=np.float32)
    for i in range(min(len(lut), AGS_MAX_LUT_BINS)):
        p.lut[i] = float(lut[i])
    for i in range(3):
        p.bg[i] = float(bg[i])
    return p


def gaussians(scene) -> AgsGaussians:
    g = AgsGaussians()
    g.mean, g.log_scale, g.quat = ptr(scene["mean"]), ptr(scene["log_scale"]), ptr(scene["quat"])
    g.opacity_logit, g.sh = ptr(scene["opacity_logit"]), ptr(scene["sh"])
    g.n = int(scene["opacity_logit"].shape[0])
    return g


def projected(proj) -> AgsProjected:
    p = AgsProjected()
    p.splat, p.depth, p.rect = ptr(proj["splat"]), ptr(proj["depth"]), ptr(proj["rect"])
    p.tiles_touched, p.flags = ptr(proj.get("tiles_touched")), ptr(proj["flags"])
    p.depth_key = ptr(proj.get("depth_key"))
    return p


def _ok(code: int, where: str):
    if code != 0:
        raise AgsError(code, where)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def ags_status_reset(d_status, stream=None):
    _ok(lib().ags_status_reset(ptr(d_status), stream_handle(stream)), "ags_status_reset")


def ags_check(d_status, stream=None, raise_on_error: bool = True):
    """Synchronise and read the status block; returns (code, detail)."""
    detail = ctypes.c_int64(0)
    code = lib().ags_check(ptr(d_status), stream_handle(stream), ctypes.byref(detail))
    if raise_on_error and code != 0:
        raise AgsError(code, "device status", detail.value)
    return code, detail.value


def ags_status_string(code: int) -> str:
    return lib().ags_status_string(int(code)).decode()


def ags_version() -> str:
    return lib().ags_version().decode()


def ags_preprocess(scene, cams, params_, proj, d_status, stream=None):
    g = gaussians(scene)
    cs = cameras(cams)
    pr = projected(proj)
    _ok(lib().ags_preprocess(ctypes.byref(g), cs, len(cams), ctypes.byref(params_), ctypes.byref(pr),
                             ptr(d_status), stream_handle(stream)), "ags_preprocess")


def ags_emit_workspace_bytes(n: int, views: int) -> int:
    return int(lib().ags_emit_workspace_bytes(int(n), int(views)))


AGS_EMIT_ELLIPSE = 2


def ags_emit_pairs(proj, n, cams, keys, vals, capacity, d_num_pairs, d_status, ws, order=None, flags=0,
                   stream=None):
    pr = projected(proj)
    cs = cameras(cams)
    _ok(lib().ags_emit_pairs(ctypes.byref(pr), int(n), len(cams), cs, ptr(order), ptr(keys), ptr(vals),
                             int(capacity), ptr(d_num_pairs), ptr(d_status), int(flags), ptr(ws),
                             ws.numel() * ws.element_size() if ws is not None else 0, stream_handle(stream)),
        "ags_emit_pairs")


AGS_EMIT_SINGLE_PASS = 1
AGS_EMIT_VIEW_SHIFT = 4
AGS_EMIT_TEST_STALL = 256     # tests only: a look-back partition that never publishes


def ags_emit_tile_pairs(proj, n, cams, keys, vals, capacity, d_num_pairs, d_status, ws, order=None,
                        order_count=None, flags=0, stream=None):
    """Pairs with 32-bit tile keys, emitted in `order` (normally the depth order);
    `order_count` (device int64) limits the entries of `order` visited."""
    pr = projected(proj)
    cs = cameras(cams)
    _ok(lib().ags_emit_tile_pairs(ctypes.byref(pr), int(n), len(cams), cs, ptr(order), ptr(order_count),
                                  ptr(keys), ptr(vals),
                                  int(capacity), ptr(d_num_pairs), ptr(d_status), int(flags), ptr(ws),
                                  ws.numel() * ws.element_size() if ws is not None else 0, stream_handle(stream)),
        "ags_emit_tile_pairs")


def ags_emit_tile_workspace_bytes(n: int, views: int) -> int:
    return int(lib().ags_emit_tile_workspace_bytes(int(n), int(views)))


def ags_compact_workspace_bytes(n: int, views: int) -> int:
    return int(lib().ags_compact_workspace_bytes(int(n), int(views)))


def ags_compact_visible(proj, n, views, keys, ids, d_count, d_status, ws, stream=None):
    """Depth keys and indices of the Gaussian-views with pairs, in index order; count in d_count."""
    pr = projected(proj)
    _ok(lib().ags_compact_visible(ctypes.byref(pr), int(n), int(views), ptr(keys), ptr(ids), ptr(d_count),
                                  ptr(d_status), ptr(ws), ws.numel() * ws.element_size(), stream_handle(stream)),
        "ags_compact_visible")


def ags_emit_pairs_noalloc(proj, n, cams, keys, vals, capacity, d_num_pairs, d_status, order=None, stream=None):
    """ags_emit_pairs with the library's static scratch (for callers that cannot allocate)."""
    pr = projected(proj)
    cs = cameras(cams)
    _ok(lib().ags_emit_pairs_noalloc(ctypes.byref(pr), int(n), len(cams), cs, ptr(order), ptr(keys), ptr(vals),
                                     int(capacity), ptr(d_num_pairs), ptr(d_status), stream_handle(stream)),
        "ags_emit_pairs_noalloc")


def ags_sort_workspace_bytes(capacity: int) -> int:
    return int(lib().ags_sort_workspace_bytes(int(capacity)))


AGS_SORT_IDENTITY_VALUES = 1
AGS_SORT_DISCARD_KEYS = 2
AGS_SORT_RANK_OR = 4
AGS_SORT_WIDE_BLOCK = 8       # 32-bit key passes on 512 x 8 partitions instead of 256 x 16
AGS_SORT_PERSISTENT = 16      # resident blocks take partitions of the device count by ticket
AGS_SORT_TEST_STALL = 256     # tests only: a look-back partition that never publishes


def ags_sort(keys, vals, keys_alt, vals_alt, d_num_pairs, capacity, begin_bit, end_bit, digit_bits, ranges,
             num_ranges, d_status, ws, flags=0, stream=None) -> bool:
    """Returns True when the sorted result is in (keys_alt, vals_alt)."""
    alt = ctypes.c_int32(0)
    _ok(lib().ags_sort(ptr(keys), ptr(vals), ptr(keys_alt), ptr(vals_alt), ptr(d_num_pairs), int(capacity),
                       int(begin_bit), int(end_bit), int(digit_bits), int(flags), ptr(ranges), int(num_ranges),
                       ctypes.byref(alt), ptr(d_status), ptr(ws), ws.numel() * ws.element_size(),
                       stream_handle(stream)), "ags_sort")
    return bool(alt.value)


def ags_sort32(keys, vals, keys_alt, vals_alt, d_num_pairs, capacity, begin_bit, end_bit, digit_bits, ranges,
               num_ranges, d_status, ws, flags=0, stream=None) -> bool:
    """ags_sort for 32-bit keys; returns True when the sorted result is in (keys_alt, vals_alt)."""
    alt = ctypes.c_int32(0)
    _ok(lib().ags_sort32(ptr(keys), ptr(vals), ptr(keys_alt), ptr(vals_alt), ptr(d_num_pairs), int(capacity),
                         int(begin_bit), int(end_bit), int(digit_bits), int(flags), ptr(ranges), int(num_ranges),
                         ctypes.byref(alt), ptr(d_status), ptr(ws), ws.numel() * ws.element_size(),
                         stream_handle(stream)), "ags_sort32")
    return bool(alt.value)


def ags_sort_tiles(keys, vals, keys_alt, vals_alt, d_num_pairs, capacity, tile_bits, digit_bits, ranges, views,
                   tiles_per_view, d_status, ws, flags=0, stream=None) -> bool:
    """Sort of view-shifted tile keys by their tile bits; returns True when the result is in the alt buffers."""
    alt = ctypes.c_int32(0)
    _ok(lib().ags_sort_tiles(ptr(keys), ptr(vals), ptr(keys_alt), ptr(vals_alt), ptr(d_num_pairs), int(capacity),
                             int(tile_bits), int(digit_bits), int(flags), ptr(ranges), int(views),
                             int(tiles_per_view), ctypes.byref(alt), ptr(d_status), ptr(ws),
                             ws.numel() * ws.element_size(), stream_handle(stream)), "ags_sort_tiles")
    return bool(alt.value)


def ags_view_keys(order, d_count, capacity, n, keys, stream=None):
    _ok(lib().ags_view_keys(ptr(order), ptr(d_count), int(capacity), int(n), ptr(keys), stream_handle(stream)),
        "ags_view_keys")


def ags_rasterize(proj, n, sorted_vals, ranges, cams, params_, image, final_T, n_contrib, d_status, max_T=None,
                  stats=None, stream=None):
    pr = projected(proj)
    cs = cameras(cams)
    _ok(lib().ags_rasterize(ctypes.byref(pr), int(n), ptr(sorted_vals), ptr(ranges), cs, len(cams),
                            ctypes.byref(params_), ptr(image), ptr(final_T), ptr(n_contrib), ptr(max_T), ptr(stats),
                            ptr(d_status), stream_handle(stream)), "ags_rasterize")


def ags_calibrate_lut(max_T, depth, count, lut_bins, lut_depth_max, lut_out, stream=None):
    _ok(lib().ags_calibrate_lut(ptr(max_T), ptr(depth), int(count), int(lut_bins), float(lut_depth_max),
                                ptr(lut_out), stream_handle(stream)), "ags_calibrate_lut")


def ags_morton_workspace_bytes() -> int:
    return int(lib().ags_morton_workspace_bytes())


def ags_morton_codes(scene, codes, ws, stream=None):
    g = gaussians(scene)
    _ok(lib().ags_morton_codes(ctypes.byref(g), ptr(codes), ptr(ws), ws.numel() * ws.element_size(),
                               stream_handle(stream)), "ags_morton_codes")


def ags_gather_gaussians(scene, perm, sh_degree, dst, stream=None):
    g = gaussians(scene)
    _ok(lib().ags_gather_gaussians(ctypes.byref(g), ptr(perm), int(sh_degree), ptr(dst["mean"]),
                                   ptr(dst["log_scale"]), ptr(dst["quat"]), ptr(dst["opacity_logit"]), ptr(dst["sh"]),
                                   stream_handle(stream)), "ags_gather_gaussians")


AGS_CONTRIB_HIST_BINS = 32768
SCORE_ROWS = ("th", "eq4", "eq6", "eq7", "eq9", "max_T", "sum_alpha")


def ags_peripheral_scores(proj, n, sorted_vals, ranges, cams, params_, scores, stream=None):
    pr = projected(proj)
    cs = cameras(cams)
    _ok(lib().ags_peripheral_scores(ctypes.byref(pr), int(n), ptr(sorted_vals), ptr(ranges), cs, len(cams),
                                    ctypes.byref(params_), ptr(scores), stream_handle(stream)),
        "ags_peripheral_scores")


def ags_contribution_hist(proj, n, sorted_vals, ranges, cams, params_, rule, max_T, hist, stream=None):
    pr = projected(proj)
    cs = cameras(cams)
    _ok(lib().ags_contribution_hist(ctypes.byref(pr), int(n), ptr(sorted_vals), ptr(ranges), cs, len(cams),
                                    ctypes.byref(params_), int(rule), ptr(max_T), ptr(hist), stream_handle(stream)),
        "ags_contribution_hist")


def ags_render_skip(proj, n, sorted_vals, ranges, cams, params_, rule, max_T, thr, image, counts, stream=None):
    pr = projected(proj)
    cs = cameras(cams)
    _ok(lib().ags_render_skip(ctypes.byref(pr), int(n), ptr(sorted_vals), ptr(ranges), cs, len(cams),
                              ctypes.byref(params_), int(rule), ptr(max_T), float(thr), ptr(image), ptr(counts),
                              stream_handle(stream)), "ags_render_skip")


def ags_backward_workspace_bytes(n: int, views: int) -> int:
    return int(lib().ags_backward_workspace_bytes(int(n), int(views)))


def ags_rasterize_backward(scene, cams, params_, proj, sorted_vals, ranges, final_T, n_contrib, dL_dimage, grads,
                           d_status, ws, stream=None):
    g = gaussians(scene)
    cs = cameras(cams)
    pr = projected(proj)
    _ok(lib().ags_rasterize_backward(ctypes.byref(g), cs, len(cams), ctypes.byref(params_), ctypes.byref(pr),
                                     ptr(sorted_vals), ptr(ranges), ptr(final_T), ptr(n_contrib), ptr(dL_dimage),
                                     ptr(grads["mean"]), ptr(grads["log_scale"]), ptr(grads["quat"]),
                                     ptr(grads["opacity_logit"]), ptr(grads["sh"]), ptr(d_status), ptr(ws),
                                     ws.numel() * ws.element_size(), stream_handle(stream)),
        "ags_rasterize_backward")
