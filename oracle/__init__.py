"""FP64 CPU oracle of the AdaGScale 3D Gaussian Splatting path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
binding) never calls it.  The C source ``ags_oracle.c`` is compiled with gcc
into ``oracle/_build/libags_oracle.so`` and driven through ctypes; it shares
nothing with the CUDA code.

What each function follows (paper: AdaGScale, arXiv 2604.18980):
  preprocess      Sec. 2.1 preprocessing; Eq. 10 threshold; Sec. 3.3 cull and
                  adjusted tile test; Sec. 3.4 depth LUT
  tile_lists      Sec. 2.1 pair generation and sort (tile, then depth)
  rasterize       Eq. 1 and Eq. 2, tau = 1/255, early stop at T < 1e-4
  render_bruteforce  the same blend without tiles or key sort
  backward        exact adjoint of the blend with frozen lists (not in the paper)
  peripheral      Eq. 3 contributions summed per Gaussian over tau <= alpha < x
                  (Eq. 4), with max T and the pixel sum of alpha (Eq. 6-7)
  peripheral_scores  Eq. 4 at each Gaussian's Th (Eq. 10) beside Eq. 6, 7, 9
  render_skip     the blend with low-contribution blends skipped (Fig. 4a,
                  Fig. 5: exact, max-T and T_up rankings)
  sh_basis        real spherical harmonics from the general formula
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ags_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libags_oracle.so")

# per-Gaussian double fields
(F_U, F_V, F_A, F_B, F_C, F_OPAC, F_R, F_G, F_BL, F_DEPTH, F_TH, F_DET, F_LAMBDA,
 F_COVA, F_COVB, F_COVC, F_DEPTH32, F_RARG, F_QELL) = range(19)
NF = 19
# per-Gaussian integer fields
I_RADIUS, I_X0, I_Y0, I_X1, I_Y1, I_TOUCHED, I_CULL, I_EDGE, I_CLAMP, I_GEDGE = range(10)
NI = 10
CULL_NONE, CULL_NEAR, CULL_DET, CULL_TH, CULL_TUP, CULL_NONFINITE, CULL_EMPTY = range(7)
EDGE_NEAR, EDGE_DET, EDGE_TH, EDGE_CEIL, EDGE_RECT, EDGE_LUT, EDGE_ELLIPSE = 1, 2, 4, 8, 16, 32, 64
GEDGE_FRUSTUM, GEDGE_COLOUR = 1, 2   # decisions that change only the derivatives
TILE_SQUARE, TILE_ELLIPSE = 0, 1     # tile test: square footprint, or square and ellipse
TILE = 16

TAU = 1.0 / 255.0        # Sec. 2.1 / Sec. 3.1
T_MIN = 1e-4             # Sec. 2.1 early exit
ALPHA_MAX = 0.99         # 3D-GS alpha clamp
LUT_BINS = 20            # Sec. 3.4: 20 uniform intervals
LUT_DEPTH_MAX = 100.0    # Sec. 3.4: depth range [0, 100]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_library(_SRC, _LIB)
    return _LIB


class OcCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("campos", ctypes.c_double * 3), ("near_z", ctypes.c_double)]


class OcParams(ctypes.Structure):
    _fields_ = [("scale_mode", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("lut_bins", ctypes.c_int32), ("tile_test", ctypes.c_int32),
                ("K", ctypes.c_double), ("tau", ctypes.c_double), ("t_min", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("lut_depth_max", ctypes.c_double),
                ("lut", ctypes.c_double * 32), ("bg", ctypes.c_double * 3),
                ("edge_rel", ctypes.c_double), ("pos_err", ctypes.c_double)]


_P = ctypes.c_void_p


def compile_library(src: str, out: str) -> str:
    """gcc -O2 -fopenmp of an oracle source file into a shared library."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def camera(cam: dict) -> OcCamera:
    c = OcCamera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    vm = np.asarray(cam["viewmat"], dtype=np.float64)
    for r in range(3):
        for k in range(3):
            c.R[r * 3 + k] = vm[r, k]
        c.t[r] = vm[r, 3]
    cp = np.asarray(cam["campos"], dtype=np.float64)
    for k in range(3):
        c.campos[k] = cp[k]
    c.near_z = float(np.float32(cam.get("near", 0.2)))
    return c


def params(cam: dict | None = None, scale_mode: int = 0, K: float = 0.0, lut=None,
           sh_degree: int = 3, bg=(0.0, 0.0, 0.0), tau: float = TAU, t_min: float = T_MIN,
           alpha_max: float = ALPHA_MAX, lut_bins: int = LUT_BINS,
           lut_depth_max: float = LUT_DEPTH_MAX, edge_rel: float = 1e-5,
           pos_err: float | None = None, tile_test: int = TILE_SQUARE) -> OcParams:
    """Render parameters.  `pos_err` defaults to 8 fp32 ulps of the image extent
    (the rounding of a float32 pixel position); it only widens edge classes."""
    p = OcParams()
    p.scale_mode, p.sh_degree, p.lut_bins = int(scale_mode), int(sh_degree), int(lut_bins)
    p.tile_test = int(tile_test)
    p.K, p.tau, p.t_min, p.alpha_max = float(K), float(tau), float(t_min), float(alpha_max)
    p.lut_depth_max = float(lut_depth_max)
    lut = np.ones(lut_bins) if lut is None else np.asarray(lut, dtype=np.float64)
    for i in range(min(32, len(lut))):
        p.lut[i] = float(lut[i])
    for i in range(3):
        p.bg[i] = float(bg[i])
    p.edge_rel = float(edge_rel)
    if pos_err is None:
        ext = max(cam["width"], cam["height"]) if cam is not None else 4096
        pos_err = 8.0 * 2.0 ** -24 * 2.0 ** math.ceil(math.log2(max(ext, 2)))
    p.pos_err = float(pos_err)
    return p


class Oracle:
    """ctypes front end of one compiled oracle library."""

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        L.oracle_preprocess.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int64, _P, _P, _P, _P]
        L.oracle_preprocess.restype = None
        L.oracle_tile_lists.argtypes = [ctypes.c_int64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]
        L.oracle_tile_lists.restype = ctypes.c_int64
        L.oracle_rasterize.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                       _P, _P, _P, _P, _P, _P]
        L.oracle_rasterize.restype = None
        L.oracle_render_bruteforce.argtypes = [ctypes.c_int64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]
        L.oracle_render_bruteforce.restype = None
        L.oracle_peripheral.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                        ctypes.c_double, _P, _P, _P, _P]
        L.oracle_peripheral.restype = None
        L.oracle_render_skip.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                         ctypes.c_int, _P, ctypes.c_double, ctypes.c_double, _P, _P, _P]
        L.oracle_render_skip.restype = None
        L.oracle_backward.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int64, _P, _P, _P, _P, _P,
                                      _P, _P, _P, _P, _P, _P, _P, _P]
        L.oracle_backward.restype = None
        L.oracle_sh_basis.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P]
        L.oracle_sh_basis.restype = None
        L.oracle_num_threads.restype = ctypes.c_int
        self.L = L
        self.path = path

    def preprocess(self, scene: dict, cam: dict, par: OcParams):
        """Per-Gaussian features (double [n][NF]) and integer record ([n][NI])."""
        mean, ls, q = _d(scene["mean"]), _d(scene["log_scale"]), _d(scene["quat"])
        lg, sh = _d(scene["opacity_logit"]), _d(scene["sh"])
        n = lg.shape[0]
        dbl = np.zeros((n, NF), dtype=np.float64)
        irec = np.zeros((n, NI), dtype=np.int32)
        c = camera(cam)
        self.L.oracle_preprocess(_ptr(mean), _ptr(ls), _ptr(q), _ptr(lg), _ptr(sh), n, ctypes.byref(c),
                                 ctypes.byref(par), _ptr(dbl), _ptr(irec))
        return dbl, irec

    def tile_lists(self, dbl, irec, width: int, height: int, tile_mask=None):
        """(tile_start[num_tiles+1] int64, ids[num_pairs] int32) in (tile, depth, id) order.

        tile_mask (optional, [num_tiles]) builds the lists of the selected tiles only."""
        n = dbl.shape[0]
        nt = ((width + TILE - 1) // TILE) * ((height + TILE - 1) // TILE)
        ts = np.zeros(nt + 1, dtype=np.int64)
        mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, dtype=np.uint8)
        total = self.L.oracle_tile_lists(n, _ptr(dbl), _ptr(irec), width, height, _ptr(mask), _ptr(ts), None)
        ids = np.zeros(max(total, 1), dtype=np.int32)
        self.L.oracle_tile_lists(n, _ptr(dbl), _ptr(irec), width, height, _ptr(mask), _ptr(ts), _ptr(ids))
        return ts, ids[:total]

    def rasterize(self, dbl, tile_start, ids, width: int, height: int, par: OcParams, tile_mask=None,
                  want_max_T: bool = False, want_state: bool = False) -> dict:
        n = dbl.shape[0]
        img = np.zeros((3, height, width), dtype=np.float64)
        fT = np.zeros((height, width), dtype=np.float64)
        nc = np.zeros((height, width), dtype=np.int32)
        bud = np.zeros((height, width), dtype=np.float64)
        mT = np.zeros(n, dtype=np.float64) if want_max_T else None
        st = np.zeros((height, width, 3), dtype=np.int32) if want_state else None
        mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, dtype=np.uint8)
        ids = np.ascontiguousarray(ids, dtype=np.int32) if len(ids) else np.zeros(1, dtype=np.int32)
        self.L.oracle_rasterize(n, _ptr(_d(dbl)), _ptr(np.ascontiguousarray(tile_start, dtype=np.int64)),
                                _ptr(ids), width, height, ctypes.byref(par), _ptr(mask), _ptr(img), _ptr(fT),
                                _ptr(nc), _ptr(bud), _ptr(mT), _ptr(st))
        return dict(image=img, final_T=fT, n_contrib=nc, budget=bud, max_T=mT, state=st)

    def render(self, scene: dict, cam: dict, par: OcParams, tile_mask=None, want_max_T: bool = False,
               want_state: bool = False) -> dict:
        """Full forward: preprocess, tile lists, blend."""
        dbl, irec = self.preprocess(scene, cam, par)
        ts, ids = self.tile_lists(dbl, irec, cam["width"], cam["height"], tile_mask)
        out = self.rasterize(dbl, ts, ids, cam["width"], cam["height"], par, tile_mask, want_max_T, want_state)
        out.update(dbl=dbl, irec=irec, tile_start=ts, ids=ids)
        return out

    def render_bruteforce(self, scene: dict, cam: dict, par: OcParams):
        dbl, irec = self.preprocess(scene, cam, par)
        img = np.zeros((3, cam["height"], cam["width"]), dtype=np.float64)
        self.L.oracle_render_bruteforce(dbl.shape[0], _ptr(dbl), _ptr(irec), cam["width"], cam["height"],
                                        ctypes.byref(par), _ptr(img))
        return img

    def backward(self, scene: dict, cam: dict, par: OcParams, tile_start, ids, dL_dimage) -> dict:
        """Gradients of sum(dL_dimage * image) w.r.t. the raw parameters, lists frozen.

        Also `edge` [n]: per Gaussian, the number of pixel decisions (alpha vs
        tau, alpha vs its clamp, p vs 0, the transmittance stop) within their
        edge band; with the gradient-only bits of the preprocess record
        (frustum and colour clamps, I_GEDGE) these mark the Gaussians whose
        derivative can jump under a one-rounding change of the inputs.
        And `budget`: per raw gradient entry (the gradients' shapes), a bound
        on what a near-threshold decision of another Gaussian at a shared
        pixel can change in it (that decision's T and colour-behind
        perturbation, chained through the absolute derivatives)."""
        mean, ls, q = _d(scene["mean"]), _d(scene["log_scale"]), _d(scene["quat"])
        lg, sh = _d(scene["opacity_logit"]), _d(scene["sh"])
        n = lg.shape[0]
        nc = (par.sh_degree + 1) ** 2
        g = dict(mean=np.zeros((3, n)), log_scale=np.zeros((3, n)), quat=np.zeros((4, n)),
                 opacity_logit=np.zeros(n), sh=np.zeros((nc, 3, n)), feat=np.zeros((n, 9)), edge=np.zeros(max(n, 1)))
        c = camera(cam)
        bud = np.zeros((max(n, 1), 11 + 48))
        ids = np.ascontiguousarray(ids, dtype=np.int32) if len(ids) else np.zeros(1, dtype=np.int32)
        self.L.oracle_backward(_ptr(mean), _ptr(ls), _ptr(q), _ptr(lg), _ptr(sh), n, ctypes.byref(c),
                               ctypes.byref(par), _ptr(np.ascontiguousarray(tile_start, dtype=np.int64)),
                               _ptr(ids), _ptr(_d(dL_dimage)), _ptr(g["mean"]), _ptr(g["log_scale"]),
                               _ptr(g["quat"]), _ptr(g["opacity_logit"]), _ptr(g["sh"]), _ptr(g["feat"]),
                               _ptr(g["edge"]), _ptr(bud))
        g["edge"] = g["edge"][:n]
        nj = 11
        g["budget"] = dict(mean=np.ascontiguousarray(bud[:n, 0:3].T), log_scale=np.ascontiguousarray(bud[:n, 3:6].T),
                           quat=np.ascontiguousarray(bud[:n, 6:10].T), opacity_logit=bud[:n, 10].copy(),
                           sh=np.ascontiguousarray(bud[:n, nj:nj + 3 * nc].reshape(n, nc, 3).transpose(1, 2, 0)))
        return g

    def sh_basis(self, degree: int, dirs: np.ndarray) -> np.ndarray:
        """Real SH basis values [len(dirs)][(degree+1)^2] at unit directions [k][3]."""
        nc = (degree + 1) ** 2
        out = np.zeros((len(dirs), nc))
        buf = np.zeros(16)
        for i, d in enumerate(np.asarray(dirs, dtype=np.float64)):
            self.L.oracle_sh_basis(degree, float(d[0]), float(d[1]), float(d[2]), _ptr(buf))
            out[i] = buf[:nc]
        return out

    def num_threads(self) -> int:
        return int(self.L.oracle_num_threads())

    # -- peripheral-score diagnostics (Sec. 3.1 Eq. 4, Sec. 3.2 Eq. 6-9, Fig. 4a, Fig. 5) --
    def peripheral(self, dbl, tile_start, ids, width: int, height: int, par: OcParams, level,
                   level_rel: float = 1e-4) -> dict:
        """Eq. 4 per Gaussian at the level x_i = level[i] over the blend of the
        given lists: ps (sum of alpha T with alpha < x_i), sum_alpha (the same
        pixels' alpha), max_T (over every pixel where it blends) and edge (the
        alpha T of blends within the edge width of x_i or tau)."""
        n = dbl.shape[0]
        out = {k: np.zeros(n, dtype=np.float64) for k in ("ps", "sum_alpha", "max_T", "edge")}
        ids = np.ascontiguousarray(ids, dtype=np.int32) if len(ids) else np.zeros(1, dtype=np.int32)
        self.L.oracle_peripheral(n, _ptr(_d(dbl)), _ptr(np.ascontiguousarray(tile_start, dtype=np.int64)),
                                 _ptr(ids), width, height, ctypes.byref(par), _ptr(_d(level)), float(level_rel),
                                 _ptr(out["ps"]), _ptr(out["sum_alpha"]), _ptr(out["max_T"]), _ptr(out["edge"]))
        return out

    def render_skip(self, dbl, tile_start, ids, width: int, height: int, par: OcParams, rule: int, weight,
                    thr: float, thr_rel: float = 1e-4) -> dict:
        """The plain render's blends, each skipped when its contribution is below
        thr (rule 0: alpha T, Eq. 3; rule 1/2: weight[i] alpha with weight max T_i
        (Eq. 6) or T_up(depth_i) (Eq. 7)).  Returns image, budget, blends, skipped."""
        n = dbl.shape[0]
        img = np.zeros((3, height, width), dtype=np.float64)
        bud = np.zeros((height, width), dtype=np.float64)
        counts = np.zeros(2, dtype=np.int64)
        w = _d(np.zeros(max(n, 1)) if weight is None else weight)
        ids = np.ascontiguousarray(ids, dtype=np.int32) if len(ids) else np.zeros(1, dtype=np.int32)
        self.L.oracle_render_skip(n, _ptr(_d(dbl)), _ptr(np.ascontiguousarray(tile_start, dtype=np.int64)),
                                  _ptr(ids), width, height, ctypes.byref(par), int(rule), _ptr(w), float(thr),
                                  float(thr_rel), _ptr(img), _ptr(counts), _ptr(bud))
        return dict(image=img, budget=bud, blends=int(counts[0]), skipped=int(counts[1]))

    def peripheral_scores(self, scene: dict, cam: dict, K: float, lut, sh_degree: int = 3,
                          level_rel: float = 1e-4, **pkw) -> dict:
        """The scores of every Gaussian at its AdaGScale level Th (Eq. 10 with K
        and the T_up table lut), over the plain render (the alpha >= tau region
        Eq. 4 sums over):
          th   Eq. 10 (inf where T_up = 0),
          eq4  exact peripheral score (sum of alpha T with tau <= alpha < Th),
          eq6  max T_i times the pixel sum of alpha (Eq. 6),
          eq7  T_up(depth_i) times the same sum (Eq. 7),
          eq9  T_up 2 pi sqrt(det Sigma2D) (min(Th, opacity) - tau) (Eq. 9; alpha
               never exceeds the opacity, so the band ends there),
          max_T, sum_alpha, edge, and the plain and AdaGScale preprocess records."""
        plain = params(cam, scale_mode=0, lut=lut, sh_degree=sh_degree, **pkw)
        ada = params(cam, scale_mode=1, K=K, lut=lut, sh_degree=sh_degree, **pkw)
        dbl, irec = self.preprocess(scene, cam, plain)
        dbl_a, irec_a = self.preprocess(scene, cam, ada)
        ts, ids = self.tile_lists(dbl, irec, cam["width"], cam["height"])
        th = np.where(irec_a[:, I_CULL] == CULL_TUP, np.inf, dbl_a[:, F_TH])
        pr = self.peripheral(dbl, ts, ids, cam["width"], cam["height"], plain, th, level_rel)
        tup = lut_value(dbl[:, F_DEPTH], lut, ada.lut_bins, ada.lut_depth_max)
        band = np.minimum(th, dbl[:, F_OPAC]) - ada.tau
        return dict(th=th, eq4=pr["ps"], eq6=pr["max_T"] * pr["sum_alpha"], eq7=tup * pr["sum_alpha"],
                    eq9=tup * 2.0 * math.pi * np.sqrt(np.maximum(dbl[:, F_DET], 0.0)) * band,
                    max_T=pr["max_T"], sum_alpha=pr["sum_alpha"], edge=pr["edge"], dbl=dbl, irec=irec,
                    dbl_ada=dbl_a, irec_ada=irec_a, tile_start=ts, ids=ids)


_default = None


def default() -> Oracle:
    """The oracle built from oracle/ags_oracle.c (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def preprocess(*a, **k):
    return default().preprocess(*a, **k)


def tile_lists(*a, **k):
    return default().tile_lists(*a, **k)


def rasterize(*a, **k):
    return default().rasterize(*a, **k)


def render(*a, **k):
    return default().render(*a, **k)


def render_bruteforce(*a, **k):
    return default().render_bruteforce(*a, **k)


def backward(*a, **k):
    return default().backward(*a, **k)


def sh_basis(*a, **k):
    return default().sh_basis(*a, **k)


def num_threads() -> int:
    return default().num_threads()


def peripheral(*a, **k):
    return default().peripheral(*a, **k)


def render_skip(*a, **k):
    return default().render_skip(*a, **k)


def peripheral_scores(*a, **k):
    return default().peripheral_scores(*a, **k)


def lut_value(depth, lut, bins: int = LUT_BINS, depth_max: float = LUT_DEPTH_MAX):
    """T_up of each depth (Sec. 3.4): bin floor(depth / (depth_max / bins)),
    depths beyond the range in the last bin."""
    lut = np.ones(bins) if lut is None else np.asarray(lut, dtype=np.float64)
    b = np.floor(np.asarray(depth, dtype=np.float64) / (depth_max / bins))
    b = np.clip(b, 0, bins - 1).astype(np.int64)
    return lut[b]


def psnr(a, b, peak: float = 1.0) -> float:
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse)
