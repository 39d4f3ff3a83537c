"""Offline calibration of AdaGScale's two scene parameters (Sec. 3.4).

* ``calibrate_lut``: T_up(depth), a piecewise-constant upper bound of the
  per-Gaussian maximum transmittance: plain-mode renders of the calibration
  views record, per Gaussian, the largest T seen before it is blended
  (``ags_rasterize`` max_T output); ``ags_calibrate_lut`` bins those maxima by
  depth (20 uniform bins of [0, 100] in the paper) and keeps each bin's maximum.
* ``search_K``: binary search of the peripheral-loss budget K so that the
  AdaGScale renders of the calibration views stay at a target PSNR against the
  plain renders (the paper searches against a target PSNR drop; the synthetic
  scenes have no ground truth, so the target is expressed against plain 3-sigma
  renders).  Larger K removes more pairs and costs more PSNR, which makes the
  search well posed.

Run as a script to write the parameters of a named workload:
    python -m paper_2604_18980_gb300.calibrate --workload c2_clusters1m_1080p --write
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np
import torch

from . import binding as B
from . import render as R
from . import synth

PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_params.json")
# Synthetic stand-in for the paper's -0.5 dB target (Sec. 4.2-4.3): with the
# AdaGScale error uncorrelated with the baseline error, a 0.5 dB drop at a
# baseline PSNR P means MSE_ada / MSE_base = 10^0.05 - 1, i.e. PSNR against the
# plain render of P + 9.14 dB: 36.1 dB for the 27.0 dB mean of the original
# 3D-GS models (Table II), 29.8 dB for the 20.65 dB CityGaussian mean.
TARGET_PSNR = {"c1": 36.1, "c2": 36.1, "c3": 29.8, "c4": 29.8, "c5": 36.1}


def psnr(a: torch.Tensor, b: torch.Tensor) -> float:
    mse = torch.mean((a.double() - b.double()) ** 2).item()
    return math.inf if mse == 0 else 10.0 * math.log10(1.0 / mse)


def calibrate_lut(scene: dict, calib_cams: list, sh_degree: int = 3, lut_bins: int = 20,
                  lut_depth_max: float = 100.0, batch: int = 8) -> np.ndarray:
    """T_up(depth) table from plain-mode renders of the calibration views (Sec. 3.4).

    Bins that no Gaussian reached read 1.0."""
    dev = scene["mean"].device
    n = int(scene["opacity_logit"].shape[0])
    total = len(calib_cams) * n
    maxT = torch.zeros(total, dtype=torch.float32, device=dev)
    depth = torch.zeros(total, dtype=torch.float32, device=dev)
    for s in range(0, len(calib_cams), batch):
        cams = calib_cams[s:s + batch]
        r = R.Renderer(scene, cams, B.AGS_SCALE_PLAIN, sh_degree=sh_degree)
        r.forward(max_T=maxT[s * n:(s + len(cams)) * n])
        depth[s * n:(s + len(cams)) * n].copy_(r.proj["depth"])
        r.check()
        del r
    lut = torch.zeros(lut_bins, dtype=torch.float32, device=dev)
    B.ags_calibrate_lut(maxT, depth, total, lut_bins, lut_depth_max, lut)
    return lut.cpu().numpy()


def search_K(scene: dict, calib_cams: list, lut, target_psnr: float, sh_degree: int = 3, batch: int = 8,
             k_lo: float = 0.0, k_hi: float = 4096.0, iters: int = 16, tile_test: int = B.AGS_TILE_SQUARE) -> tuple:
    """Largest K (geometric bisection) whose AdaGScale renders keep PSNR >= target vs plain
    (with the given tile test; the plain reference is the same with either test)."""
    groups = [calib_cams[s:s + batch] for s in range(0, len(calib_cams), batch)]
    plains, rens = [], []
    for cams in groups:
        r = R.Renderer(scene, cams, B.AGS_SCALE_PLAIN, sh_degree=sh_degree)
        plains.append(r.forward().clone())
        r.check()
        ra = R.Renderer(scene, cams, B.AGS_SCALE_ADAGSCALE, 0.0, lut, sh_degree, capacity=r.capacity,
                        tile_test=tile_test)
        rens.append(ra)

    def score(K):
        num = 0.0
        for ra, pl in zip(rens, plains):
            ra.set_params(K=K)
            img = ra.forward()
            ra.check()
            num += torch.sum((img.double() - pl.double()) ** 2).item()
        mse = num / sum(p.numel() for p in plains)
        return math.inf if mse == 0 else 10.0 * math.log10(1.0 / mse)

    lo, hi = k_lo, k_hi
    if score(hi) >= target_psnr:
        return hi, score(hi)
    for _ in range(iters):
        mid = math.sqrt(max(lo, 1e-3) * hi) if lo > 0 else hi / 64.0
        if score(mid) >= target_psnr:
            lo = mid
        else:
            hi = mid
    return lo, score(lo)


def calibrate_workload(name: str, device="cuda") -> dict:
    """LUT, K and the ellipse test's K of a named workload, with the wall-clock
    seconds each took on this GPU (the scene already on the device)."""
    import time
    scene, cams, calib = synth.workload(name)
    sc = R.scene_to_device(scene, device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lut = calibrate_lut(sc, calib)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    target = TARGET_PSNR[name[:2]]
    K, p = search_K(sc, calib, lut, target)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # the ellipse tile test drops more of each footprint: its own K for the same target
    Ke, pe = search_K(sc, calib, lut, target, tile_test=B.AGS_TILE_ELLIPSE)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    return dict(K=float(np.float32(K)), lut=[float(x) for x in lut], target_psnr=target, calib_psnr=p,
                calibration_views=len(calib), K_ellipse=float(np.float32(Ke)), calib_psnr_ellipse=pe,
                seconds=dict(lut=round(t1 - t0, 3), K_search=round(t2 - t1, 3), K_search_ellipse=round(t3 - t2, 3)))


def load_params(name: str) -> dict | None:
    if not os.path.exists(PARAMS_FILE):
        return None
    return json.load(open(PARAMS_FILE)).get(name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2_clusters1m_1080p")
    ap.add_argument("--write", action="store_true")
    ap.add_argument("--ellipse-only", action="store_true",
                    help="keep the stored LUT and K; add the K of the ellipse tile test")
    a = ap.parse_args()
    if a.ellipse_only:
        out = dict(load_params(a.workload))
        scene, _, calib = synth.workload(a.workload)
        sc = R.scene_to_device(scene)
        Ke, pe = search_K(sc, calib, np.asarray(out["lut"], np.float32), out["target_psnr"],
                          tile_test=B.AGS_TILE_ELLIPSE)
        out.update(K_ellipse=float(np.float32(Ke)), calib_psnr_ellipse=pe)
    else:
        out = calibrate_workload(a.workload)
    print(json.dumps({a.workload: out}, indent=1))
    if a.write:
        data = json.load(open(PARAMS_FILE)) if os.path.exists(PARAMS_FILE) else {}
        data[a.workload] = out
        json.dump(data, open(PARAMS_FILE, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
