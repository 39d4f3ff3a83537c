"""Peripheral-score diagnostics over a plain render (Sec. 2.2 Fig. 4a, Sec. 3.1
Eq. 4, Sec. 3.2 Eq. 6-9 and Fig. 5-6).

``Diagnostics`` wraps a ``Renderer`` in plain mode (its pair lists cover the
whole alpha >= tau region that Eq. 4 sums over) and runs the libags
diagnostic kernels on it:

  scores()       per Gaussian-view, at its AdaGScale level Th (Eq. 10 with K
                 and the T_up table): the exact peripheral score (Eq. 4) and
                 its estimates Eq. 6, Eq. 7, Eq. 9, with max T and the pixel
                 sum of alpha;
  hist(rule)     the distribution of the blends' contributions under one
                 ranking (0: alpha T, 1: max T alpha, 2: T_up(depth) alpha);
  skip_curve()   PSNR against the plain image when the lowest-ranked blends
                 are skipped, for several skip fractions (Fig. 4a, Fig. 5);
  max_T_by_depth()  the max-T statistic binned by depth (Fig. 6).

Every per-pixel step runs in the library; this module only chooses
thresholds from the histogram and summarises with torch reductions.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

RULES = {0: "exact alpha*T (Eq. 3)", 1: "max T * alpha (Eq. 6)", 2: "T_up(depth) * alpha (Eq. 7)"}


def bin_lower_edge(b: int) -> float:
    """Smallest float whose bits >> 16 equal b (the lower edge of histogram bin b)."""
    return float(np.array([b << 16], dtype=np.uint32).view(np.float32)[0])


class Diagnostics:
    def __init__(self, renderer, K: float, lut, lut_bins: int = 20, lut_depth_max: float = 100.0):
        r = renderer
        self.r = r
        self.K = float(K)
        prev = r._pargs
        self.params = B.params(scale_mode=B.AGS_SCALE_ADAGSCALE, K=K, lut=lut, sh_degree=prev["sh_degree"],
                               bg=prev["bg"], lut_bins=lut_bins, lut_depth_max=lut_depth_max)
        self.lut_bins, self.lut_depth_max = lut_bins, lut_depth_max
        dev = r.image.device
        self.scores_buf = torch.empty(7, r.V * r.n, dtype=torch.float32, device=dev)
        self.hist_buf = torch.empty(B.AGS_CONTRIB_HIST_BINS, dtype=torch.int32, device=dev)
        self.skip_image = torch.empty_like(r.image)
        self.counts = torch.zeros(2, dtype=torch.int64, device=dev)

    def scores(self) -> dict:
        """Rows th, eq4, eq6, eq7, eq9, max_T, sum_alpha ([views*n] each)."""
        r = self.r
        B.ags_peripheral_scores(r.proj, r.n, r.sorted_vals, r.ranges, r.cams, self.params, self.scores_buf)
        return {name: self.scores_buf[k] for k, name in enumerate(B.SCORE_ROWS)}

    def hist(self, rule: int, max_T=None) -> torch.Tensor:
        r = self.r
        B.ags_contribution_hist(r.proj, r.n, r.sorted_vals, r.ranges, r.cams, self.params, rule, max_T,
                                self.hist_buf)
        return self.hist_buf

    def render_skip(self, rule: int, thr: float, max_T=None):
        """(image [views][3][H][W], blends, skipped)."""
        r = self.r
        self.counts.zero_()
        B.ags_render_skip(r.proj, r.n, r.sorted_vals, r.ranges, r.cams, self.params, rule, max_T, thr,
                          self.skip_image, self.counts)
        c = self.counts.cpu().tolist()
        return self.skip_image, int(c[0]), int(c[1])

    @staticmethod
    def threshold_for(hist: np.ndarray, fraction: float) -> float:
        """The histogram bin edge whose share of blends below it is closest to `fraction`."""
        cum = np.concatenate([[0], np.cumsum(hist.astype(np.int64))])
        tot = cum[-1]
        if tot == 0:
            return 0.0
        b = int(np.argmin(np.abs(cum / tot - fraction)))
        return 0.0 if b == 0 else bin_lower_edge(b)

    def skip_curve(self, rules=(0, 1, 2), fractions=(0.2, 0.4, 0.6, 0.8), reference=None) -> list:
        """PSNR (dB, peak 1) of the skip render against the plain image per
        (rule, target fraction), with the realised fraction of skipped blends."""
        ref = self.r.image if reference is None else reference
        sc = self.scores()
        max_T = sc["max_T"].contiguous()
        out = []
        for rule in rules:
            h = self.hist(rule, max_T).cpu().numpy().view(np.uint32)
            for f in fractions:
                thr = self.threshold_for(h, f)
                img, blends, skipped = self.render_skip(rule, thr, max_T)
                mse = float(torch.mean((img - ref) ** 2))
                psnr = float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)
                out.append(dict(rule=rule, target=f, skipped_fraction=skipped / max(blends, 1), threshold=thr,
                                psnr_vs_plain_db=psnr))
        return out

    def summary(self, sc: dict | None = None) -> dict:
        """How the estimates bound the exact score at Th, over the Gaussian-views that blend."""
        sc = self.scores() if sc is None else sc
        live = sc["max_T"] > 0
        e4 = sc["eq4"][live].double()
        res = dict(gaussian_views=int(live.sum()), K=self.K)
        if e4.numel() == 0:
            return res
        res["exact_over_K_fraction"] = float((e4 > self.K).double().mean())
        res["exact_mean_over_K"] = float(e4.mean() / self.K) if self.K > 0 else None
        pos = e4 > 0
        for name in ("eq6", "eq7", "eq9"):
            est = sc[name][live].double()
            res[name + "_ge_exact_fraction"] = float((est >= e4 * (1 - 1e-5)).double().mean())
            if pos.any():
                res[name + "_over_exact_median"] = float(torch.median(est[pos] / e4[pos]))
        return res

    def max_T_by_depth(self, sc: dict | None = None, depth_bins: int = 20) -> list:
        """Per depth bin of the T_up table (Sec. 3.4): Gaussian-views that blend,
        and the median and max of their max T (the statistic T_up bounds)."""
        sc = self.scores() if sc is None else sc
        r = self.r
        depth = r.proj["depth"]
        live = sc["max_T"] > 0
        b = torch.clamp((depth[live] * (depth_bins / self.lut_depth_max)).floor(), 0, depth_bins - 1).long()
        mt = sc["max_T"][live]
        rows = []
        for k in range(depth_bins):
            v = mt[b == k]
            if v.numel():
                rows.append(dict(bin=k, count=int(v.numel()), median=float(v.median()), max=float(v.max())))
        return rows
