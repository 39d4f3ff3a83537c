"""Peripheral-score diagnostics on the GPU against the oracle: the exact score
of Eq. 4 at each Gaussian's Th with the estimates of Eq. 6, 7 and 9, the
contribution histogram and the contribution-skip render of Fig. 4a / Fig. 5,
all through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import compare_image, compare_lists, gpu_render, oracle_params
from paper_2604_18980_gb300 import binding as B
from paper_2604_18980_gb300 import diagnostics as D
from paper_2604_18980_gb300 import synth

pytestmark = pytest.mark.gpu

LUT = np.linspace(1.0, 0.4, 20).astype(np.float32)
K = 0.3
F32 = dict(tau=float(np.float32(1.0 / 255.0)), t_min=float(np.float32(1e-4)), alpha_max=float(np.float32(0.99)))


def _setup(n=8000, W=256, H=200, views=2):
    scene, cams, _ = synth.workload("c1_cube16k_256", n=n, width=W, height=H, views=views)
    r = gpu_render(scene, cams, 0, 0.0, LUT, want_stats=True)
    outs = [oracle.render(scene, cam, oracle_params(cam, 0, 0.0, LUT)) for cam in cams]
    ties, edge_tiles = compare_lists(r, outs)
    return scene, cams, r, outs, edge_tiles


def _touches(irec, tiles, gx):
    """Gaussians whose rectangle holds one of `tiles`."""
    hit = np.zeros(irec.shape[0], dtype=bool)
    for t in tiles:
        ty, tx = divmod(int(t), gx)
        hit |= ((irec[:, oracle.I_X0] <= tx) & (tx < irec[:, oracle.I_X1]) & (irec[:, oracle.I_Y0] <= ty)
                & (ty < irec[:, oracle.I_Y1]))
    return hit


def test_peripheral_scores_parity():
    scene, cams, r, outs, edge_tiles = _setup()
    d = D.Diagnostics(r, K, LUT)
    sc = {k: v.view(r.V, r.n).cpu().numpy() for k, v in d.scores().items()}
    # max T is the blend's own calibration statistic, bit for bit
    mt = torch.zeros(r.V * r.n, dtype=torch.float32, device="cuda")
    r.rasterize(max_T=mt)
    np.testing.assert_array_equal(mt.view(r.V, r.n).cpu().numpy(), sc["max_T"])
    gx = (r.W + 15) // 16
    compared = 0
    for v, cam in enumerate(cams):
        o = oracle.peripheral_scores(scene, cam, float(np.float32(K)), LUT.astype(np.float64), **F32)
        live = o["irec"][:, oracle.I_TOUCHED] > 0
        skip = ((o["irec"][:, oracle.I_EDGE] != 0) | ((o["irec_ada"][:, oracle.I_EDGE] & oracle.EDGE_LUT) != 0)
                | _touches(o["irec"], edge_tiles[v], gx))
        sel = live & ~skip
        g = {k: sc[k][v] for k in sc}
        # Th (Eq. 10) and Eq. 9 depend on the Gaussian alone
        fin = sel & np.isfinite(o["th"])
        np.testing.assert_allclose(g["th"][fin], o["th"][fin], rtol=1e-5)
        assert np.all(np.isinf(g["th"][sel & ~np.isfinite(o["th"])]))
        np.testing.assert_allclose(g["eq9"][sel], o["eq9"][sel], rtol=3e-5, atol=1e-7)
        # sums over the blend: tight where no blend of the Gaussian sits near a threshold
        clean = sel & (o["edge"] == 0)
        for k, rt in (("eq4", 2e-4), ("sum_alpha", 2e-4), ("max_T", 1e-4), ("eq6", 3e-4), ("eq7", 3e-4)):
            np.testing.assert_allclose(g[k][clean], o[k][clean], rtol=rt, atol=1e-6, err_msg=k)
        near = sel & (o["edge"] > 0)
        assert np.all(np.abs(g["eq4"][near] - o["eq4"][near]) <= 2e-4 * o["eq4"][near] + 2 * o["edge"][near] + 1e-6)
        assert clean.sum() > 0.5 * live.sum()
        compared += int(clean.sum())
        # Eq. 6 never falls below the exact score (max T >= T at every pixel)
        assert np.all(g["eq6"][live] >= g["eq4"][live] * (1 - 1e-5))
    assert compared > 1000


def test_contribution_hist_and_skip_parity():
    scene, cams, r, outs, edge_tiles = _setup(n=6000, W=173, H=94)
    d = D.Diagnostics(r, K, LUT)
    sc = d.scores()
    max_T = sc["max_T"].contiguous()
    blends = int(r.stats[1].item())
    # no threshold: the skip render is the plain image, bit for bit
    img, nb, ns = d.render_skip(0, 0.0, max_T)
    assert torch.equal(img, r.image) and nb == blends and ns == 0
    o_maxT = []
    for v, cam in enumerate(cams):
        oo = outs[v]
        pr = oracle.peripheral(oo["dbl"], oo["tile_start"], oo["ids"], cam["width"], cam["height"],
                               oracle_params(cam, 0, 0.0, LUT), np.full(r.n, np.inf))
        o_maxT.append(pr["max_T"])
    for rule in (0, 1, 2):
        h = d.hist(rule, max_T).cpu().numpy().view(np.uint32).astype(np.int64)
        assert h.sum() == blends
        for frac in (0.3, 0.7):
            thr = D.Diagnostics.threshold_for(h, frac)
            b = int(np.array([thr], dtype=np.float32).view(np.uint32)[0] >> 16)
            img, nb, ns = d.render_skip(rule, thr, max_T)
            assert nb == blends and ns == h[:b].sum()          # the two kernels rank alike
            o_skipped = 0
            for v, cam in enumerate(cams):
                oo = outs[v]
                par = oracle_params(cam, 0, 0.0, LUT)
                w = None if rule == 0 else (o_maxT[v] if rule == 1 else
                                            oracle.lut_value(oo["dbl"][:, oracle.F_DEPTH], LUT.astype(np.float64)))
                os_ = oracle.render_skip(oo["dbl"], oo["tile_start"], oo["ids"], cam["width"], cam["height"], par,
                                         rule, w, thr)
                o_skipped += os_["skipped"]
                compare_image(img[v].cpu().numpy(), os_, edge_tiles=edge_tiles[v])
            assert abs(o_skipped - ns) <= 1e-3 * blends + 5


def test_diagnostics_degenerate():
    """No visible Gaussian: zero scores, an empty histogram and the background."""
    scene, cams, _ = synth.workload("c1_cube16k_256", n=256, width=64, height=48, views=1)
    scene = dict(scene)
    scene["mean"] = np.array(scene["mean"], copy=True)
    scene["mean"][:] = np.asarray(cams[0]["campos"], dtype=np.float32)[:, None]   # at the camera centre
    r = gpu_render(scene, cams, 0, 0.0, LUT, bg=(0.25, 0.5, 0.75))
    assert r.pairs() == 0
    d = D.Diagnostics(r, K, LUT)
    sc = d.scores()
    assert all(float(v.abs().sum()) == 0.0 for v in sc.values())
    assert int(d.hist(0).sum()) == 0
    img, nb, ns = d.render_skip(0, 0.5)
    assert nb == 0 and ns == 0 and torch.equal(img, r.image)


def test_diagnostics_reject_bad_arguments():
    scene, cams, _ = synth.workload("c1_cube16k_256", n=256, width=64, height=48, views=1)
    r = gpu_render(scene, cams, 0, 0.0, LUT)
    d = D.Diagnostics(r, K, LUT)
    with pytest.raises(B.AgsError):
        d.hist(3)
    with pytest.raises(B.AgsError):
        d.hist(1, None)                   # rule 1 needs the max-T weights
    with pytest.raises(B.AgsError):
        d.render_skip(0, -1.0)
