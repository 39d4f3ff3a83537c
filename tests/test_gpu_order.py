"""Storage order of the Gaussians along a Morton curve of their means (a
setup step, not in the paper): codes, permutation and gathered arrays against
a numpy restatement, and the same images as the original order."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_pairs, gpu_render
from paper_2604_18980_gb300 import binding as B
from paper_2604_18980_gb300 import render as R
from paper_2604_18980_gb300 import synth

pytestmark = pytest.mark.gpu


def morton_numpy(mean):
    """30-bit Morton codes in float32 arithmetic, 10 bits per axis over the
    bounding box of the finite means (bit 3b + a holds bit b of axis a)."""
    m = np.asarray(mean, dtype=np.float32)
    fin = np.all(np.isfinite(m), axis=0)
    lo, hi = m[:, fin].min(axis=1), m[:, fin].max(axis=1)
    codes = np.zeros(m.shape[1], dtype=np.uint64)
    for a in range(3):
        ext = np.float32(hi[a] - lo[a])
        with np.errstate(invalid="ignore"):
            f = (m[a] - lo[a]) / ext if ext > 0 else np.zeros_like(m[a])
            q = np.minimum(np.maximum(f * np.float32(1024.0), np.float32(0.0)), np.float32(1023.0))
        q = np.where(fin, q, 0).astype(np.uint64)
        for b in range(10):
            codes |= ((q >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    codes[~fin] = 0xFFFFFFFF
    return codes.astype(np.uint32)


def test_morton_order_and_gather():
    scene, cams, _ = synth.workload("c1_cube16k_256", n=5000, width=64, height=48, views=1)
    scene = {k: np.array(v, copy=True) for k, v in scene.items()}
    scene["mean"][:, 17] = np.nan                       # sorted last
    sc = R.scene_to_device(scene)
    codes = torch.empty(5000, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.ags_morton_workspace_bytes(), dtype=torch.uint8, device="cuda")
    B.ags_morton_codes(sc, codes, ws)
    exp = morton_numpy(scene["mean"])
    np.testing.assert_array_equal(codes.cpu().numpy().view(np.uint32), exp)
    out, perm = R.spatial_order(sc)
    p = perm.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(p, np.argsort(exp, kind="stable"))
    assert p[-1] == 17
    for k in sc:
        src = sc[k].cpu().numpy().reshape(-1, 5000)
        np.testing.assert_array_equal(out[k].cpu().numpy().reshape(-1, 5000), src[:, p])


@pytest.mark.parametrize("mode,K", [(0, 0.0), (1, 0.3)])
def test_spatial_order_renders_the_same_images(mode, K):
    scene, cams, _ = synth.workload("c1_cube16k_256", n=12000, width=173, height=94, views=2)
    lut = np.linspace(1.0, 0.4, 20).astype(np.float32)
    a = gpu_render(scene, cams, mode, K, lut if mode else None)
    sc = R.scene_to_device(scene)
    so, perm = R.spatial_order(sc)
    b = R.Renderer(so, cams, mode, K, lut if mode else None)
    b.forward()
    b.check()
    assert a.pairs() == b.pairs()
    # pixels may differ only in tiles where two Gaussians have exactly the same
    # depth (their order follows the index, which the permutation changes)
    keys, _ = gpu_pairs(a)
    tied = np.unique(keys[1:][keys[1:] == keys[:-1]] >> np.uint64(32)).astype(np.int64)
    diff = (a.image != b.image).any(dim=1).cpu().numpy()           # [views][H][W]
    gx = (a.W + 15) // 16
    v, y, x = np.nonzero(diff)
    tiles = v * a.T + (y // 16) * gx + x // 16
    assert np.isin(tiles, tied).all(), "pixels differ outside tiles with equal-depth ties"
    assert diff.mean() < 1e-3
