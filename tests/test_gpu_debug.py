"""The index-checking build (libags_debug.so, compiled with -DAGS_DEBUG).

On a clean frame it gives the release library's results bit for bit; on
planted out-of-range indices -- a pair value past the splat records, a tile
range with start > end, an emission order entry past the Gaussian-views -- it
records AGS_ERR_BOUNDS with the check's id and sets the check's bit, skipping
the access, so nothing out of range is ever read or written.  The planted
values are consumed only by the debug kernels, whose checks come before the
access.  The binding loads one library per process, so each side runs in a
child process (AGS_DEBUG=1 selects the debug library)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import torch
sys.path.insert(0, ROOT)
from paper_2604_18980_gb300 import binding as B, render as R, synth

scene, cams, _ = synth.workload("c1_cube16k_256", n=6000, width=150, height=100, views=2)
sc = R.scene_to_device(scene)
r = R.Renderer(sc, cams, 1, 0.3, want_backward=True)
img = r.forward().clone()
r.check()
dL = torch.linspace(-1.0, 1.0, img.numel(), device="cuda").reshape(img.shape)
g = r.backward(dL)
r.check()
torch.save(dict(img=img.cpu(), T=r.final_T.cpu(), nc=r.n_contrib.cpu(),
                grads={k: v.cpu() for k, v in g.items()}), OUT + ".pt")
res = dict(version=B.ags_version())
if PLANT:
    bad = r.V * r.n + 7                     # one past the records, plus a margin
    rg = r.ranges.view(-1, 2)
    t = int(torch.argmax(rg[:, 1] - rg[:, 0]))     # the longest list: its pixels blend
    s0, e0 = int(rg[t, 0]), int(rg[t, 1])

    def status():
        st = r.status.cpu().tolist()
        B.ags_status_reset(r.status)
        return [st[0], st[1], st[3]]

    keep = int(r.sorted_vals[s0])
    r.sorted_vals[s0] = bad                 # a pair value out of range
    r.rasterize()
    res["blend_value"] = status()
    r.backward(dL)
    res["backward_value"] = status()
    r.sorted_vals[s0] = keep
    rg[t, 0], rg[t, 1] = e0, s0             # a range with start > end (both inside the pairs)
    r.rasterize()
    res["blend_range"] = status()
    r.backward(dL)
    res["backward_range"] = status()
    rg[t, 0], rg[t, 1] = s0, e0
    r.rasterize()
    res["clean_again"] = status()
    r.preprocess()
    r.depth_sort()
    assert int(r.n_visible.item()) > 0
    r.emit_order[0] = bad                   # an emission order entry out of range
    r.emit()
    res["emit_order"] = status()
json.dump(res, open(OUT + ".json", "w"))
'''


def _run(tmp_path, name, debug, plant):
    out = str(tmp_path / name)
    env = dict(os.environ, AGS_DEBUG="1" if debug else "0")
    code = "ROOT = %r\nOUT = %r\nPLANT = %r\n" % (ROOT, out, plant) + CHILD
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr
    import torch
    return json.load(open(out + ".json")), torch.load(out + ".pt")


@pytest.mark.gpu
def test_debug_build_matches_release_and_reports_planted_indices(tmp_path):
    import torch
    from paper_2604_18980_gb300 import binding as B
    from paper_2604_18980_gb300 import build as cuda_build
    cuda_build.build(debug=True)
    rel_info, rel = _run(tmp_path, "release", debug=False, plant=False)
    dbg_info, dbg = _run(tmp_path, "debug", debug=True, plant=True)
    assert "AGS_DEBUG" in dbg_info["version"] and "AGS_DEBUG" not in rel_info["version"]
    assert torch.equal(dbg["img"], rel["img"])
    assert torch.equal(dbg["T"], rel["T"])
    assert torch.equal(dbg["nc"], rel["nc"])
    for k, v in rel["grads"].items():          # float atomics: summation order may differ
        torch.testing.assert_close(dbg["grads"][k], v, rtol=1e-5, atol=1e-7 * float(v.abs().max()))
    for key, chk in (("blend_value", B.AGS_CHECK_BLEND_VALUE), ("backward_value", B.AGS_CHECK_BACKWARD_VALUE),
                     ("blend_range", B.AGS_CHECK_BLEND_RANGE), ("backward_range", B.AGS_CHECK_BACKWARD_RANGE),
                     ("emit_order", B.AGS_CHECK_EMIT_ORDER)):
        assert dbg_info[key] == [B.AGS_ERR_BOUNDS, chk, 1 << chk], (key, dbg_info[key])
    assert dbg_info["clean_again"] == [0, 0, 0]
