"""The double-buffered host driver: every frame renders its own uploaded
parameters (no stale buffers across the two slots) and returns the image of a
plain single-stream render, bit for bit."""
import numpy as np
import pytest
import torch

from paper_2604_18980_gb300 import render as R
from paper_2604_18980_gb300 import synth

pytestmark = pytest.mark.gpu


def test_host_pipeline_frames_match_single_renders():
    scene, cams, _ = synth.workload("c1_cube16k_256", n=6000, width=96, height=64, views=2)
    lut = np.linspace(1.0, 0.4, 20).astype(np.float32)
    sc = R.scene_to_device(scene)
    frames = []
    for f in range(5):                                 # a different scene every frame
        s = {k: v.clone() for k, v in sc.items()}
        s["opacity_logit"] += 0.3 * f
        s["mean"][0] += 0.01 * f
        frames.append(s)
    host = [{k: v.cpu().pin_memory() for k, v in s.items()} for s in frames]
    outs = [torch.empty(2, 3, 64, 96).pin_memory() for _ in frames]
    pipe = R.HostPipeline(sc, cams, 1, 0.3, lut, keep_state=False, capacity=1 << 20)
    pipe.begin()
    for f in range(5):
        pipe.submit(host[f], outs[f])
    pipe.wait()
    torch.cuda.synchronize()
    pipe.check()
    for f in range(5):
        r = R.Renderer(frames[f], cams, 1, 0.3, lut, keep_state=False, capacity=1 << 20)
        assert torch.equal(outs[f], r.forward().cpu()), f
