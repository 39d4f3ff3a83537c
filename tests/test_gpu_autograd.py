"""The autograd wrapper and the fine-tune loop with AdaGScale in it."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import GRAD_KEYS, compare_gradients, gradient_edge_gaussians, oracle_params
from paper_2604_18980_gb300 import binding as B
from paper_2604_18980_gb300 import finetune as F
from paper_2604_18980_gb300 import render as R
from paper_2604_18980_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_18980_gb300 import build
    build.build()
    B.lib()


def _params(scene):
    return [torch.nn.Parameter(torch.as_tensor(scene[k], dtype=torch.float32).cuda()) for k in GRAD_KEYS]


def test_agsrender_gradients_match_backward_and_oracle():
    """loss.backward() through AgsRender gives Renderer.backward's gradients
    and, against the FP64 oracle, the parity bar of the gradient tests."""
    scene, cam = synth.fd_subscene()
    scene["opacity_logit"][:4] = 5.5
    rng = np.random.default_rng(5)
    w = rng.normal(size=(3, cam["height"], cam["width"])).astype(np.float32)
    wt = torch.from_numpy(w).cuda()[None]
    ps = _params(scene)
    r = R.Renderer({k: p.detach() for k, p in zip(GRAD_KEYS, ps)}, [cam], B.AGS_SCALE_ADAGSCALE, 0.05,
                   want_backward=True)
    img = R.AgsRender.apply(*ps, r)
    (img * wt).sum().backward()
    got = {k: p.grad for k, p in zip(GRAD_KEYS, ps)}
    # the same frame through the renderer directly
    r2 = R.Renderer(R.scene_to_device(scene), [cam], B.AGS_SCALE_ADAGSCALE, 0.05, want_backward=True)
    r2.forward()
    ref = r2.backward(wt)
    r2.check()
    for k in GRAD_KEYS:   # the per-splat sums are float atomics: equal up to their order
        torch.testing.assert_close(got[k], ref[k], rtol=1e-5, atol=1e-6 * float(ref[k].abs().max()), msg=k)
    par = oracle_params(cam, 1, 0.05)
    oo = oracle.render(scene, cam, par)
    og = oracle.backward(scene, cam, par, oo["tile_start"], oo["ids"], w.astype(np.float64))
    compare_gradients(got, og, skip=gradient_edge_gaussians(oo, og))


def test_agsrender_refuses_a_stale_blend_state():
    scene, cam = synth.fd_subscene()
    ps = _params(scene)
    r = R.Renderer({k: p.detach() for k, p in zip(GRAD_KEYS, ps)}, [cam], B.AGS_SCALE_PLAIN, want_backward=True)
    first = R.AgsRender.apply(*ps, r)
    second = R.AgsRender.apply(*ps, r)          # overwrites the renderer's blend state
    with pytest.raises(RuntimeError, match="another forward"):
        first.sum().backward()
    second.sum().backward()                     # the latest frame still differentiates
    assert all(p.grad is not None for p in ps)


def test_agsrender_grows_the_pair_capacity():
    """A scene that moved after the buffers were sized: the forward finds the
    overflow in the status block, grows the capacity and renders again."""
    scene, cams, _ = synth.workload("c1_cube16k_256", n=3000, width=96, height=80)
    ps = _params(scene)
    r = R.Renderer({k: p.detach() for k, p in zip(GRAD_KEYS, ps)}, cams, B.AGS_SCALE_PLAIN, capacity=1024,
                   want_backward=True)
    img = R.AgsRender.apply(*ps, r)
    assert r.capacity >= r.pairs() > 1024
    ref = R.Renderer(R.scene_to_device(scene), cams, B.AGS_SCALE_PLAIN)
    assert torch.equal(img, ref.forward())


def test_finetune_with_adagscale_in_the_loop_lowers_the_loss():
    """Adam on every attribute, the AdaGScale pair selection recomputed every
    step from the current parameters: the L2 loss against the perturbed
    scene's render falls step after step."""
    scene, cams, _ = synth.workload("c1_cube16k_256", n=4000, width=128, height=96, views=2)
    pert = synth.perturb_scene(scene, 77)
    tgt = R.Renderer(R.scene_to_device(pert), cams, B.AGS_SCALE_PLAIN).forward().clone()
    out = F.finetune(R.scene_to_device(scene), cams, tgt, B.AGS_SCALE_ADAGSCALE, 0.3, steps=15)
    L = out["losses"]
    assert all(b <= a * (1 + 1e-3) for a, b in zip(L, L[1:])), L
    assert L[-1] < 0.6 * L[0], L
    assert len(set(out["pairs"])) > 1          # the selection followed the parameters


def test_train_step_one_rank_matches_the_batched_backward_and_oracle():
    """multiview.train_step over one rank with the libags renderer: the loss
    and gradients of one batched render of all views, and the oracle's
    gradient summed over the views."""
    from paper_2604_18980_gb300 import multiview as MV
    scene, cams, _ = synth.workload("c1_cube16k_256", n=3000, width=96, height=80, views=3)
    pert = synth.perturb_scene(scene, 31)
    tgt = R.Renderer(R.scene_to_device(pert), cams, B.AGS_SCALE_PLAIN).forward().clone()
    inv = 1.0 / tgt.numel()
    r = R.Renderer(R.scene_to_device(scene), cams, B.AGS_SCALE_ADAGSCALE, 0.2, want_backward=True)
    loss, g = MV.train_step([0, 1, 2], MV.renderer_grads(r, tgt, inv))
    r2 = R.Renderer(R.scene_to_device(scene), cams, B.AGS_SCALE_ADAGSCALE, 0.2, want_backward=True)
    img = r2.forward()
    assert abs(loss - float(((img - tgt) ** 2).sum().item()) * inv) <= 1e-6 * loss
    ref = r2.backward((img - tgt) * (2.0 * inv))
    for k in GRAD_KEYS:
        torch.testing.assert_close(g[k], ref[k], rtol=1e-5, atol=1e-6 * float(ref[k].abs().max()), msg=k)
    tot, edge = None, None
    timg = tgt.cpu().numpy().astype(np.float64)
    for v, cam in enumerate(cams):
        par = oracle_params(cam, 1, 0.2)
        oo = oracle.render(scene, cam, par)
        og = oracle.backward(scene, cam, par, oo["tile_start"], oo["ids"], 2.0 * inv * (oo["image"] - timg[v]))
        e = gradient_edge_gaussians(oo, og)
        if tot is None:
            tot, edge = og, e
        else:
            tot = dict({k: tot[k] + og[k] for k in GRAD_KEYS},
                       budget={k: tot["budget"][k] + og["budget"][k] for k in GRAD_KEYS})
            edge = edge | e
    compare_gradients(g, tot, skip=edge)
