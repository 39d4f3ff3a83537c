"""Fine-tuning a scene with AdaGScale in the loop.

Every step renders the views through ``AgsRender`` -- preprocess with the
AdaGScale threshold (Eq. 10) and its culling, pair emission, sort and blend,
so the pair selection is recomputed from the current parameters -- takes the
L2 loss against target images, runs the hand-written backward with that
step's pair lists held fixed (the selection is piecewise constant in the
parameters), and applies one Adam update to every Gaussian attribute.  The
renderer, its kernels and its adjoints are libags's; the loss, its image
gradient and the optimiser are plain PyTorch tensor arithmetic outside the
rendering path.
"""
from __future__ import annotations

import torch

from . import binding as B
from . import render as R

# Adam step sizes per attribute (scene units: means in world units, log-scales
# and logits dimensionless, SH coefficients in colour units)
DEFAULT_LR = dict(mean=2e-4, log_scale=2e-3, quat=2e-3, opacity_logit=1e-2, sh=2e-3)


def finetune(scene: dict, cams: list, target: torch.Tensor, scale_mode: int = B.AGS_SCALE_ADAGSCALE,
             K: float = 0.0, lut=None, steps: int = 20, lr: dict | None = None, renderer_kwargs: dict | None = None,
             timed: bool = False) -> dict:
    """Adam on every attribute of `scene` (device tensors, copied) so that its
    render of `cams` approaches `target` ([views][3][H][W]).  Returns the
    fitted scene, the loss before each step and, with timed=True, the
    CUDA-event milliseconds of each step (forward, backward and update)."""
    lr = dict(DEFAULT_LR, **(lr or {}))
    params = {k: torch.nn.Parameter(scene[k].detach().clone()) for k in R.SCENE_KEYS}
    r = R.Renderer({k: v.detach() for k, v in params.items()}, cams, scale_mode, K, lut, want_backward=True,
                   headroom=1.5, **(renderer_kwargs or {}))
    opt = torch.optim.Adam([{"params": [params[k]], "lr": lr[k]} for k in R.SCENE_KEYS], eps=1e-15)
    losses, ms, pairs = [], [], []
    for _ in range(steps):
        if timed:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
        img = R.AgsRender.apply(*[params[k] for k in R.SCENE_KEYS], r)
        loss = torch.mean((img - target) ** 2)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        if timed:
            b.record()
        losses.append(float(loss.item()))
        pairs.append(r.pairs())
        if timed:
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    return dict(scene={k: v.detach() for k, v in params.items()}, losses=losses, pairs=pairs, ms=ms)
