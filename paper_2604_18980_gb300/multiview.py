"""Host-side logic for rendering and training over many views on several GPUs.

Views are independent in the forward pass (each GPU holds a replica of the
scene and renders its own views; no exchange).  Training over views needs one
exchange: the sum of the per-view parameter gradients.  This module holds the
view partition, that sum, and the data-parallel training step built on them
(`train_step`, with `renderer_grads` as the libags renderer's part); with one
GPU the sum is the identity.
"""
from __future__ import annotations


def shard_views(cams: list, rank: int, world: int) -> list:
    """Contiguous block of views for `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    n = len(cams)
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return cams[lo:hi]


def sum_gradients(grads: dict, group=None) -> dict:
    """All-reduce (sum) every gradient tensor across the process group, in place.

    The tensors of one dtype and device travel in a single flat buffer (one
    collective of 236 B per Gaussian rather than one per attribute)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return grads
    keys = sorted(grads)
    groups = {}
    for k in keys:
        groups.setdefault((grads[k].dtype, grads[k].device), []).append(k)
    for ks in groups.values():
        flat = torch.cat([grads[k].reshape(-1) for k in ks])
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
        off = 0
        for k in ks:
            n = grads[k].numel()
            grads[k].copy_(flat[off:off + n].view_as(grads[k]))
            off += n
    return grads


GRAD_KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def train_step(my_views: list, view_grads, group=None) -> tuple:
    """One data-parallel step over views: `view_grads(my_views)` returns
    (loss, grads) summed over this rank's views -- normally renderer_grads
    over one batched render -- then the loss and every gradient tensor are
    summed over the ranks of `group` (one all-reduce for the gradients, one
    for the loss).  Returns (total loss, gradients of the whole view set)."""
    import torch
    import torch.distributed as dist
    loss, grads = view_grads(my_views)
    grads = {k: grads[k] for k in GRAD_KEYS}
    sum_gradients(grads, group)
    lt = torch.tensor([float(loss)], dtype=torch.float64,
                      device=grads["mean"].device if grads["mean"].is_cuda else "cpu")
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(lt, op=dist.ReduceOp.SUM, group=group)
    return float(lt.item()), grads


def renderer_grads(renderer, targets, inv_count: float):
    """view_grads for train_step over one libags Renderer that holds this
    rank's views: render them (one batch), take L = inv_count * sum (image -
    target)^2 and run the hand-written backward with the pair lists of this
    render (the AdaGScale selection held fixed).  Returns (L, grads)."""
    import torch

    def fn(_views):
        img = renderer.forward_fitted()
        diff = img - targets
        loss = float(torch.sum(diff * diff).item()) * inv_count
        g = renderer.backward(diff * (2.0 * inv_count))
        renderer.check()
        return loss, g
    return fn
