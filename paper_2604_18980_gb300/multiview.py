"""Host-side logic for rendering many views on several GPUs.

Views are independent in the forward pass (each GPU holds a replica of the
scene and renders its own views; no exchange).  Training over views needs one
exchange: the sum of the per-view parameter gradients.  This module holds the
view partition and that sum; with one GPU it is the identity.
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
