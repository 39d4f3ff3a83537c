"""Multi-rank view sharding and gradient sum, world size 2 over gloo on CPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2604_18980_gb300.multiview import shard_views, sum_gradients, train_step

KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def test_shard_views_partition():
    cams = list(range(10))
    for world in (1, 2, 3, 4, 7, 10, 12):
        parts = [shard_views(cams, r, world) for r in range(world)]
        assert sum(parts, []) == cams
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_views(cams, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import oracle
    from paper_2604_18980_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scene, cams, _ = synth.workload("c1_cube16k_256", n=300, width=48, height=40, views=4)
    mine = shard_views(list(range(len(cams))), rank, world)
    acc = None
    rng = np.random.default_rng(0)
    ws = [rng.normal(size=(3, 40, 48)) for _ in cams]
    for v in mine:
        cam = cams[v]
        par = oracle.params(cam)
        oo = oracle.render(scene, cam, par)
        g = oracle.backward(scene, cam, par, oo["tile_start"], oo["ids"], ws[v])
        acc = g if acc is None else {k: acc[k] + g[k] for k in KEYS}
    grads = {k: torch.from_numpy(np.ascontiguousarray(acc[k])) for k in KEYS}
    sum_gradients(grads)
    if rank == 0:
        torch.save(grads, out_path)
    dist.barrier()
    dist.destroy_process_group()


def test_gradient_sum_over_two_ranks(tmp_path):
    import oracle
    from paper_2604_18980_gb300 import synth
    out = str(tmp_path / "g.pt")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = torch.load(out)
    scene, cams, _ = synth.workload("c1_cube16k_256", n=300, width=48, height=40, views=4)
    rng = np.random.default_rng(0)
    ws = [rng.normal(size=(3, 40, 48)) for _ in cams]
    ref = None
    for v, cam in enumerate(cams):
        par = oracle.params(cam)
        oo = oracle.render(scene, cam, par)
        g = oracle.backward(scene, cam, par, oo["tile_start"], oo["ids"], ws[v])
        ref = g if ref is None else {k: ref[k] + g[k] for k in KEYS}
    for k in got:
        np.testing.assert_allclose(got[k].numpy(), ref[k], rtol=1e-12, atol=1e-14)


def _oracle_view_grads(scene, cams, targets, inv_count):
    """view_grads for train_step with the FP64 oracle standing in for the renderer."""
    import oracle

    def fn(views):
        loss, acc = 0.0, None
        for v in views:
            cam = cams[v]
            par = oracle.params(cam, scale_mode=1, K=0.2)
            oo = oracle.render(scene, cam, par)
            diff = oo["image"] - targets[v]
            loss += float((diff * diff).sum()) * inv_count
            g = oracle.backward(scene, cam, par, oo["tile_start"], oo["ids"], 2.0 * inv_count * diff)
            acc = {k: g[k] for k in KEYS} if acc is None else {k: acc[k] + g[k] for k in KEYS}
        return loss, {k: torch.from_numpy(np.ascontiguousarray(acc[k])) for k in KEYS}
    return fn


def _train_problem():
    import oracle
    from paper_2604_18980_gb300 import synth
    scene, cams, _ = synth.workload("c1_cube16k_256", n=300, width=48, height=40, views=5)
    pert = synth.perturb_scene(scene, 9)
    targets = [oracle.render(pert, c, oracle.params(c))["image"] for c in cams]
    return scene, cams, targets, 1.0 / (len(cams) * 3 * 40 * 48)


def _train_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scene, cams, targets, inv = _train_problem()
    mine = shard_views(list(range(len(cams))), rank, world)
    loss, grads = train_step(mine, _oracle_view_grads(scene, cams, targets, inv))
    if rank == 0:
        torch.save(dict(loss=loss, grads=grads), out_path)
    dist.barrier()
    dist.destroy_process_group()


def test_train_step_over_two_ranks_equals_one(tmp_path):
    """Views sharded over two gloo ranks (3 + 2 of 5): the all-reduced loss and
    gradients equal one process's step over all five views."""
    out = str(tmp_path / "t.pt")
    mp.start_processes(_train_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = torch.load(out)
    scene, cams, targets, inv = _train_problem()
    loss, ref = train_step(list(range(len(cams))), _oracle_view_grads(scene, cams, targets, inv))
    assert abs(got["loss"] - loss) <= 1e-12 * abs(loss)
    for k in KEYS:
        np.testing.assert_allclose(got["grads"][k].numpy(), ref[k].numpy(), rtol=1e-12, atol=1e-14)
