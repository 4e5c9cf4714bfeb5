"""Multi-process paths on the CPU with gloo (world size 2).

* Camera sharding (the operator's natural multi-GPU split): each rank computes
  its camera subset, one sum all-reduce of the partial outputs equals the
  unsharded result; feature gradients of a camera stay on its rank and equal
  the matching rows of the unsharded gradient.  Each rank's compute here is
  the FP64 oracle (no GPU on this host); on a GPU it is msda.forward.
* The benchmark's timing reduction: the job time is the max over ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2601_10819_gb300 import inputs, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sharded(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        oracle.build()
        gen = torch.Generator().manual_seed(7)
        maps = [[(9, 11), (5, 6)], [(7, 7), (4, 4)], [(12, 5), (6, 3)], [(6, 10), (3, 5)], [(8, 8), (4, 4)]]
        pr = inputs.make_problem(gen, B=2, cam_maps=maps, C=16, G=4, A=9, P=3, loc_range=(-0.2, 1.2))
        cams = shard.split_cameras(len(maps), world)[rank]
        sub = shard.shard_problem(*pr.tensors(), cams)
        part = torch.from_numpy(oracle.forward(*sub))
        shard.reduce_partials(part)
        gf, gl, gw = oracle.backward(*sub, pr.grad_out)
        if rank == 0:
            full = oracle.forward(*pr.tensors())
            q.put(("out", float(np.abs(part.numpy() - full).max() / np.abs(full).max())))
        # feature-gradient rows of this rank's maps equal the unsharded gradient's rows
        fgf, fgl, fgw = oracle.backward(*pr.tensors(), pr.grad_out)
        rows = []
        for k in cams:
            for s in range(pr.spatial_shape.shape[1]):
                h, w = int(pr.spatial_shape[k, s, 0]), int(pr.spatial_shape[k, s, 1])
                st = int(pr.scale_start_index[k, s])
                rows.extend(range(st, st + h * w))
        q.put((f"dfeat{rank}", float(np.abs(gf - fgf[:, rows]).max())))
        q.put((f"dw{rank}", float(np.abs(gw - fgw[:, :, :, cams]).max())))
        q.put((f"dloc{rank}", float(np.abs(gl - fgl[:, :, :, cams]).max())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_camera_sharding_all_reduce_matches_unsharded():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    res = {}
    while not q.empty():
        k, v = q.get()
        res[k] = v
    assert res["out"] <= 1e-13
    for r in range(2):
        assert res[f"dfeat{r}"] <= 1e-13 and res[f"dw{r}"] <= 1e-13 and res[f"dloc{r}"] <= 1e-13


def test_split_cameras_covers_each_camera_once():
    for ncam in (0, 1, 5, 64, 96):
        for world in (1, 2, 3, 8):
            parts = shard.split_cameras(ncam, world)
            assert len(parts) == world
            assert sorted(k for p in parts for k in p) == list(range(ncam))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def _bench_split(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        oracle.build()
        gen = torch.Generator().manual_seed(8)
        maps = [[(9, 11), (5, 6)], [(7, 7), (4, 4)], [(12, 5), (6, 3)], [(6, 10), (3, 5)], [(8, 8), (4, 4)]]
        pr = inputs.make_problem(gen, B=2, cam_maps=maps, C=16, G=4, A=9, P=3, loc_range=(-0.2, 1.2))
        cams, sub = bench.split_shard(pr.tensors(), rank, world)
        fwd = lambda *t: torch.from_numpy(oracle.forward(*t))  # noqa: E731  the kernels' stand-in on a CPU
        bwd = lambda *t: oracle.backward(*t)  # noqa: E731
        out, (gf, gl, gw) = bench.split_step(sub, pr.grad_out, fwd, bwd)
        full = oracle.forward(*pr.tensors())
        fgf, fgl, fgw = oracle.backward(*pr.tensors(), pr.grad_out)
        q.put((f"out{rank}", float(np.abs(out.numpy() - full).max() / np.abs(full).max())))
        q.put((f"cams{rank}", cams))
        q.put((f"dloc{rank}", float(np.abs(gl - fgl[:, :, :, cams]).max())))
        q.put((f"dw{rank}", float(np.abs(gw - fgw[:, :, :, cams]).max())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_bench_camera_split_step():
    """bench.py --split cameras: every rank ends the forward with the frame's output (its shard's partial
    output plus the other rank's, one sum all-reduce) and holds its cameras' gradients."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_split, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    res = {}
    while not q.empty():
        k, v = q.get()
        res[k] = v
    assert sorted(res["cams0"] + res["cams1"]) == list(range(5))
    for r in range(2):
        assert res[f"out{r}"] <= 1e-13
        assert res[f"dloc{r}"] <= 1e-13 and res[f"dw{r}"] <= 1e-13


def _timing(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        vals = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 3.0], torch.device("cpu"))
        q.put((rank, vals))
    finally:
        dist.destroy_process_group()


def test_bench_time_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_timing, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get() for _ in range(2))
    assert got[0] == got[1] == [2.0, 5.0, 3.0]
