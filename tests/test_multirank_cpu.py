"""The benchmark's multi-GPU host logic on two gloo ranks (CPU): each rank holds
the same objects and its own share of the candidates (no data exchange), and the
job time is the slowest rank's."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        w = bench.build_workload("cpu", rank, n_obj=2, per_obj=6, grid_n=12)
        q = torch.tensor(w.q0)
        qs = [torch.empty_like(q) for _ in range(world)]
        dist.all_gather(qs, q)
        g = torch.stack([o["grid"] for o in w.objects])
        gs = [torch.empty_like(g) for _ in range(world)]
        dist.all_gather(gs, g)
        slowest = bench.max_over_ranks(1.5 + rank, world)
        out.put((rank, [x.numpy() for x in qs], [x.numpy() for x in gs], slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_hold_disjoint_candidates_and_report_the_slowest():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, qs, gs, slowest in res:
        assert slowest == 2.5
        np.testing.assert_array_equal(gs[0], gs[1])          # same objects on every rank
        assert qs[0].shape == qs[1].shape
        assert not np.any(np.all(np.isclose(qs[0][:, None, :], qs[1][None, :, :]), axis=-1))   # no shared candidate
