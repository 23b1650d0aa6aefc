"""Multi-GPU partition by object, on two gloo ranks (CPU): each rank builds only the
grids of its own objects and optimises only their candidates, with no exchange in
the step loop; the results gathered on rank 0 equal a one-rank run bit for bit.
On CPU ranks the FP64 oracle stands in for the kernel (the partition and gather
are the benchmark's own host logic)."""

import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

SIZES = dict(n_obj=5, per_obj=3, grid_n=14, points_per_link=8)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_share(w, steps=2):
    """One rank's share: the oracle's optimisation of its candidates (q, last loss)."""
    from oracle import fastgraspd_oracle as O
    S = O.Setup(w.hand, w.objects, w.params)
    return O.optimize(S, w.q0, w.obj_of_cand, 0, steps, w.steps)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    from paper_2306_08132_gb300 import shard
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        w, info = bench.build_workload("cpu", rank, world, "superquadric8", **SIZES)
        q, loss = _run_share(w)
        Q = shard.gather_rows(q, info["candidates"], info["total_candidates"])
        Lo = shard.gather_rows(loss, info["candidates"], info["total_candidates"])
        slowest = bench.max_over_ranks(1.5 + rank, world)
        out.put((rank, info["objects"].tolist(), len(w.objects), info["grid_bytes"], Q, Lo, slowest))
    finally:
        dist.destroy_process_group()


def test_partition_by_object_gathers_the_one_rank_result():
    import bench
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=600) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, objs0, n0, gb0, Q, Lo, s0), (r1, objs1, n1, gb1, Q1, Lo1, s1) = res
    assert s0 == s1 == 2.5                                  # the job's time is the slowest rank's
    assert objs0 == [0, 1, 2] and objs1 == [3, 4]           # disjoint blocks of objects
    assert n0 == 3 and n1 == 2                              # each rank built only its own grids
    assert Q1 is None and Lo1 is None                       # results are gathered on rank 0
    w, info = bench.build_workload("cpu", 0, 1, "superquadric8", **SIZES)
    assert gb0 + gb1 == info["grid_bytes"]
    q, loss = _run_share(w)
    np.testing.assert_array_equal(Q, q)
    np.testing.assert_array_equal(Lo, loss)


def test_object_and_candidate_shards():
    from paper_2306_08132_gb300 import shard
    blocks = [shard.object_shard(10, r, 4).tolist() for r in range(4)]
    assert blocks == [[0, 1, 2], [3, 4, 5], [6, 7], [8, 9]]
    oc = np.array([0, 0, 1, 2, 2, 3, 1, 0], dtype=np.int32)
    cand, local = shard.candidate_shard(oc, np.array([1, 3]))
    assert cand.tolist() == [2, 5, 6] and local.tolist() == [0, 1, 0]
    # one process, no process group: the rows are placed at their candidates
    rows = np.arange(3, dtype=np.float32)[:, None] * np.ones((1, 2), dtype=np.float32)
    full = shard.gather_rows(rows, cand, 8)
    assert full.shape == (8, 2) and full[5, 0] == 1 and full[0, 0] == 0
    with pytest.raises(ValueError):
        shard.object_shard(3, 2, 2)


def test_requests_routed_by_hbm_budget():
    """Serving on several GPUs: each request goes to the GPU where it adds the fewest
    bytes (its object already resident first), then to the one with the most free
    budget; requests that fit nowhere are refused until others release their bytes."""
    from paper_2306_08132_gb300.shard import RequestRouter
    r = RequestRouter([1000, 1000])
    assert r.route(100, "a", 500) == 0                 # both empty: the lower index
    assert r.route(100, "b", 500) == 1                 # GPU 1 has more free budget
    assert r.route(50, "a", 500) == 0                  # object a resident on GPU 0: 50 bytes there
    assert r.used == [650, 600]
    assert r.route(300, "c", 400) is None              # 700 fits neither (350 and 400 left)
    assert r.route(300, "b", 500) == 1                 # b resident on GPU 1
    r.release(0, 100, "a")
    r.release(0, 50, "a")                              # a's last request: its grid leaves GPU 0
    assert r.used == [0, 900] and "a" not in r.objects[0]
    assert r.route(300, "c", 400) == 0
