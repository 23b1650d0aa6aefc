"""The oracle's flop counter (oracle/flop_count.py): pinned on expressions whose
operation counts are known by hand, then applied to the oracle's step, whose
count must scale with the number of candidates and points and not depend on
which candidates are counted (the oracle evaluates every branch)."""

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O
from oracle.flop_count import FlopCounter, count_step


def test_counter_on_known_expressions():
    x = torch.rand(100, dtype=torch.float64)
    y = torch.rand(100, dtype=torch.float64)
    with FlopCounter() as fc:
        z = x * y + 1.0                       # 100 mul + 100 add
    assert fc.flops == 200 and fc.special == 0
    with FlopCounter() as fc:
        s = x.sum()                           # 99 additions
    assert fc.flops == 99
    a = torch.rand(4, 5, dtype=torch.float64)
    b = torch.rand(5, 3, dtype=torch.float64)
    with FlopCounter() as fc:
        c = a @ b                             # 2 * 4 * 3 * 5
    assert fc.flops == 120
    with FlopCounter() as fc:
        r = torch.sqrt(x) + torch.where(x > 0.5, x, y)   # 100 special + 100 add; where is free
    assert fc.flops == 100 and fc.special == 100
    i = torch.arange(10)
    with FlopCounter() as fc:
        j = i * 3 + 1                          # integer arithmetic is not counted
    assert fc.flops == 0
    del z, s, c, r, j


def test_oracle_count_scales_with_work():
    w = synth.tiny_sphere_workload(n_cand=8)
    S = O.Setup(w.hand, w.objects, w.params)
    r = 0.004
    c2 = count_step(S, w.q0[:2], 0, r)
    c4 = count_step(S, w.q0[:4], 0, r)
    c4b = count_step(S, w.q0[4:8], 0, r)
    assert c4["flops"] > 0
    # per point-step figures agree across batch sizes and across candidates (every
    # branch is evaluated), up to the per-candidate terms (FK, loss) spread over the points
    assert c4["flops_per_point_step"] == pytest.approx(c2["flops_per_point_step"], rel=0.02)
    assert c4b["flops_per_point_step"] == pytest.approx(c4["flops_per_point_step"], rel=0.02)
    fwd = count_step(S, w.q0[:4], 0, r, want_grad=False)
    assert 0 < fwd["flops"] < c4["flops"]


def test_benchmark_constants_are_the_oracle_counts():
    """bench.py's algorithmic work per point-step (the roofline's numerator) is the
    counter's figure for the benchmark hand (4-finger, 4,352 points): the Jacobi,
    Gauss-Seidel and T-step forms; the per-point figure does not depend on the grid size."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w = synth.batched_superquadric_workload(n_obj=1, per_obj=8, grid_n=32, device="cpu")
    forms = [({}, bench.FLOPS_PER_POINT_STEP), ({"gauss_seidel": 1}, bench.GS_FLOPS_PER_POINT_STEP)]
    forms += [({"sim_steps": T}, n) for T, n in bench.TSTEP_FLOPS_PER_POINT_STEP.items()]
    for extra, const in forms:
        S = O.Setup(w.hand, w.objects, dict(w.params, **extra))
        c = count_step(S, w.q0[:2], 0, O.dilation_radius(S.prm, 0, w.steps))
        assert round(c["flops_per_point_step"]) == const, (extra, c["flops_per_point_step"])
