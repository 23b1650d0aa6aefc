"""Candidate claiming in the persistent kernels (csrc/fg_work.cuh): CTAs take
candidates from a counter that each launch draws from a pool and leaves at zero.
A counter left dirty, or shared by two launches, would silently skip candidates,
so these tests check that every candidate is computed, bit for bit as in a plain
eager call: across CUDA-graph replays (a captured launch keeps its counter),
across more launches than the pool holds (every counter reused), and with
launches on two streams at once.  Output buffers are filled with NaN before each
launch so that a skipped candidate shows."""

import math

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

NAN = float("nan")


@pytest.fixture(scope="module")
def fg():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as m
    return m


@pytest.fixture(scope="module")
def case(fg):
    w = synth.batched_superquadric_workload(n_obj=2, per_obj=96, grid_n=48, points_per_link=32, steps=50,
                                            device="cuda")
    hand = fg.Hand.from_synth(w.hand)
    sdfs = [fg.Sdf.from_synth(o) for o in w.objects]
    scene = fg.Scene(sdfs)
    q0 = torch.tensor(w.q0, device="cuda")
    oc = torch.tensor(w.obj_of_cand, device="cuda", dtype=torch.int32)
    return w, hand, sdfs, scene, q0, oc


FORMS = {"jacobi": {}, "gauss_seidel": {"gauss_seidel": 1}, "tstep": {"sim_steps": 1}}


@pytest.mark.parametrize("form", list(FORMS))
def test_graph_replays_match_eager(fg, case, form):
    """Two optimisation steps per launch, captured once and replayed three times."""
    w, hand, _, scene, q0, oc = case
    params = dict(w.params, **FORMS[form])
    q_e = q0.clone()
    loss_e = fg.optimize_step(hand, scene, q_e, params, 0, w.steps, 2, obj_of_cand=oc)
    torch.cuda.synchronize()
    assert torch.isfinite(loss_e).all()
    qg = torch.empty_like(q0)
    lg = torch.empty(w.B, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        qg.copy_(q0)
        fg.optimize_step(hand, scene, qg, params, 0, w.steps, 2, obj_of_cand=oc, loss=lg)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        qg.copy_(q0)
        fg.optimize_step(hand, scene, qg, params, 0, w.steps, 2, obj_of_cand=oc, loss=lg)
    for _ in range(3):
        lg.fill_(NAN)
        qg.fill_(NAN)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(lg, loss_e)
        assert torch.equal(qg, q_e)


def test_more_launches_than_the_pool(fg, case):
    """1,100 launches of the fused loss and gradient (the pool holds 1,024 counters),
    each on 5 candidates: every launch computes every candidate, identically."""
    w, hand, _, scene, q0, oc = case
    q = q0[90:95].contiguous()
    o = oc[90:95].contiguous()
    ref_l, ref_g = fg.loss_and_grad(hand, scene, q, w.params, 0.004, obj_of_cand=o)
    torch.cuda.synchronize()
    assert torch.isfinite(ref_l).all() and torch.isfinite(ref_g).all()
    L = torch.full((1100, 5), NAN, device="cuda")
    G = torch.full((1100, 5, q.shape[1]), NAN, device="cuda")
    for i in range(1100):
        l, g = fg.loss_and_grad(hand, scene, q, w.params, 0.004, obj_of_cand=o)
        L[i] = l
        G[i] = g
    torch.cuda.synchronize()
    assert torch.equal(L, ref_l.expand_as(L))
    assert torch.equal(G, ref_g.expand_as(G))


def test_launches_on_two_streams(fg, case):
    """Two candidate sets on two streams, 40 launches each, interleaved: each result
    equals the eager one (each launch draws its own counter)."""
    w, hand, _, scene, q0, oc = case
    half = w.B // 2
    qa, qb = q0[:half].contiguous(), q0[half:].contiguous()
    oa, ob = oc[:half].contiguous(), oc[half:].contiguous()
    ref_a = fg.loss_and_grad(hand, scene, qa, w.params, 0.004, obj_of_cand=oa)[0]
    ref_b = fg.loss_and_grad(hand, scene, qb, w.params, 0.004, obj_of_cand=ob)[0]
    torch.cuda.synchronize()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    sa.wait_stream(torch.cuda.current_stream())
    sb.wait_stream(torch.cuda.current_stream())
    outs_a, outs_b = [], []
    for _ in range(40):
        with torch.cuda.stream(sa):
            outs_a.append(fg.loss_and_grad(hand, scene, qa, w.params, 0.004, obj_of_cand=oa)[0])
        with torch.cuda.stream(sb):
            outs_b.append(fg.loss_and_grad(hand, scene, qb, w.params, 0.004, obj_of_cand=ob)[0])
    torch.cuda.synchronize()
    for la, lb in zip(outs_a, outs_b):
        assert torch.equal(la, ref_a)
        assert torch.equal(lb, ref_b)


def test_quality_kernels_repeat(fg, case):
    """The contact measure and epsilon kernels claim candidates too: repeated
    launches give the same per-candidate results, and every candidate is written."""
    w, hand, _, scene, q0, oc = case
    areas = torch.tensor(w.hand["point_area"], device="cuda")
    dirs = torch.tensor(synth.unit_directions(256), device="cuda")
    ca0 = fg.contact_measure(hand, scene, q0, areas, 0.005, obj_of_cand=oc)
    e0, n0 = fg.grasp_epsilon(hand, scene, q0, 0.005, 0.5, 8, 1.0 / 0.08, dirs, obj_of_cand=oc)
    torch.cuda.synchronize()
    assert torch.isfinite(ca0).all() and (n0 >= 0).all()
    for _ in range(5):
        ca = fg.contact_measure(hand, scene, q0, areas, 0.005, obj_of_cand=oc)
        e, n = fg.grasp_epsilon(hand, scene, q0, 0.005, 0.5, 8, 1.0 / 0.08, dirs, obj_of_cand=oc)
        torch.cuda.synchronize()
        assert torch.equal(ca, ca0)
        assert torch.equal(n, n0)
        assert torch.equal(torch.nan_to_num(e, nan=math.inf), torch.nan_to_num(e0, nan=math.inf))


def test_graph_replays_beside_more_eager_launches_than_the_pool(fg, case):
    """A captured launch keeps its counter on every replay; eager launches cycle
    through the pool.  Captured launches draw from a range that eager launches never
    use, so a graph replayed on one stream while 1,100 eager launches (more than the
    pool's 1,024 counters) run on another stream still computes every candidate of
    both, bit for bit as serial calls do."""
    w, hand, _, scene, q0, oc = case
    qa, oa = q0[:64].contiguous(), oc[:64].contiguous()
    qb, ob = q0[90:95].contiguous(), oc[90:95].contiguous()
    ref_a = fg.loss_and_grad(hand, scene, qa, w.params, 0.004, obj_of_cand=oa)
    ref_b = fg.loss_and_grad(hand, scene, qb, w.params, 0.004, obj_of_cand=ob)
    torch.cuda.synchronize()
    la = torch.empty(64, device="cuda")
    ga = torch.empty_like(qa)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s1):
        l, g_ = fg.loss_and_grad(hand, scene, qa, w.params, 0.004, obj_of_cand=oa)    # warm before capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s1):
        l, g_ = fg.loss_and_grad(hand, scene, qa, w.params, 0.004, obj_of_cand=oa)
        la.copy_(l)
        ga.copy_(g_)
    torch.cuda.synchronize()
    outs_a, outs_b = [], []
    for i in range(1100):
        with torch.cuda.stream(s2):
            outs_b.append(fg.loss_and_grad(hand, scene, qb, w.params, 0.004, obj_of_cand=ob))
        if i % 25 == 0:
            with torch.cuda.stream(s1):
                la.fill_(NAN)
                ga.fill_(NAN)
                graph.replay()
                outs_a.append((la.clone(), ga.clone()))
    torch.cuda.synchronize()
    assert len(outs_a) == 44
    for l_, g_ in outs_a:
        assert torch.equal(l_, ref_a[0]) and torch.equal(g_, ref_a[1])
    for l_, g_ in outs_b:
        assert torch.equal(l_, ref_b[0]) and torch.equal(g_, ref_b[1])
