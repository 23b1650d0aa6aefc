"""Request queue (continuous batching) on the GPU: results match direct steps,
a request's result is the same alone and in a mix, admission respects the HBM
budget, and errors are reported without hanging."""

import time

import numpy as np
import pytest
import torch

import synth
from synth.workloads import build_request

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as m
    return m


def _queue_config_index(fg):
    """Configuration the queue's kernel uses (4 warps, >= 5 CTAs per SM, 1 point per thread)."""
    return fg.fused_configs().index((4, 5, 1))


@pytest.fixture(scope="module")
def requests(fg):
    """Three requests with different hands, objects and sizes (serving-stream shapes)."""
    specs = synth.serving_stream(n_requests=3, grid_sizes=(32, 48), cand_range=(17, 90), step_range=(7, 23))
    kinds = [3, 4, 5]
    out = []
    for spec, kind in zip(specs, kinds):
        spec = dict(spec, hand_kind=kind)
        hand_d, obj, q0, params, steps = build_request(spec, device="cuda")
        out.append((fg.Hand.from_synth(hand_d), fg.Sdf.from_synth(obj), q0, params, steps))
    return out


def _run(fg, queue, reqs):
    ids = [queue.submit(h, s, q0, steps, p) for (h, s, q0, p, steps) in reqs]
    res = []
    for rid in ids:
        queue.wait(rid, 120000)
        res.append(queue.result(rid))
    return res


def test_single_request_matches_direct_steps(fg, requests):
    hand, sdf, q0, params, steps = requests[1]
    q_direct = torch.tensor(q0, device="cuda")
    fg.fused_config_select(_queue_config_index(fg))
    try:
        scene = fg.Scene([sdf])
        loss = fg.optimize_step(hand, scene, q_direct, params, 0, steps, steps)
    finally:
        fg.fused_config_select(-1)
    torch.cuda.synchronize()
    queue = fg.Queue(1 << 30, steps_per_launch=4)
    try:
        (q, l, lat), = _run(fg, queue, [requests[1]])
    finally:
        queue.close()
    np.testing.assert_array_equal(q, q_direct.cpu().numpy())
    np.testing.assert_array_equal(l, loss.cpu().numpy())
    assert lat > 0


def test_result_alone_equals_result_in_mix(fg, requests):
    """Each request alone, then all three together (different hands, grids, B,
    step counts and therefore different rounds): identical results."""
    alone = []
    for r in requests:
        queue = fg.Queue(1 << 30, steps_per_launch=5)
        try:
            alone.append(_run(fg, queue, [r])[0])
        finally:
            queue.close()
    queue = fg.Queue(1 << 30, steps_per_launch=5)
    try:
        mixed = _run(fg, queue, requests)
        st = queue.stats()
    finally:
        queue.close()
    for (qa, la, _), (qm, lm, _) in zip(alone, mixed):
        np.testing.assert_array_equal(qa, qm)
        np.testing.assert_array_equal(la, lm)
    # the mix shared rounds: fewer rounds than the three runs alone
    assert st["rounds"] < sum(-(-r[4] // 5) for r in requests)


def test_admission_respects_budget(fg, requests):
    """With room for one request's state and object but not a second state, the
    requests run one at a time, bytes in use never exceed the budget and drop to
    0 at the end; a request that could never fit is refused at submit."""
    from paper_2306_08132_gb300 import _lib
    hand, sdf, q0, params, steps = requests[0]
    state = 4 * q0.shape[0] * (hand.D + 1)
    queue = fg.Queue(1 << 30, steps_per_launch=1)
    try:
        rid = queue.submit(hand, sdf, q0, 300, params)
        in_use = 0
        for _ in range(20000):
            in_use = queue.stats()["bytes_in_use"]
            if in_use:
                break
            time.sleep(0.0002)
        queue.wait(rid, 120000)
        queue.result(rid)
        assert queue.stats()["bytes_in_use"] == 0
    finally:
        queue.close()
    assert in_use > state                       # the object's grid and pyramid are counted
    budget = in_use + state // 2
    queue = fg.Queue(budget, steps_per_launch=2)
    try:
        ids = [queue.submit(hand, sdf, q0, steps, params) for _ in range(3)]
        peak, done = 0, set()
        while len(done) < 3:
            st = queue.stats()
            assert st["bytes_in_use"] <= budget
            peak = max(peak, st["active"])
            for rid in ids:
                if rid not in done and queue.poll(rid):
                    done.add(rid)
            time.sleep(0.0002)
        assert peak == 1
        for rid in ids:
            queue.result(rid)
        assert queue.stats()["bytes_in_use"] == 0
        big = np.repeat(q0, 1 + budget // state, axis=0)
        with pytest.raises(_lib.FgError) as e:
            queue.submit(hand, sdf, big, steps, params)
        assert e.value.name == "FG_ERR_BUDGET"
    finally:
        queue.close()


def test_queue_errors_and_destroy(fg, requests):
    from paper_2306_08132_gb300 import _lib
    hand, sdf, q0, params, steps = requests[2]
    queue = fg.Queue(1 << 30, steps_per_launch=1)
    rid = queue.submit(hand, sdf, q0, 400, params)
    with pytest.raises(_lib.FgError) as e:
        queue.result(rid)                         # not finished yet
    assert e.value.name == "FG_ERR_BUSY"
    with pytest.raises(_lib.FgError) as e:
        queue.wait(rid, 1)
    assert e.value.name == "FG_ERR_TIMEOUT"
    with pytest.raises(_lib.FgError) as e:
        queue.poll(987654321)
    assert e.value.name == "FG_ERR_NOT_FOUND"
    for _ in range(5):
        queue.submit(hand, sdf, q0, 400, params)
    t0 = time.time()
    queue.close()                                # drops waiting work, finishes the round in flight
    assert time.time() - t0 < 30


def test_mesh_request_in_the_mix(fg, requests):
    """A request on a mesh object (Phong SDF) and a grid request: each result alone and
    in the mix.  The mix runs in the kernel that dispatches per object kind; the mesh
    request runs in it either way (identical results), the grid request's result may
    differ from its grid-only run by float32 rounding only."""
    from synth import meshes as SM
    w = synth.tiny_sphere_workload(n_cand=20)
    mesh_req = (fg.Hand.from_synth(w.hand), fg.Sdf.from_synth(SM.icosphere(0.04, 3)), w.q0, w.params, 9)
    h, s, q0, p, _ = requests[1]
    reqs = [mesh_req, (h, s, q0, p, 1)]        # one step: the two kernels start from the same state
    alone = []
    for r in reqs:
        queue = fg.Queue(1 << 30, steps_per_launch=4)
        try:
            alone.append(_run(fg, queue, [r])[0])
        finally:
            queue.close()
    queue = fg.Queue(1 << 30, steps_per_launch=4)
    try:
        mixed = _run(fg, queue, reqs)
    finally:
        queue.close()
    np.testing.assert_array_equal(alone[0][0], mixed[0][0])
    np.testing.assert_array_equal(alone[0][1], mixed[0][1])
    np.testing.assert_allclose(mixed[1][0], alone[1][0], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(mixed[1][1], alone[1][1], rtol=1e-4)
    assert np.isfinite(mixed[0][0]).all() and np.isfinite(mixed[0][1]).all()


def test_round_time_limit_fails_the_round_and_destroy_returns(fg, requests):
    """A queue whose round limit (timeout_ms = 1) is far below one round's duration
    (2,048 candidates of the 5-finger hand for 200 steps, tens of milliseconds): the
    round's request fails with FG_ERR_TIMEOUT, the queue refuses further work, and
    fg_queue_destroy returns (it waits for the still-running round with a bounded
    wait and frees its state).  Nothing on the GPU waits: the kernel finishes its
    round on its own.  The device then serves a fresh queue normally."""
    from paper_2306_08132_gb300 import _lib
    hand, sdf, q0, params, _ = requests[2]
    big = np.repeat(q0, -(-2048 // len(q0)), axis=0)[:2048]
    queue = fg.Queue(1 << 30, steps_per_launch=200, timeout_ms=1)
    try:
        rid = queue.submit(hand, sdf, big, 400, params)
        queue.wait(rid, 60000)
        with pytest.raises(_lib.FgError) as e:
            queue.result(rid)
        assert e.value.name == "FG_ERR_TIMEOUT"
        with pytest.raises(_lib.FgError) as e:
            queue.submit(hand, sdf, q0, 5, params)
        assert e.value.name == "FG_ERR_CUDA" and "timeout_ms" in str(e.value)
        assert queue.stats()["failed"] == 1
    finally:
        t0 = time.time()
        queue.close()
        assert time.time() - t0 < 30
    torch.cuda.synchronize()
    queue = fg.Queue(1 << 30, steps_per_launch=5)
    try:
        rid = queue.submit(hand, sdf, q0, 5, params)
        queue.wait(rid, 60000)
        q, loss, _ = queue.result(rid)
        assert np.isfinite(q).all() and np.isfinite(loss).all()
    finally:
        queue.close()


def test_allocation_failures_are_reported_cleanly(fg, requests):
    """The library's allocation-failure injection: a hand, an object, a request's host
    copy and a request's device state at admission each fail with FG_ERR_OOM when
    their allocation fails, leave nothing half-built, and the next attempt succeeds;
    the queue keeps serving after a request failed at admission."""
    from paper_2306_08132_gb300 import _lib
    w = synth.tiny_sphere_workload(n_cand=8)
    try:
        for make in (lambda: fg.Hand.from_synth(w.hand), lambda: fg.Sdf.from_synth(w.objects[0])):
            fg.test_fail_allocation(0)
            with pytest.raises(_lib.FgError) as e:
                make()
            assert e.value.name == "FG_ERR_OOM"
            assert make() is not None                # disarmed after one failure
        hand, sdf, q0, params, _ = requests[0]
        queue = fg.Queue(1 << 30, steps_per_launch=5)
        try:
            fg.test_fail_allocation(0)               # the submit's host copy
            with pytest.raises(_lib.FgError) as e:
                queue.submit(hand, sdf, q0, 5, params)
            assert e.value.name == "FG_ERR_OOM"
            fg.test_fail_allocation(1)               # the submit passes, its admission fails
            rid = queue.submit(hand, sdf, q0, 5, params)
            queue.wait(rid, 60000)
            with pytest.raises(_lib.FgError) as e:
                queue.result(rid)
            assert e.value.name == "FG_ERR_OOM"
            assert queue.stats()["bytes_in_use"] == 0
            rid = queue.submit(hand, sdf, q0, 5, params)
            queue.wait(rid, 60000)
            q, loss, _ = queue.result(rid)
            assert np.isfinite(q).all()
        finally:
            queue.close()
    finally:
        fg.test_fail_allocation(-1)
