"""The adjoint through torch.autograd (GraspLoss) against central finite
differences of the FP64 oracle, on the 5-finger hand and convex polyhedra
(64 candidates of the polyhedra workload), and the loss-only path."""

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as m
    return m


def _repeat_decisions(dec: O.Decisions, n: int) -> O.Decisions:
    rep = lambda t: t.repeat((n,) + (1,) * (t.dim() - 1))
    out = O.Decisions()
    for k, v in dec.__dict__.items():
        if isinstance(v, dict):
            setattr(out, k, {kk: rep(vv) for kk, vv in v.items()})
        elif isinstance(v, torch.Tensor):
            setattr(out, k, rep(v))
    return out


def _fd_gradient(S, obj, q_row, r, prm, h):
    """Central differences of the oracle's loss with every branch frozen at q_row
    (non-contact constraints as the leaky surrogate anchored at q_row)."""
    q = torch.tensor(q_row[None].astype(np.float64))
    base = O.evaluate(S.hand, obj, q, r, prm)
    D = q.shape[1]
    E = torch.eye(D, dtype=torch.float64) * h
    qp = torch.cat([q + E, q - E])
    dec = _repeat_decisions(base["dec"], 2 * D)
    L = O.evaluate(S.hand, obj, qp, r, prm, dec=dec, anchor_mode=True)["L"]
    return ((L[:D] - L[D:]) / (2 * h)).numpy()


def test_autograd_gradient_matches_oracle_finite_differences(fg):
    w = synth.polyhedra_workload(n_obj=8, per_obj=8, grid_n=128, steps=100, device="cuda")
    S = O.Setup(w.hand, w.objects, w.params)
    hand = fg.Hand.from_synth(w.hand)
    sdfs = [fg.Sdf.from_synth(o) for o in w.objects]
    scene = fg.Scene(sdfs)
    oc = torch.tensor(w.obj_of_cand, device="cuda", dtype=torch.int32)
    r = O.dilation_radius(S.prm, 0, w.steps)
    q = torch.tensor(w.q0, device="cuda", requires_grad=True)
    loss = fg.grasp_loss(q, hand, scene, w.params, r, oc)
    (loss * torch.arange(1, w.B + 1, device="cuda", dtype=torch.float32)).sum().backward()
    weights = np.arange(1, w.B + 1, dtype=np.float64)
    g_gpu = q.grad.cpu().numpy().astype(np.float64) / weights[:, None]
    compared = 0
    for b in range(w.B):
        obj = S.objs[int(w.obj_of_cand[b])]
        if not O.clean_candidates(S.hand, obj, w.q0[b:b + 1], r, S.prm)[0]:
            continue
        # h = 1e-9: points can sit a fraction of a micrometre outside the grid,
        # where the excess-distance term curves like 1/e; FP64 round-off stays ~1e-9
        fd = _fd_gradient(S, obj, w.q0[b], r, S.prm, 1e-9)
        rel = np.linalg.norm(g_gpu[b] - fd) / max(np.linalg.norm(fd), 1e-6)
        assert rel < 1e-3, (b, rel)
        compared += 1
    assert compared >= 40, compared


def test_loss_only_path_equals_loss_with_gradient(fg):
    w = synth.tiny_sphere_workload(n_cand=32)
    hand = fg.Hand.from_synth(w.hand)
    scene = fg.Scene([fg.Sdf.from_synth(w.objects[0])])
    q = torch.tensor(w.q0, device="cuda")
    l1, g = fg.loss_and_grad(hand, scene, q, w.params, 0.004, want_grad=True)
    l2, none = fg.loss_and_grad(hand, scene, q, w.params, 0.004, want_grad=False)
    assert none is None
    assert torch.equal(l1, l2)
    # no gradient requested through autograd: forward only
    l3 = fg.grasp_loss(q, hand, scene, w.params, 0.004)
    assert torch.equal(l1, l3)


def _repeat_tstep_decisions(dec: O.TStepDecisions, n: int) -> O.TStepDecisions:
    rep = lambda t: t.repeat((n,) + (1,) * (t.dim() - 1))
    steps = []
    for sd in dec.steps:
        out = O.StepDecisions()
        for k, v in sd.__dict__.items():
            setattr(out, k, {kk: rep(vv) for kk, vv in v.items()} if isinstance(v, dict) else rep(v))
        steps.append(out)
    return O.TStepDecisions(steps=steps, **{k: rep(getattr(dec, k))
                                           for k in ("v_nz", "w_nz", "range_nz", "above", "below")})


def _fd_tstep(S, obj, q_row, r, T):
    """Richardson-extrapolated central differences (h = 2e-10, 1e-10) of the
    oracle's T-step loss with every branch frozen at q_row."""
    qb = torch.tensor(q_row[None].astype(np.float64))
    base = O.evaluate_tstep(S.hand, obj, qb, r, S.prm, T)
    D = qb.shape[1]
    dec = _repeat_tstep_decisions(base["dec"], 2 * D)
    fd = np.zeros(D)
    for h, wgt in ((2e-10, -1.0 / 3.0), (1e-10, 4.0 / 3.0)):
        E = torch.eye(D, dtype=torch.float64) * h
        L = O.evaluate_tstep(S.hand, obj, torch.cat([qb + E, qb - E]), r, S.prm, T, dec=dec, anchor_mode=True)["L"]
        fd += wgt * ((L[:D] - L[D:]) / (2 * h)).numpy()
    return fd


def test_autograd_tstep_gradient_matches_oracle_finite_differences(fg):
    """The T-step metric (T = 2) through GraspLoss against finite differences of the
    oracle's branch-frozen T-step loss."""
    w = synth.tiny_sphere_workload(n_cand=32)
    params = dict(w.params, sim_steps=2)
    S = O.Setup(w.hand, w.objects, params)
    hand = fg.Hand.from_synth(w.hand)
    scene = fg.Scene([fg.Sdf.from_synth(w.objects[0])])
    q = torch.tensor(w.q0, device="cuda", requires_grad=True)
    fg.grasp_loss(q, hand, scene, params, 0.004).sum().backward()
    g_gpu = q.grad.cpu().numpy().astype(np.float64)
    compared = 0
    for b in range(w.B):
        if not O.clean_candidates(S.hand, S.objs[0], w.q0[b:b + 1], 0.004, S.prm)[0]:
            continue
        fd = _fd_tstep(S, S.objs[0], w.q0[b], 0.004, 2)
        rel = np.linalg.norm(g_gpu[b] - fd) / max(np.linalg.norm(fd), 1e-6)
        assert rel < 1e-3, (b, rel)
        compared += 1
    assert compared >= 16, compared


def test_autograd_gauss_seidel_gradient_matches_oracle_finite_differences(fg):
    """The Gauss-Seidel form through GraspLoss against central finite differences of the
    oracle's branch-frozen Gauss-Seidel loss (non-contact constraints as the leaky
    surrogate with the state frozen at the decision point), on a mesh object."""
    from synth import meshes as SM
    w = synth.tiny_sphere_workload(n_cand=16)
    objs = [SM.icosphere(0.04, 2)]
    params = dict(w.params, gauss_seidel=1)
    S = O.Setup(w.hand, objs, params)
    hand = fg.Hand.from_synth(w.hand)
    scene = fg.Scene([fg.Sdf.from_synth(objs[0])])
    q = torch.tensor(w.q0, device="cuda", requires_grad=True)
    fg.grasp_loss(q, hand, scene, params, 0.004).sum().backward()
    g_gpu = q.grad.cpu().numpy().astype(np.float64)
    compared = 0
    for b in range(w.B):
        if not O.clean_candidates(S.hand, S.objs[0], w.q0[b:b + 1], 0.004, S.prm)[0]:
            continue
        qb = torch.tensor(w.q0[b:b + 1].astype(np.float64))
        base = O.evaluate_gs(S.hand, S.objs[0], qb, 0.004, S.prm)
        if compared < 2 and base["N"].sum() == 0:
            continue                                   # compare the touching candidates first
        h = 1e-8
        D = qb.shape[1]
        E = torch.eye(D, dtype=torch.float64) * h
        rep = lambda t: t.repeat((2 * D,) + (1,) * (t.dim() - 1))
        dec = O.GSDecisions()
        for k, v in base["dec"].__dict__.items():
            if isinstance(v, dict):
                setattr(dec, k, {kk: rep(vv) for kk, vv in v.items()})
            elif isinstance(v, torch.Tensor):
                setattr(dec, k, rep(v))
        L = O.evaluate_gs(S.hand, S.objs[0], torch.cat([qb + E, qb - E]), 0.004, S.prm, dec=dec,
                          anchor_mode=True)["L"]
        fd = ((L[:D] - L[D:]) / (2 * h)).numpy()
        rel = np.linalg.norm(g_gpu[b] - fd) / max(np.linalg.norm(fd), 1e-6)
        assert rel < 1e-3, (b, rel)
        compared += 1
        if compared == 4:
            break
    assert compared >= 3, compared
