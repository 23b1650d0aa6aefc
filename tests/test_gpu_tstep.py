"""GPU parity of the T-step metric (params.sim_steps = T >= 1: each simulation
runs T PBD steps with the SDF re-queried at the predicted object pose) against
the FP64 oracle's evaluate_tstep, through the C ABI.

Tolerances as for the one-step path: loss 1e-4 relative, gradient and update
1e-3 relative per candidate, compared on candidates whose every decision (over
all steps and simulations) sits outside the guard band."""

import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-4
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def fg():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as m
    return m


def _dev():
    return torch.device("cuda:0")


class Case:
    def __init__(self, fg, w):
        self.w = w
        self.hand = fg.Hand.from_synth(w.hand)
        self.sdfs = [fg.Sdf.from_synth(o) for o in w.objects]
        self.scene = fg.Scene(self.sdfs)
        self.oc = torch.tensor(w.obj_of_cand, device=_dev(), dtype=torch.int32)

    def oracle(self, params):
        return O.Setup(self.w.hand, self.w.objects, params)

    def clean(self, S, q, r):
        mask = np.zeros(len(q), dtype=bool)
        for k in np.unique(self.w.obj_of_cand):
            idx = np.nonzero(self.w.obj_of_cand == k)[0]
            mask[idx] = O.clean_candidates(S.hand, S.objs[int(k)], q[idx], r, S.prm)
        return mask


def _rel_rows(a, b, floor=1e-6):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)


def _compare(loss, grad, ref, clean):
    idx = np.nonzero(clean)[0]
    L = loss.astype(np.float64)[idx]
    lrel = np.abs(L - ref["L"][idx]) / np.maximum(np.abs(ref["L"][idx]), 1e-6)
    grel = _rel_rows(grad.astype(np.float64)[idx], ref["grad"][idx])
    assert lrel.max() < LOSS_TOL, (idx[np.argmax(lrel)], lrel.max())
    assert grel.max() < GRAD_TOL, (idx[np.argmax(grel)], grel.max())


@pytest.fixture(scope="module")
def tiny(fg):
    return Case(fg, synth.tiny_sphere_workload(n_cand=64))


@pytest.mark.parametrize("T,alpha", [(1, 0.1), (2, 0.1), (3, 0.1), (2, 0.0), (8, 0.1)])
def test_tstep_loss_and_grad_match_oracle(fg, tiny, T, alpha):
    w, r = tiny.w, 0.004
    params = dict(w.params, sim_steps=T, alpha_leak=alpha)
    q = torch.tensor(w.q0, device=_dev())
    loss, grad = fg.loss_and_grad(tiny.hand, tiny.scene, q, params, r, obj_of_cand=tiny.oc)
    S = tiny.oracle(params)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    clean = tiny.clean(S, w.q0, r)
    assert clean.sum() >= 0.5 * len(clean), clean.sum()
    assert (ref["N"].sum(axis=1) > 0).sum() >= 8, "workload must exercise contacts"
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_tstep_mixed_objects_four_finger(fg):
    w = synth.batched_superquadric_workload(n_obj=3, per_obj=12, grid_n=48, points_per_link=32, steps=50,
                                            device="cuda")
    case = Case(fg, w)
    params = dict(w.params, sim_steps=2)
    S = case.oracle(params)
    r = O.dilation_radius(S.prm, 7, w.steps)
    loss, grad = fg.loss_and_grad(case.hand, case.scene, torch.tensor(w.q0, device=_dev()), params, r,
                                  obj_of_cand=case.oc)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    clean = case.clean(S, w.q0, r)
    assert clean.sum() >= 0.5 * len(clean)
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_tstep_optimize_step_matches_oracle_and_is_reproducible(fg, tiny):
    w = tiny.w
    params = dict(w.params, sim_steps=2, r0=0.01, schedule="linear")
    S = tiny.oracle(params)
    K = 20
    q0 = torch.tensor(w.q0, device=_dev())
    q1 = q0.clone()
    loss = fg.optimize_step(tiny.hand, tiny.scene, q1, params, 3, K, 1, obj_of_cand=tiny.oc)
    r = O.dilation_radius(S.prm, 3, K)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    step = (q1 - q0).cpu().numpy().astype(np.float64)
    _compare(loss.cpu().numpy(), -step / params["lr"], ref, tiny.clean(S, w.q0, r))
    # nsteps in one launch == repeated launches, bit for bit
    qa = q0.clone()
    la = fg.optimize_step(tiny.hand, tiny.scene, qa, params, 3, K, 3, obj_of_cand=tiny.oc)
    qb = q0.clone()
    for s in range(3):
        lb = fg.optimize_step(tiny.hand, tiny.scene, qb, params, 3 + s, K, 1, obj_of_cand=tiny.oc)
    torch.cuda.synchronize()
    assert torch.equal(qa, qb) and torch.equal(la, lb)
    # loss-only call equals the loss of the gradient call
    l1, _ = fg.loss_and_grad(tiny.hand, tiny.scene, q0, params, 0.004, obj_of_cand=tiny.oc)
    l2, none = fg.loss_and_grad(tiny.hand, tiny.scene, q0, params, 0.004, obj_of_cand=tiny.oc, want_grad=False)
    assert none is None and torch.equal(l1, l2)


def test_tstep_one_step_agrees_with_plane_form_on_flat_contact(fg, tiny):
    """On a linear field the plane linearisation is exact: T = 1 on the GPU gives the
    one-step kernel's loss and gradient to float32 rounding."""
    w = tiny.w
    n0 = np.array([0.48, -0.6, 0.64])
    n0 /= np.linalg.norm(n0)
    obj = synth.linear_grid(tuple(n0), -0.07, 80, 0.008)
    sdf = fg.Sdf.from_synth(obj)
    scene = fg.Scene([sdf])
    q = torch.tensor(w.q0, device=_dev())
    l0, g0 = fg.loss_and_grad(tiny.hand, scene, q, w.params, 0.004)
    l1, g1 = fg.loss_and_grad(tiny.hand, scene, q, dict(w.params, sim_steps=1), 0.004)
    torch.cuda.synchronize()
    L0, L1 = l0.cpu().numpy().astype(np.float64), l1.cpu().numpy().astype(np.float64)
    assert np.abs(L1 - L0).max() <= 1e-5 * np.abs(L0).max()
    rel = _rel_rows(g1.cpu().numpy().astype(np.float64), g0.cpu().numpy().astype(np.float64))
    assert np.median(rel) < 1e-4 and rel.max() < 1e-2


def test_tstep_is_refused_where_only_the_one_step_metric_exists(fg, tiny):
    from paper_2306_08132_gb300 import _lib
    w = tiny.w
    q = torch.tensor(w.q0[:4], device=_dev())
    params = dict(w.params, sim_steps=2)
    with pytest.raises(_lib.FgError) as e:
        fg.contact_wrench(tiny.hand, tiny.scene, q, params, 0.004)
    assert e.value.name == "FG_ERR_INVALID"
    with pytest.raises(_lib.FgError):
        fg.optimize_step_plain(tiny.hand, tiny.scene, q.clone(), params, 0, 10, 1)
    for bad in (-1, 9):
        with pytest.raises(_lib.FgError):
            fg.loss_and_grad(tiny.hand, tiny.scene, q, dict(w.params, sim_steps=bad), 0.004)
