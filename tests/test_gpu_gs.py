"""GPU parity of the Gauss-Seidel form (params.gauss_seidel = 1: each simulation
projects the constraints one after another in point order, Sec. III-C) against
the FP64 oracle's evaluate_gs, through the C ABI.

Tolerances as for the Jacobi form: loss 1e-4 relative, gradient and update 1e-3
relative per candidate, on candidates whose every decision (constraint values,
friction regimes and tangential directions at the state the sweep reaches each
point with) sits outside the guard band."""

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
    return Case(fg, synth.tiny_sphere_workload(n_cand=48))


@pytest.mark.parametrize("alpha,w_pen", [(0.1, 0.0), (0.0, 0.0), (0.1, 2.0)])
def test_gs_loss_and_grad_match_oracle(fg, tiny, alpha, w_pen):
    w, r = tiny.w, 0.004
    params = dict(w.params, gauss_seidel=1, alpha_leak=alpha, w_pen=w_pen)
    q = torch.tensor(w.q0, device=_dev())
    loss, grad = fg.loss_and_grad(tiny.hand, tiny.scene, q, params, r, obj_of_cand=tiny.oc)
    S = tiny.oracle(params)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    clean = tiny.clean(S, w.q0, r)
    assert clean.sum() >= 0.5 * len(clean), clean.sum()
    assert (ref["N"] >= 2).any(axis=1).sum() >= 8, "workload must chain several projections"
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)
    # the Gauss-Seidel loss is not the Jacobi loss on candidates with chained contacts
    lj, _ = fg.loss_and_grad(tiny.hand, tiny.scene, q, dict(params, gauss_seidel=0), r, obj_of_cand=tiny.oc)
    chained = (ref["N"] >= 2).any(axis=1) & clean
    assert (np.abs(lj.cpu().numpy() - loss.cpu().numpy())[chained] > 1e-3).any()


def test_gs_mixed_objects_four_finger(fg):
    """Three superquadrics in one batch, 4-finger hand (17 links, 32 points per link)."""
    w = synth.batched_superquadric_workload(n_obj=3, per_obj=10, grid_n=48, points_per_link=32, steps=50,
                                            device="cuda")
    case = Case(fg, w)
    params = dict(w.params, gauss_seidel=1)
    S = case.oracle(params)
    r = O.dilation_radius(S.prm, 7, w.steps)
    loss, grad = fg.loss_and_grad(case.hand, case.scene, torch.tensor(w.q0, device=_dev()), params, r,
                                  obj_of_cand=case.oc)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    clean = case.clean(S, w.q0, r)
    assert clean.sum() >= 0.5 * len(clean)
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_gs_five_finger_polyhedra(fg):
    """5-finger hand (23 links, 64 points per link: 47 chunks) on convex polyhedra."""
    w = synth.polyhedra_workload(n_obj=2, per_obj=6, grid_n=48, points_per_link=64, steps=20, device="cuda")
    case = Case(fg, w)
    params = dict(w.params, gauss_seidel=1)
    S = case.oracle(params)
    r = O.dilation_radius(S.prm, 2, w.steps)
    loss, grad = fg.loss_and_grad(case.hand, case.scene, torch.tensor(w.q0, device=_dev()), params, r,
                                  obj_of_cand=case.oc)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    clean = case.clean(S, w.q0, r)
    assert clean.sum() >= 0.5 * len(clean)
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_gs_optimize_step_matches_oracle_and_is_reproducible(fg, tiny):
    w = tiny.w
    params = dict(w.params, gauss_seidel=1, r0=0.01, schedule="linear")
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


def test_gs_single_contact_equals_jacobi_on_the_gpu(fg, tiny):
    """Candidates on which both forms see the same at most one contact per simulation
    give the Jacobi kernel's loss to float32 rounding (the two forms coincide there).
    A single Gauss-Seidel projection alone is not enough: it can resolve points that
    the Jacobi form, evaluating every point at the predicted pose, counts too."""
    w, r = tiny.w, 0.004
    params = dict(w.params, gauss_seidel=1)
    S = tiny.oracle(params)
    Sj = tiny.oracle(w.params)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    refj = O.batch_loss_and_grad(Sj, w.q0, w.obj_of_cand, r)
    single = ((ref["N"] <= 1).all(axis=1) & (refj["N"] <= 1).all(axis=1) &
              (ref["kappa"] == refj["kappa"]).all(axis=(1, 2)) & tiny.clean(S, w.q0, r) & tiny.clean(Sj, w.q0, r))
    assert single.sum() >= 2
    q = torch.tensor(w.q0, device=_dev())
    lg, _ = fg.loss_and_grad(tiny.hand, tiny.scene, q, params, r, obj_of_cand=tiny.oc)
    lj, _ = fg.loss_and_grad(tiny.hand, tiny.scene, q, w.params, r, obj_of_cand=tiny.oc)
    a, b = lg.cpu().numpy()[single], lj.cpu().numpy()[single]
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


def test_gs_is_refused_where_unsupported(fg, tiny):
    from paper_2306_08132_gb300 import _lib
    w = tiny.w
    q = torch.tensor(w.q0[:4], device=_dev())
    params = dict(w.params, gauss_seidel=1)
    with pytest.raises(_lib.FgError) as e:
        fg.optimize_step_plain(tiny.hand, tiny.scene, q.clone(), params, 0, 10, 1)
    assert e.value.name == "FG_ERR_INVALID"
    with pytest.raises(_lib.FgError):
        fg.contact_wrench(tiny.hand, tiny.scene, q, dict(params, sim_steps=1), 0.004)
    with pytest.raises(_lib.FgError):
        fg.loss_and_grad(tiny.hand, tiny.scene, q, dict(params, sim_steps=2), 0.004)
    with pytest.raises(_lib.FgError):
        fg.loss_and_grad(tiny.hand, tiny.scene, q, dict(params, gauss_seidel=2), 0.004)
    qu = fg.Queue(1 << 30)
    try:
        with pytest.raises(_lib.FgError):
            qu.submit(tiny.hand, tiny.sdfs[0], w.q0[:4], 10, params)
    finally:
        qu.close()


def test_gs_ragged_hand_and_edge_cases(fg):
    """Links whose point ranges are not 32-aligned (chunks straddle links and are never
    culled), a last chunk of 18 points; an empty batch, a hand far from the object
    (6V/7 exactly), object indices outside the scene (NaN, q left alone)."""
    w = synth.tiny_sphere_workload(n_cand=24)
    h = synth.make_hand(3, 21)                          # P = 210
    qs = synth.sample_candidates(np.random.default_rng(7), h, 24, 0.095)
    w2 = synth.Workload("ragged", h, w.objects, qs, np.zeros(24, dtype=np.int32), w.params, 10)
    case = Case(fg, w2)
    params = dict(w.params, gauss_seidel=1)
    S = case.oracle(params)
    loss, grad = fg.loss_and_grad(case.hand, case.scene, torch.tensor(qs, device=_dev()), params, 0.004)
    ref = O.batch_loss_and_grad(S, qs, w2.obj_of_cand, 0.004)
    clean = case.clean(S, qs, 0.004)
    assert clean.sum() >= 12 and (ref["N"][clean] > 0).any()
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)
    e = torch.zeros(0, h["D"], device=_dev())
    l0, _ = fg.loss_and_grad(case.hand, case.scene, e, params, 0.004)
    assert l0.numel() == 0
    far = np.zeros((3, h["D"]), dtype=np.float32)
    far[:, 0] = [0.5, -0.4, 0.3]
    far[:, 6:] = 0.5 * (h["q_low"] + h["q_up"])
    lf, gf = fg.loss_and_grad(case.hand, case.scene, torch.tensor(far, device=_dev()), params, 0.004)
    assert np.allclose(lf.cpu().numpy(), 6.0 / 7.0, rtol=1e-6)
    bad = torch.tensor([0, 3, -1], device=_dev(), dtype=torch.int32)
    qq = torch.tensor(qs[:3], device=_dev())
    lb, _ = fg.loss_and_grad(case.hand, case.scene, qq, params, 0.004, obj_of_cand=bad)
    lb = lb.cpu().numpy()
    assert np.isfinite(lb[0]) and np.isnan(lb[1]) and np.isnan(lb[2])
    q2 = qq.clone()
    fg.optimize_step(case.hand, case.scene, q2, params, 0, 10, 2, obj_of_cand=bad)
    assert torch.equal(q2[1:], qq[1:])


def test_gs_on_mesh_objects(fg):
    """The paper's own combination: the Phong SDF of a mesh (an icosphere and a
    superquadric mesh in one batch) with the Gauss-Seidel projection."""
    from synth import meshes as SM
    w = synth.tiny_sphere_workload(n_cand=32)
    rng = np.random.default_rng(5)
    objects = [SM.icosphere(0.04, 3), SM.random_superquadric_mesh(rng, 16, 32)]
    oc = np.repeat(np.arange(2, dtype=np.int32), 16)
    w2 = synth.Workload("gs-mesh", w.hand, objects, w.q0, oc, w.params, 10)
    case = Case(fg, w2)
    params = dict(w.params, gauss_seidel=1)
    S = case.oracle(params)
    loss, grad = fg.loss_and_grad(case.hand, case.scene, torch.tensor(w.q0, device=_dev()), params, 0.004,
                                  obj_of_cand=case.oc)
    ref = O.batch_loss_and_grad(S, w.q0, oc, 0.004)
    clean = case.clean(S, w.q0, 0.004)
    assert clean.sum() >= 12 and (ref["N"][clean] >= 2).any()
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_gs_contact_wrench_matches_oracle(fg, tiny):
    """fg_contact_wrench in the Gauss-Seidel form: per simulation the sums of the applied
    corrections (f, d x f), the number of points projected and their bits, against the
    oracle's sweep (counts and bits bit-exact on clean candidates)."""
    w, r = tiny.w, 0.004
    params = dict(w.params, gauss_seidel=1)
    S = tiny.oracle(params)
    W, N, bits = fg.contact_wrench(tiny.hand, tiny.scene, torch.tensor(w.q0, device=_dev()), params, r,
                                   obj_of_cand=tiny.oc, want_bits=True)
    torch.cuda.synchronize()
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    clean = tiny.clean(S, w.q0, r)
    assert clean.sum() >= 0.5 * len(clean) and (ref["N"][clean] >= 2).any()
    Wg, Ng, bw = W.cpu().numpy().astype(np.float64), N.cpu().numpy(), bits.cpu().numpy().view(np.uint32)
    P = w.hand["P"]
    for b in np.nonzero(clean)[0]:
        assert np.array_equal(Ng[b], ref["N"][b].astype(np.int32)), b
        for m in range(7):
            got = np.unpackbits(bw[b, m].view(np.uint8), bitorder="little")[:P].astype(bool)
            assert np.array_equal(got, ref["kappa"][b][:, m]), (b, m)
        nrm = np.linalg.norm(ref["W"][b])
        assert nrm == 0 or np.linalg.norm(Wg[b] - ref["W"][b]) / nrm < GRAD_TOL, b
