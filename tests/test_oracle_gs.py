"""Pins of the oracle's Gauss-Seidel form (Sec. III-C: a Gauss-Seidel step over the
constraints of Eq. 1) against closed forms, the Jacobi form where the two must
agree, and finite differences of the frozen-branch loss (no GPU)."""

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O

from test_oracle_pins import multi_point_hand, obj_from

F64 = torch.float64


@pytest.fixture(scope="module")
def plane():
    """phi = z: the object fills z < 0 and the contact normal is +z everywhere."""
    return synth.linear_grid((0.0, 0.0, 1.0), 0.0, 32, 0.005)


def _gs(prm):
    return O.Params(**{**prm.__dict__, "gauss_seidel": 1})


def test_single_contact_equals_jacobi(plane):
    """With one point in contact (the others far above the plane) the sweep applies one
    projection, which is the Jacobi form's correction with N = 1: the same wrench,
    counts and loss in every simulation."""
    ob = obj_from(plane, 1.0, 30.0)
    pts = [[0.01, 0.02, 0.03], [0.004, -0.006, -0.0025], [-0.02, 0.01, 0.04], [0.0, -0.01, 0.05]]
    hand = multi_point_hand(pts)
    for mu in (0.0, 0.5, 10.0):
        prm = O.Params(mu=mu, w_pen=1.0)
        q = torch.zeros(1, 6, dtype=F64)
        a = O.evaluate(hand, ob, q, 0.0, prm)
        b = O.evaluate_gs(hand, ob, q, 0.0, _gs(prm))
        assert torch.equal(a["N"], b["N"])
        assert torch.allclose(a["W"], b["W"], rtol=0, atol=1e-15)
        assert torch.allclose(a["L"], b["L"], rtol=1e-14, atol=0)


@pytest.mark.parametrize("order", ["shallow_first", "deep_first"])
def test_two_contacts_push_out_to_the_deepest(plane, order):
    """Translation only (I^-1 = 0), no friction, normals +z.  The first projection
    moves the object down by its depth C_1; the second point then sees
    phi = -d_2 + C_1, so the sweep ends with the object moved down by the largest
    depth: x_dot_z = v_z - (max_i d_i + dt v_z)/dt in every simulation whose contact is
    active.  Shallow point first: both points project (N = 2).  Deep point first: the
    shallow one is already resolved (N = 1).  The Jacobi form would move the object by
    the mean depth instead."""
    ob = obj_from(plane, 1.0, 0.0)
    d1, d2 = 0.0015, 0.0032
    pts = [[0.01, 0.0, -d1], [-0.02, 0.01, -d2]]
    if order == "deep_first":
        pts = pts[::-1]
    hand = multi_point_hand(pts)
    prm = O.Params(mu=0.0)
    out = O.evaluate_gs(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, _gs(prm))
    expect = 0.0
    for m, dvec in enumerate(O.TEST_DIRECTIONS):
        v = np.array(dvec, dtype=np.float64) * prm.v_test
        Cdeep = d2 + prm.dt * v[2]
        dz = -max(Cdeep, 0.0)
        # grid samples are float32: depths hold to ~1e-9 m
        assert abs(float(out["dx"][0, m, 2]) - dz) < 1e-8
        assert float(out["dx"][0, m, :2].abs().max()) < 1e-12
        n_exp = 2 if order == "shallow_first" and d1 + prm.dt * v[2] > 0 else 1
        assert int(out["N"][0, m]) == n_exp, (m, order)
        expect += np.linalg.norm(v + np.array([0.0, 0.0, dz / prm.dt]))
    assert abs(float(out["L_stable"][0]) - expect / 7) < 1e-5
    jac = O.evaluate(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, prm)
    assert abs(float(jac["L_stable"][0]) - expect / 7) > 1e-3      # the mean, not the deepest


def test_each_projection_zeroes_its_constraint(plane):
    """Eq. (1) in the sweep: after the last active projection (rotation allowed, no
    friction) the linearised constraint of that point vanishes at the final state,
    phi_hat - n . (x~ + dx + dth x d) = 0, while earlier contacts need not hold."""
    ob = obj_from(plane, 1.0, 25.0)
    pts = [[0.012, -0.007, -0.0021], [-0.015, 0.004, -0.0012], [0.003, 0.016, -0.0030]]
    hand = multi_point_hand(pts)
    prm = O.Params(mu=0.0)
    out = O.evaluate_gs(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, _gs(prm))
    for m, dvec in enumerate(O.TEST_DIRECTIONS):
        kap = out["kappa"][0, :, m]
        last = int(torch.nonzero(kap)[-1])
        x_pred = prm.dt * np.array(dvec, dtype=np.float64) * prm.v_test
        d = np.array(pts[last]) - x_pred
        disp = x_pred + out["dx"][0, m].numpy() + np.cross(out["dth"][0, m].numpy(), d)
        g = out["grad_phi"][0, last].numpy()
        n = g / np.linalg.norm(g)
        phi_end = float(out["phi_hat"][0, last]) - n @ disp
        assert abs(phi_end) < 1e-15, (m, phi_end)
        # on the plane, phi_hat = p_z and n = +z up to the float32 grid samples
        assert abs(pts[last][2] - disp[2]) < 1e-8, m
    # a chained sweep: some simulation projects more than one point
    assert (out["N"][0] >= 2).any()


def test_static_friction_stops_the_slide_for_later_points(plane):
    """Translation along +x with a high friction coefficient: the first contact's
    static friction cancels the tangential displacement dt V, so the second contact
    sees sigma = 0 and adds no friction; the object stops sliding (x_dot_x = 0) and
    is pushed out by the deeper depth."""
    ob = obj_from(plane, 1.0, 0.0)
    d1, d2 = 0.002, 0.003
    hand = multi_point_hand([[0.004, 0.002, -d1], [-0.01, 0.003, -d2]])
    prm = O.Params(mu=10.0)
    out = O.evaluate_gs(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, _gs(prm))
    m = O.TEST_DIRECTIONS.index((1, 0, 0))
    xdot = prm.v_test * np.array([1.0, 0.0, 0.0]) + out["dx"][0, m].numpy() / prm.dt
    assert abs(xdot[0]) < 1e-9
    assert abs(xdot[1]) < 1e-9
    assert abs(out["dx"][0, m, 2].item() + d2) < 1e-8
    assert float(out["sigma"][0, 1, m]) < 1e-15


def test_no_contact_gives_six_sevenths_v():
    w = synth.tiny_sphere_workload()
    S = O.Setup(w.hand, w.objects, dict(w.params, gauss_seidel=1))
    q = np.zeros((2, S.hand.D))
    q[:, 0] = [0.5, -0.4]
    out = O.loss_and_grad(S.hand, S.objs[0], q, 0.004, S.prm)
    assert torch.all(out["N"] == 0)
    assert torch.all(out["L_stable"] == 6.0 * S.prm.v_test / 7.0)


@pytest.fixture(scope="module")
def tiny_gs():
    w = synth.tiny_sphere_workload()
    S = O.Setup(w.hand, w.objects, dict(w.params, gauss_seidel=1))
    return w, S


def _fd_frozen(S, q, r, prm, dec, h):
    B, D = q.shape
    g = np.zeros((B, D))
    for k in range(D):
        e = np.zeros(D)
        e[k] = h
        lp = O.evaluate_gs(S.hand, S.objs[0], torch.tensor(q + e), r, prm, dec=dec, anchor_mode=True)["L"]
        lm = O.evaluate_gs(S.hand, S.objs[0], torch.tensor(q - e), r, prm, dec=dec, anchor_mode=True)["L"]
        g[:, k] = ((lp - lm) / (2 * h)).detach().numpy()
    return g


@pytest.mark.parametrize("alpha", [0.0, 0.1])
def test_gradient_matches_frozen_branch_differences(tiny_gs, alpha):
    """alpha = 0: the exact gradient of the piece of the loss the decisions select,
    through the whole chain of projections.  alpha = 0.1: the leaky gradient, the
    exact gradient of the surrogate whose non-contact constraints are
    -alpha (phi_m - anchor) with the state before the point frozen at the decision
    point."""
    w, S = tiny_gs
    prm = O.Params(**{**S.prm.__dict__, "alpha_leak": alpha})
    sel = [i for i in range(w.B) if i in (1, 2, 5, 6, 12)]
    q = w.q0[sel].astype(np.float64)
    out = O.loss_and_grad(S.hand, S.objs[0], q, 0.004, prm)
    assert (out["N"].sum(-1) > 0).sum() >= 3, "the candidates must touch the object"
    assert (out["N"] >= 2).any(), "some simulation must chain several projections"
    fd = _fd_frozen(S, q, 0.004, prm, out["dec"], 1e-8)
    g = out["grad"].numpy()
    rel = np.linalg.norm(fd - g, axis=1) / np.maximum(np.linalg.norm(g, axis=1), 1e-12)
    assert rel.max() < 1e-6, rel


def test_frozen_decisions_reproduce_the_method(tiny_gs):
    w, S = tiny_gs
    q = torch.tensor(w.q0[:6].astype(np.float64))
    a = O.evaluate_gs(S.hand, S.objs[0], q, 0.004, S.prm)
    b = O.evaluate_gs(S.hand, S.objs[0], q, 0.004, S.prm, dec=a["dec"], anchor_mode=True)
    assert torch.equal(a["L"], b["L"])


def test_unfrozen_differences_where_branches_hold(tiny_gs):
    """Central differences of the method's own loss match the alpha = 0 gradient on
    coordinates whose perturbation changes no decision."""
    w, S = tiny_gs
    prm = O.Params(**{**S.prm.__dict__, "alpha_leak": 0.0})
    q = w.q0.astype(np.float64)[[1, 2, 5, 6]]
    out = O.loss_and_grad(S.hand, S.objs[0], q, 0.004, prm)
    g = out["grad"].numpy()
    h = 1e-8
    used, total = 0, 0
    for k in range(S.hand.D):
        e = np.zeros(S.hand.D)
        e[k] = h
        ap = O.evaluate_gs(S.hand, S.objs[0], torch.tensor(q + e), 0.004, prm)
        am = O.evaluate_gs(S.hand, S.objs[0], torch.tensor(q - e), 0.004, prm)
        for b in range(q.shape[0]):
            total += 1
            same = all(torch.equal(x["dec"].kappa[b], out["dec"].kappa[b]) and
                       torch.equal(x["dec"].sdf["i0"][b], out["dec"].sdf["i0"][b]) and
                       torch.equal(x["dec"].static[b], out["dec"].static[b]) for x in (ap, am))
            if not same:
                continue
            used += 1
            fd = float((ap["L"][b] - am["L"][b]) / (2 * h))
            assert abs(fd - g[b, k]) <= 1e-5 * max(1.0, abs(g[b, k])), (b, k, fd, g[b, k])
    assert used >= 0.8 * total


def test_point_order_matters_only_through_shared_contacts(tiny_gs):
    """Reversing the point order changes the result only when a simulation chains two
    or more projections; with at most one contact per simulation it is identical
    (and then equal to the Jacobi form)."""
    w, S = tiny_gs
    hand = S.hand
    perm = torch.arange(hand.P - 1, -1, -1)
    rev = O.Hand(hand.L, hand.J, hand.D, hand.P, hand.parent, hand.T_fix, hand.axis, hand.q_low, hand.q_up,
                 hand.s[perm], hand.link[perm])
    q = torch.tensor(w.q0.astype(np.float64))
    a = O.evaluate_gs(hand, S.objs[0], q, 0.004, S.prm)
    b = O.evaluate_gs(rev, S.objs[0], q, 0.004, S.prm)
    # at most one projection per simulation in both orders, and the same points in contact
    single = (a["N"] <= 1).all(-1) & (b["N"] <= 1).all(-1) & (a["kappa"] == b["kappa"][:, perm]).all(-1).all(-1)
    assert single.any() and (~single).any()
    assert torch.allclose(a["L"][single], b["L"][single], rtol=1e-12)
    jac = O.evaluate(hand, S.objs[0], q, 0.004, S.prm)
    assert torch.allclose(a["L"][single], jac["L"][single], rtol=1e-12)
    assert (~torch.isclose(a["L"][~single], b["L"][~single], rtol=1e-6)).any()


def test_repeated_sweeps_converge_to_a_feasible_state(plane):
    """Listing a contact set k times makes one Gauss-Seidel pass k cyclic sweeps of
    projections onto the constraints' half-spaces (Eq. 1 in the metric of M, rotation
    allowed, no friction).  Cyclic projection onto intersecting half-spaces converges to
    a point of their intersection: with a small inertia (I^-1 = 1e4, so a push at one
    point rotates the object enough to re-open another) a single sweep leaves some
    constraint violated, three sweeps less so, and after 60 sweeps every linearised
    constraint of the set holds at the final state."""
    ob = obj_from(plane, 1.0, 1.0e4)
    pts = np.array([[0.012, -0.007, -0.0021], [-0.015, 0.004, -0.0012], [0.003, 0.016, -0.0030],
                    [-0.006, -0.013, -0.0026]])
    prm = _gs(O.Params(mu=0.0))
    x_pred_all = [prm.dt * np.array(d, dtype=np.float64) * prm.v_test for d in O.TEST_DIRECTIONS]

    def violation(out, n_pts):
        worst = 0.0
        for m, x_pred in enumerate(x_pred_all):
            dx, dth = out["dx"][0, m].numpy(), out["dth"][0, m].numpy()
            for i in range(n_pts):
                d = pts[i] - x_pred
                disp = x_pred + dx + np.cross(dth, d)
                g = out["grad_phi"][0, i].numpy()
                phi = float(out["phi_hat"][0, i]) - (g / np.linalg.norm(g)) @ disp
                worst = max(worst, -phi)
        return worst

    v = {}
    for k in (1, 3, 60):
        out = O.evaluate_gs(multi_point_hand(np.tile(pts, (k, 1))), ob, torch.zeros(1, 6, dtype=F64), 0.0, prm)
        v[k] = violation(out, len(pts))
    assert v[1] > 1e-4
    assert 0 < v[3] < 0.1 * v[1]
    assert v[60] < 1e-12
