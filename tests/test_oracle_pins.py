"""Pins of the FP64 oracle against closed forms, invariants, library routines and
finite differences (no GPU).  Each test names the passage of the paper it checks."""

import math
import os

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import synth
from oracle import fastgraspd_oracle as O

F64 = torch.float64
HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------- helpers

def one_point_hand(point):
    """A one-link 'hand' holding a single point at ``point`` in the base frame."""
    return O.Hand(L=1, J=0, D=6, P=1, parent=[-1],
                  T_fix=torch.eye(3, 4, dtype=F64)[None], axis=torch.zeros(1, 3, dtype=F64),
                  q_low=torch.zeros(0, dtype=F64), q_up=torch.zeros(0, dtype=F64),
                  s=torch.tensor(np.asarray([point], dtype=np.float64)), link=torch.zeros(1, dtype=torch.long))


def multi_point_hand(points):
    pts = torch.tensor(np.asarray(points, dtype=np.float64))
    return O.Hand(L=1, J=0, D=6, P=len(pts), parent=[-1],
                  T_fix=torch.eye(3, 4, dtype=F64)[None], axis=torch.zeros(1, 3, dtype=F64),
                  q_low=torch.zeros(0, dtype=F64), q_up=torch.zeros(0, dtype=F64),
                  s=pts, link=torch.zeros(len(pts), dtype=torch.long))


def obj_from(o, inv_mass=None, inv_inertia=None):
    ob = O.Obj.from_synth(o)
    if inv_mass is not None:
        ob.inv_mass = inv_mass
    if inv_inertia is not None:
        ob.inv_inertia = inv_inertia
    return ob


def zero_q(B=1, D=6):
    return np.zeros((B, D))


@pytest.fixture(scope="module")
def tiny():
    w = synth.tiny_sphere_workload()
    return w, O.Setup(w.hand, w.objects, w.params)


# ----------------------------------------------------------------------------- constants

def test_paper_constants_golden():
    """The constants the paper prints (Sec. III-C, Sec. IV-A) are the oracle's defaults
    and the workloads' parameters."""
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                vals[parts[0]] = parts[1:]
    prm = O.Params()
    assert prm.alpha_leak == float(vals["alpha_leak"][0])
    assert prm.dt == float(vals["dt"][0])
    assert prm.lr == float(vals["lr"][0])
    assert O.M_SIMS == int(vals["n_sims"][0])
    dirs = {tuple(int(float(c)) for c in d.split(",")) for d in vals["test_directions"]}
    assert set(O.TEST_DIRECTIONS) == dirs and len(O.TEST_DIRECTIONS) == len(dirs)
    dp = synth.default_params()
    assert (dp["alpha_leak"], dp["dt"], dp["lr"]) == (prm.alpha_leak, prm.dt, prm.lr)


# ----------------------------------------------------------------------------- FK (Sec. III-C, p = FK(q_h))

@pytest.mark.parametrize("kind", [3, 4, 5])
def test_fk_rest_pose(kind):
    """q = 0 puts every point where the generator placed it from the rest frames."""
    h = synth.make_hand(kind, 16)
    hand = O.Hand.from_synth(h)
    R, o = O.forward_kinematics(hand, torch.zeros(1, hand.D, dtype=F64))
    p = O.hand_points(hand, R, o)[0].numpy()
    assert np.abs(p - h["rest_pts"]).max() < 1e-7


def test_fk_base_pose_matches_scipy():
    """The base is R_b = Exp(w), t: compare with scipy's rotation-vector map."""
    h = synth.make_hand(4, 16)
    hand = O.Hand.from_synth(h)
    rng = np.random.default_rng(0)
    for _ in range(5):
        t = rng.normal(size=3) * 0.1
        w = rng.normal(size=3)
        q = np.concatenate([t, w, np.zeros(hand.J)])[None]
        R, o = O.forward_kinematics(hand, torch.tensor(q))
        p = O.hand_points(hand, R, o)[0].numpy()
        ref = h["rest_pts"] @ Rotation.from_rotvec(w).as_matrix().T + t
        assert np.abs(p - ref).max() < 1e-7


def test_so3_exp_small_angle():
    w = torch.tensor([[0.0, 0.0, 0.0], [1e-10, -2e-10, 3e-10]], dtype=F64)
    R = O.so3_exp(w)
    assert torch.equal(R[0], torch.eye(3, dtype=F64))
    ref = Rotation.from_rotvec(w[1].numpy()).as_matrix()
    assert np.abs(R[1].numpy() - ref).max() < 1e-18


def test_fk_single_joint_quarter_turn():
    """theta = pi/2 on a flexion joint turns the finger's points by 90 degrees about
    the world x axis through the joint (flexion axes are local x, rest frames are
    axis-aligned); every other point stays put."""
    h = synth.make_hand(3, 16)
    hand = O.Hand.from_synth(h)
    names = h["names"]
    link = names.index("f1_flex1")
    q = np.zeros((1, hand.D))
    q[0, 6 + link - 1] = math.pi / 2
    R, o = O.forward_kinematics(hand, torch.tensor(q))
    p = O.hand_points(hand, R, o)[0].numpy()
    rest = h["rest_pts"]
    moved = np.isin(h["link_of_point"], [names.index(n) for n in ("f1_flex1", "f1_flex2", "f1_flex3")])
    o0 = h["rest_o"][link]
    rel = rest[moved] - o0
    expect = np.stack([rel[:, 0], -rel[:, 2], rel[:, 1]], axis=1) + o0     # Rx(90): y->z, z->-y
    assert np.abs(p[moved] - expect).max() < 1e-7
    assert np.abs(p[~moved] - rest[~moved]).max() < 1e-7


@pytest.mark.parametrize("kind", [3, 5])
def test_fk_rigidity(kind):
    """Distances between points of one link are invariant under any q."""
    h = synth.make_hand(kind, 12)
    hand = O.Hand.from_synth(h)
    rng = np.random.default_rng(1)
    q = np.concatenate([rng.normal(size=(3, 3)) * 0.1, rng.normal(size=(3, 3)),
                        rng.uniform(-2, 2, size=(3, hand.J))], axis=1)
    R, o = O.forward_kinematics(hand, torch.tensor(q))
    p = O.hand_points(hand, R, o).numpy()
    for l in range(hand.L):
        sel = h["link_of_point"] == l
        ref = h["rest_pts"][sel]
        dref = np.linalg.norm(ref[:, None] - ref[None], axis=-1)
        for b in range(3):
            pb = p[b][sel]
            assert np.abs(np.linalg.norm(pb[:, None] - pb[None], axis=-1) - dref).max() < 1e-7


# ----------------------------------------------------------------------------- SDF (Sec. III-A grid, III-B dilation)

COEF = (0.3, -0.7, 1.1)


@pytest.fixture(scope="module")
def linear_obj():
    return obj_from(synth.linear_grid(COEF, 0.01, 24, 0.004))


def test_sdf_linear_field_is_exact(linear_obj):
    """Trilinear interpolation reproduces a linear field and its gradient exactly;
    distinct per-axis slopes catch any transposed axis or misplaced corner."""
    rng = np.random.default_rng(2)
    half = 0.5 * 23 * 0.004
    p = torch.tensor(rng.uniform(-half * 0.99, half * 0.99, size=(500, 3)))
    phi, g = O.sdf_query(linear_obj, p, 0.0)
    ref = p @ torch.tensor(COEF, dtype=F64) + 0.01
    # the grid holds float32 samples: exactness up to their rounding
    assert (phi - ref).abs().max() < 1e-8
    assert (g - torch.tensor(COEF, dtype=F64)).abs().max() < 1e-5


def test_sdf_dilation_shifts_value(linear_obj):
    p = torch.tensor([[0.01, -0.02, 0.005]], dtype=F64)
    a, ga = O.sdf_query(linear_obj, p, 0.0)
    b, gb = O.sdf_query(linear_obj, p, 0.003)
    assert torch.allclose(a - b, torch.tensor([0.003], dtype=F64), atol=1e-15)
    assert torch.equal(ga, gb)


def test_sdf_outside_grid_excess(linear_obj):
    """Beyond the +x face by delta: value at the clamped point plus delta, gradient
    (1, a_y, a_z): the excess distance replaces the clamped axis."""
    half = 0.5 * 23 * 0.004
    delta = 0.013
    p = torch.tensor([[half + delta, 0.01, -0.02]], dtype=F64)
    phi, g = O.sdf_query(linear_obj, p, 0.0)
    inner = torch.tensor([[half, 0.01, -0.02]], dtype=F64)
    ref = (inner @ torch.tensor(COEF, dtype=F64) + 0.01) + delta
    assert abs(float(phi[0] - ref[0])) < 1e-8
    assert np.allclose(g[0].numpy(), [1.0, COEF[1], COEF[2]], atol=1e-5)
    # beyond an edge (two axes clamped): excess = Euclidean distance to the edge
    p2 = torch.tensor([[half + 0.003, -half - 0.004, 0.0]], dtype=F64)
    phi2, g2 = O.sdf_query(linear_obj, p2, 0.0)
    edge = torch.tensor([[half, -half, 0.0]], dtype=F64)
    ref2 = float(edge @ torch.tensor(COEF, dtype=F64) + 0.01) + 0.005
    assert abs(float(phi2[0]) - ref2) < 1e-8
    assert np.allclose(g2[0].numpy(), [0.6, -0.8, COEF[2]], atol=1e-5)


def test_sdf_nodes_exact():
    ob = synth.sphere_grid(0.04, 16, 0.008)
    o = obj_from(ob)
    g = ob["grid"].double()
    idx = [(0, 0, 0), (3, 7, 11), (15, 15, 15), (14, 1, 8)]
    p = torch.tensor([[o.origin[0] + i * o.pitch, o.origin[1] + j * o.pitch, o.origin[2] + k * o.pitch]
                      for (i, j, k) in idx], dtype=F64)
    phi, _ = O.sdf_query(o, p, 0.0)
    ref = torch.tensor([float(g[k, j, i]) for (i, j, k) in idx], dtype=F64)
    assert (phi - ref).abs().max() < 1e-12


def test_sdf_sphere_within_interpolation_bound():
    """|trilinear(|x| - R) - (|x| - R)| <= (h^2/8) * sum_i |d^2 phi/dx_i^2| <= 3 h^2 / (8 r_min)."""
    R, n, h = 0.04, 64, 0.002
    o = obj_from(synth.sphere_grid(R, n, h))
    rng = np.random.default_rng(3)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = rng.uniform(R - 0.01, R + 0.01, size=2000)
    p = torch.tensor(d * rad[:, None])
    phi, g = O.sdf_query(o, p, 0.0)
    exact = p.norm(dim=-1) - R
    rmin = torch.tensor(rad) - math.sqrt(3) * h
    bound = 3 * h * h / (8 * rmin) + 1e-7       # + float32 storage of the samples
    assert torch.all((phi - exact).abs() <= bound)
    # the interpolated gradient points along the radius to within a few degrees
    cosang = (g * p).sum(-1) / (g.norm(dim=-1) * p.norm(dim=-1))
    assert cosang.min() > 0.99


def test_sdf_gradient_matches_finite_differences():
    """The analytic gradient of the interpolant equals central differences of the
    interpolated value (points kept away from voxel faces, where it jumps)."""
    o = obj_from(synth.box_grid((0.03, 0.02, 0.025), 40, 0.003))
    rng = np.random.default_rng(4)
    p = rng.uniform(-0.055, 0.055, size=(400, 3))
    u = (p - o.origin.numpy()) / o.pitch
    keep = (np.abs(u - np.round(u)) > 1e-3).all(axis=1)
    p = torch.tensor(p[keep])
    _, g = O.sdf_query(o, p, 0.0)
    h = 1e-7
    fd = torch.zeros_like(p)
    for k in range(3):
        e = torch.zeros(3, dtype=F64)
        e[k] = h
        fd[:, k] = (O.sdf_query(o, p + e, 0.0)[0] - O.sdf_query(o, p - e, 0.0)[0]) / (2 * h)
    assert (fd - g).abs().max() < 1e-6


# ----------------------------------------------------------------------------- contacts (Sec. III-C, Eq. 1)

@pytest.fixture(scope="module")
def plane():
    """phi = z: the object fills z < 0 and the contact normal is +z everywhere."""
    return synth.linear_grid((0.0, 0.0, 1.0), 0.0, 32, 0.005)


def test_no_contact_gives_six_sevenths_v(tiny):
    """No point in contact: every correction is zero, x_dot+ = v_m, and
    L_stable = (1/7) * 6 V exactly (Eq. 2)."""
    w, S = tiny
    q = np.zeros((2, S.hand.D))
    q[:, 0] = [0.5, -0.4]                           # hand half a metre away
    out = O.loss_and_grad(S.hand, S.objs[0], q, 0.004, S.prm)
    assert torch.all(out["N"] == 0)
    assert torch.all(out["W"] == 0)
    assert torch.all(out["L_stable"] == 6.0 * S.prm.v_test / 7.0)


def _constraint_at(ob, pt, x_pred):
    """C(x, theta) = max(0, -phi(R(theta)^T (p - x))) for the object pose (x_pred + x,
    theta), rotations about the object's centre of mass (scipy rotation vectors)."""
    def C(xv):
        x, th = x_pred + xv[:3], xv[3:]
        r = Rotation.from_rotvec(th).as_matrix().T @ (pt - x)
        phi, _ = O.sdf_query(ob, torch.tensor(r[None]), 0.0)
        return max(0.0, -float(phi[0]))
    return C


def _fd_jacobian(C, h=1e-7):
    return np.array([(C(np.eye(6)[k] * h) - C(-np.eye(6)[k] * h)) / (2 * h) for k in range(6)])


@pytest.mark.parametrize("seed", range(4))
def test_single_contact_on_a_sphere(seed):
    """One hand point at depth delta inside a sphere centred at the object's origin, in
    the zero-velocity simulation (Eq. 1 and Sec. IV-A): the lever d = p is parallel to
    the outward normal u, so the projection is a pure push along -u of size delta m
    (lambda_n = C / w_n with w_n = 1/m, since d x n = 0), no torque, and no friction
    (the test velocity is 0, so sigma = 0).  The sphere is sampled on a 2 mm grid: the
    value errs by at most (3/8) h^2 / R (2.5% of delta here) and the normal's direction
    by O(h / R) = 0.05, which set the tolerances."""
    R, h, delta = 0.04, 0.002, 0.0015
    ob = obj_from(synth.sphere_grid(R, 64, h), 1.0)
    u = np.random.default_rng(seed).normal(size=3)
    u /= np.linalg.norm(u)
    p = (R - delta) * u
    out = O.evaluate(multi_point_hand([p]), ob, torch.zeros(1, 6, dtype=F64), 0.0, O.Params(mu=0.5))
    W = out["W"][0, 0].numpy()
    assert int(out["N"][0, 0]) == 1
    assert np.linalg.norm(W[:3] + u * delta) <= (0.025 + 0.05) * delta
    assert np.linalg.norm(W[3:]) <= 0.05 * np.linalg.norm(p) * delta
    assert float(out["sigma"][0, 0, 0]) == 0.0


@pytest.mark.parametrize("m", range(7))
@pytest.mark.parametrize("inv_mass,inv_inertia", [(1.0, 0.0), (0.0, 30.0), (1.0, 25.0)])
def test_single_contact_projection_satisfies_eq1(plane, inv_mass, inv_inertia, m):
    """Eq. (1) for one constraint at the predicted pose x_pred = dt v_m: the correction
    (dx, dth) zeroes the linearised constraint, C + J [dx; dth] = 0, and is M^-1 J^T
    times a scalar.  J is taken by finite differences of the constraint built from
    the oracle's grid lookup and scipy rotations (friction off; on a plane the
    plane-linearised depth is exact, so C is the true penetration at x_pred)."""
    ob = obj_from(plane, inv_mass, inv_inertia)
    pt = np.array([0.012, -0.007, -0.0021])
    hand = one_point_hand(pt)
    prm = O.Params(mu=0.0)
    out = O.evaluate(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, prm)
    v = np.array(O.TEST_DIRECTIONS[m], dtype=np.float64) * prm.v_test
    x_pred = prm.dt * v
    dx = out["W"][0, m, :3].numpy() * inv_mass             # N = 1: no averaging
    dth = out["W"][0, m, 3:].numpy() * inv_inertia
    C = _constraint_at(ob, pt, x_pred)
    Jc = _fd_jacobian(C)
    c0 = C(np.zeros(6))
    assert c0 > 0
    step = np.concatenate([dx, dth])
    assert abs(c0 + Jc @ step) < 1e-9
    Minv_JT = np.concatenate([Jc[:3] * inv_mass, Jc[3:] * inv_inertia])
    lam = step @ Minv_JT / (Minv_JT @ Minv_JT)
    assert np.abs(step - lam * Minv_JT).max() < 1e-9


def test_prediction_moves_the_constraint(plane):
    """The object moves by x_pred = dt v_m before the projection: a contact on the
    plane z = 0 (normal +z) at depth delta has depth delta + dt V when the object
    moves up into the point, delta - dt V when it moves away, and delta for the
    lateral and zero velocities; with translation only and no friction the object
    ends with x_dot_z = v_z - C_m / dt (Eq. 1 and x_dot+ = (x+ - x-)/dt)."""
    ob = obj_from(plane, 1.0, 0.0)
    delta = 0.003
    hand = one_point_hand([0.004, 0.002, -delta])
    prm = O.Params(mu=0.0)
    out = O.evaluate(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, prm)
    for m, dvec in enumerate(O.TEST_DIRECTIONS):
        Cm = delta + prm.dt * prm.v_test * dvec[2]
        assert abs(float(out["C"][0, 0, m]) - Cm) < 1e-8
        xdot_z = prm.v_test * dvec[2] + float(out["W"][0, m, 2]) / prm.dt
        assert abs(xdot_z - (prm.v_test * dvec[2] - Cm / prm.dt)) < 1e-5


def test_friction_correction_with_rotation_sticks(plane):
    """Static friction with a rotating object: the friction part of the correction
    (full correction minus the frictionless one) moves the contact point by exactly
    -s (it cancels the tangential displacement s = dt (v - (v.n) n)), and it is
    M^-1 J_t^T times a scalar, with J_t = [t^T, (d x t)^T]."""
    inv_m, inv_I = 1.0, 40.0
    ob = obj_from(plane, inv_m, inv_I)
    pt = np.array([0.011, -0.006, -0.003])
    hand = one_point_hand(pt)
    full = O.evaluate(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, O.Params(mu=50.0))
    frictionless = O.evaluate(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, O.Params(mu=0.0))
    prm = O.Params()
    for m in (1, 2, 3, 4):                                     # lateral test velocities
        v = np.array(O.TEST_DIRECTIONS[m], dtype=np.float64) * prm.v_test
        s = prm.dt * v                                        # n = +z: v is tangential
        Wf = (full["W"][0, m] - frictionless["W"][0, m]).numpy()
        dx, dth = Wf[:3] * inv_m, Wf[3:] * inv_I
        d = pt - prm.dt * v
        moved = dx + np.cross(dth, d)
        that = s / np.linalg.norm(s)
        assert abs(moved @ that + np.linalg.norm(s)) < 1e-12
        Jt = np.concatenate([that, np.cross(d, that)])
        MJ = np.concatenate([Jt[:3] * inv_m, Jt[3:] * inv_I])
        lam = np.concatenate([dx, dth]) @ MJ / (MJ @ MJ)
        assert np.abs(np.concatenate([dx, dth]) - lam * MJ).max() < 1e-12


def test_stability_and_penetration_losses_closed_form(plane):
    """Two contacts on the plane, translation only, no friction: every simulation
    ends with x_dot = v_m - (mean depth_m / dt) z, so Eq. (2) gives
    L_stable = (1/7) sum_m |v_m - (C_m / dt) z|; the penetration sum at zero velocity
    is the sum of the two depths."""
    ob = obj_from(plane, 1.0, 0.0)
    d1, d2 = 0.002, 0.0035
    hand = multi_point_hand([[0.01, 0.0, -d1], [-0.02, 0.01, -d2]])
    prm = O.Params(mu=0.0, w_pen=1.0)
    out = O.evaluate(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, prm)
    expect = 0.0
    for dvec in O.TEST_DIRECTIONS:
        v = np.array(dvec, dtype=np.float64) * prm.v_test
        Cm = 0.5 * (d1 + d2) + prm.dt * v[2]
        expect += np.linalg.norm(v - np.array([0, 0, Cm / prm.dt]))
    assert abs(float(out["L_stable"][0]) - expect / 7) < 1e-5
    assert abs(float(out["L_pen"][0]) - (d1 + d2)) < 1e-8


@pytest.mark.parametrize("mu,regime", [(10.0, "static"), (0.3, "kinetic")])
def test_friction_point_mass_on_plane(plane, mu, regime):
    """A translating object (no rotation: I^-1 = 0) meets one contact while moving
    along +x.  Position-level Coulomb friction: if the tangential displacement
    sigma = dt V fits in the friction cone (sigma <= mu C) it is cancelled, so the
    object stops sliding; otherwise it is reduced by mu C.  The normal correction
    pushes the object out by C.  Velocities: x_dot = (dx_total)/dt."""
    ob = obj_from(plane, 1.0, 0.0)
    depth = 0.003
    hand = one_point_hand([0.004, 0.002, -depth])
    prm = O.Params(mu=mu)
    out = O.evaluate(hand, ob, torch.zeros(1, 6, dtype=F64), 0.0, prm)
    m = O.TEST_DIRECTIONS.index((1, 0, 0))
    W = out["W"][0, m].numpy()
    xdot = prm.v_test * np.array([1.0, 0, 0]) + W[:3] / prm.dt       # N = 1, m = 1
    sigma = prm.dt * prm.v_test
    # the +x motion does not change the depth along z: C = depth (up to the float32
    # storage of the grid samples, ~1e-9 m)
    assert abs(-xdot[2] * prm.dt - depth) < 1e-8
    slide = xdot[0] * prm.dt
    if regime == "static":
        assert abs(slide) < 1e-15
    else:
        assert abs(slide - (sigma - mu * depth)) < 1e-8
    assert abs(xdot[1]) < 1e-15


def test_antipodal_contacts_cancel():
    """Two equal contacts at +-x on a sphere, zero velocity: forces cancel, W = 0,
    and the zero-velocity simulation ends at rest."""
    o = obj_from(synth.sphere_grid(0.04, 64, 0.002, shift=(0.0, 0.0, 0.0)))
    hand = multi_point_hand([[0.0372, 0.0, 0.0], [-0.0372, 0.0, 0.0]])
    out = O.evaluate(hand, o, torch.zeros(1, 6, dtype=F64), 0.0, O.Params())
    assert out["N"][0, 0] == 2
    # mirrored grid samples agree to one float32 ulp (~4e-9 m), so W cancels to that level
    assert out["W"][0, 0].abs().max() < 1e-8


def test_threefold_contacts_cancel():
    """Three equal-depth contacts at 120 degrees in the xy plane: W_lin = 0 and, by
    symmetry about z, the torque about z vanishes too."""
    o = obj_from(synth.sphere_grid(0.04, 64, 0.002, shift=(0.0, 0.0, 0.0)))
    pts = [[0.0365 * math.cos(a), 0.0365 * math.sin(a), 0.0] for a in (0.0, 2 * math.pi / 3, 4 * math.pi / 3)]
    hand = multi_point_hand(pts)
    out = O.evaluate(hand, o, torch.zeros(1, 6, dtype=F64), 0.0, O.Params())
    assert out["N"][0, 0] == 3
    # the grid is not 3-fold symmetric: each depth is exact only to the trilinear
    # bound 3h^2/(8 r) ~ 4e-5 m, so |sum f| <= 2 * 3 * bound; a single uncancelled
    # force would be ~ C = 3.5e-3
    bound = 3 * 0.002 ** 2 / (8 * (0.0365 - math.sqrt(3) * 0.002))
    C = -float(out["phi_m"][0, 0, 0])
    assert C > 3e-3
    assert out["W"][0, 0, :3].abs().max() < 6 * bound
    assert abs(float(out["W"][0, 0, 5])) < 1e-6


def test_averaging_is_invariant_to_duplicated_contacts(tiny):
    """The Jacobi reading averages corrections over active contacts: listing every
    point twice doubles W and N and leaves x_dot+, theta_dot+ and L_stable unchanged
    (a plain sum would double the correction)."""
    w, S = tiny
    hand = S.hand
    dup = O.Hand(hand.L, hand.J, hand.D, 2 * hand.P, hand.parent, hand.T_fix, hand.axis,
                 hand.q_low, hand.q_up, torch.cat([hand.s, hand.s]), torch.cat([hand.link, hand.link]))
    q = torch.tensor(w.q0[[2, 5, 6, 12]].astype(np.float64))
    a = O.evaluate(hand, S.objs[0], q, 0.004, S.prm)
    b = O.evaluate(dup, S.objs[0], q, 0.004, S.prm)
    assert torch.all(a["N"] > 0)
    assert torch.allclose(2 * a["W"], b["W"], rtol=1e-12, atol=1e-15)
    assert torch.allclose(a["L_stable"], b["L_stable"], rtol=1e-12)


# ----------------------------------------------------------------------------- joint losses (Eq. 3, Eq. 4)

def test_range_and_limit_losses():
    h = synth.make_hand(3, 4)
    hand = O.Hand.from_synth(h)
    o = obj_from(synth.sphere_grid(0.04, 16, 0.008))
    mid = 0.5 * (h["q_low"] + h["q_up"]).astype(np.float64)
    q = np.zeros((3, hand.D))
    q[:, 0] = 1.0                                     # far away: no contact
    q[0, 6:] = mid
    q[1, 6:] = mid + 0.1 * np.arange(hand.J) / hand.J
    q[2, 6:] = mid
    q[2, 6] = h["q_up"][0] + 0.25
    q[2, 7] = h["q_low"][1] - 0.5
    out = O.evaluate(hand, o, torch.tensor(q), 0.0, O.Params())
    assert float(out["L_range"][0]) == 0.0
    assert abs(float(out["L_range"][1]) - np.linalg.norm(q[1, 6:] - mid)) < 1e-12
    assert float(out["L_limit"][0]) == 0.0 and float(out["L_limit"][1]) == 0.0
    assert abs(float(out["L_limit"][2]) - 0.75) < 1e-6


# ----------------------------------------------------------------------------- gradient (Sec. III-C leaky rule)

def _fd_frozen(S, obj, q, r, prm, dec, anchor_mode, h):
    """Central differences of the loss with every decision frozen at ``dec``."""
    B, D = q.shape
    g = np.zeros((B, D))
    for k in range(D):
        e = np.zeros(D)
        e[k] = h
        lp = O.evaluate(S.hand, obj, torch.tensor(q + e), r, prm, dec=dec, anchor_mode=anchor_mode)["L"]
        lm = O.evaluate(S.hand, obj, torch.tensor(q - e), r, prm, dec=dec, anchor_mode=anchor_mode)["L"]
        g[:, k] = ((lp - lm) / (2 * h)).detach().numpy()
    return g


@pytest.mark.parametrize("alpha", [0.0, 0.1])
def test_gradient_matches_frozen_branch_differences(tiny, alpha):
    """alpha = 0: the exact gradient of the piece of the loss selected by the
    decisions.  alpha = 0.1: the leaky gradient, which is the exact gradient of the
    surrogate in which every non-contact constraint is C = -alpha (phi_m - phi_m0),
    anchored at the evaluation point (value 0 there, slope -alpha)."""
    w, S = tiny
    prm = O.Params(**{**S.prm.__dict__, "alpha_leak": alpha})
    q = w.q0.astype(np.float64)
    out = O.loss_and_grad(S.hand, S.objs[0], q, 0.004, prm)
    fd = _fd_frozen(S, S.objs[0], q, 0.004, prm, out["dec"], True, 1e-8)
    g = out["grad"].numpy()
    rel = np.linalg.norm(fd - g, axis=1) / np.maximum(np.linalg.norm(g, axis=1), 1e-12)
    assert rel.max() < 1e-6, rel


def test_frozen_decisions_reproduce_the_method(tiny):
    """Evaluating with the decisions the method takes at q gives the same value, so
    the frozen pieces used above are pieces of the method's loss."""
    w, S = tiny
    q = torch.tensor(w.q0.astype(np.float64))
    a = O.evaluate(S.hand, S.objs[0], q, 0.004, S.prm)
    b = O.evaluate(S.hand, S.objs[0], q, 0.004, S.prm, dec=a["dec"], anchor_mode=True)
    assert torch.equal(a["L"], b["L"])


def test_unfrozen_differences_where_branches_hold(tiny):
    """Without freezing anything: central differences of the method's own loss (alpha
    has no effect on the value) match the alpha = 0 gradient on coordinates whose
    perturbation changes no decision."""
    w, S = tiny
    prm = O.Params(**{**S.prm.__dict__, "alpha_leak": 0.0})
    q = w.q0.astype(np.float64)[:6]
    out = O.loss_and_grad(S.hand, S.objs[0], q, 0.004, prm)
    g = out["grad"].numpy()
    h = 1e-8
    used, total = 0, 0
    for k in range(S.hand.D):
        e = np.zeros(S.hand.D)
        e[k] = h
        ap = O.evaluate(S.hand, S.objs[0], torch.tensor(q + e), 0.004, prm)
        am = O.evaluate(S.hand, S.objs[0], torch.tensor(q - e), 0.004, prm)
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


# ----------------------------------------------------------------------------- update (Sec. IV-A) and schedule (Sec. III-B)

def test_gradient_descent_step(tiny):
    w, S = tiny
    q0 = w.q0[:4]
    q1, _ = O.optimize(S, q0, w.obj_of_cand[:4], 0, 1, 100)
    g = O.batch_loss_and_grad(S, q0.astype(np.float64), w.obj_of_cand[:4], O.dilation_radius(S.prm, 0, 100))["grad"]
    assert np.abs(q1 - (q0.astype(np.float64) - 1e-3 * g)).max() < 1e-15


def test_dilation_schedule_linear_to_zero():
    prm = O.Params(r0=0.01, schedule="linear")
    K = 11
    r = [O.dilation_radius(prm, k, K) for k in range(K)]
    assert r[0] == 0.01 and r[-1] == 0.0
    assert np.allclose(np.diff(r), -0.001, atol=1e-15)
    assert O.dilation_radius(O.Params(r0=0.004), 50, 100) == 0.004


# ----------------------------------------------------------------------------- guard band

def test_guard_band_excludes_near_ties():
    """clean_candidates keeps a candidate only if every decision sits outside its guard
    band.  On the tilted plane phi = c . x (|c| = 1, no test velocity parallel to c)
    with r = 0, the +z simulation's constraint is phi_m = phi - dt V c_z: a point
    0.5 micrometres from that threshold is excluded on either side, one 0.3 mm away is
    kept; a point on a grid node plane (a tie in the cell choice) is excluded; in the
    +x simulation the friction regime flips at sigma = mu C with sigma = dt V
    sqrt(1 - c_x^2) and C = dt V c_x - phi, and a contact 0.5 micrometres from that
    boundary is excluded.  On an axis-aligned plane every candidate is excluded: the
    normal is parallel to two test velocities, where the friction direction is 0/0."""
    c = np.array([0.3, 0.2, 1.0])
    c /= np.linalg.norm(c)
    ob = obj_from(synth.linear_grid(tuple(c), 0.0, 32, 0.005), 1.0, 0.0)
    prm = O.Params(mu=0.5)
    dtv = prm.dt * prm.v_test
    h = ob.pitch
    org = ob.origin.numpy()
    x, y = org[0] + 7.31 * h, org[1] + 9.47 * h          # off the node planes
    q = np.zeros((1, 6))

    def at(phi, px=x):
        return [px, y, (phi - c[0] * px - c[1] * y) / c[2]]

    def clean(pt, o=ob):
        return bool(O.clean_candidates(multi_point_hand([pt]), o, q, 0.0, prm)[0])

    assert clean(at(dtv * c[2] + 3e-4))
    assert not clean(at(dtv * c[2] + 5e-7))
    assert not clean(at(dtv * c[2] - 5e-7))
    assert not clean(at(dtv * c[2] + 3e-4, px=org[0] + 7.0 * h))
    boundary = dtv * c[0] - dtv * np.sqrt(1.0 - c[0] ** 2) / prm.mu
    assert clean(at(boundary + 2e-4))
    assert not clean(at(boundary + 5e-7))
    flat = obj_from(synth.linear_grid((0.0, 0.0, 1.0), 0.0, 32, 0.005), 1.0, 0.0)
    assert not clean([x, y, 0.004], flat)


# ----------------------------------------------------------------------------- guard band per decision

def _tilted():
    c = np.array([0.3, 0.2, 1.0])
    c /= np.linalg.norm(c)
    return c, obj_from(synth.linear_grid(tuple(c), 0.0, 32, 0.005), 1.0, 0.0)


def test_decision_band_on_a_linear_field():
    """decision_band locates each near tie at its (point, simulation).  On the tilted
    plane phi = c . x the trilinear interpolant is exact in every cell, so a point on a
    node plane has the same value and normal in both cells: its flags are fixed and the
    candidate stays comparable (clean_candidates drops it).  A point 0.5 micrometres
    from the +z simulation's threshold phi_m = phi - dt V c_z = 0 has that one flag
    ambiguous and its candidate is not robust, while the other six flags of the point
    and the flags of a second, distant point are fixed."""
    c, ob = _tilted()
    prm = O.Params(mu=0.5)
    dtv = prm.dt * prm.v_test
    h = ob.pitch
    org = ob.origin.numpy()
    x, y = org[0] + 7.31 * h, org[1] + 9.47 * h

    def at(phi, px=x):
        return [px, y, (phi - c[0] * px - c[1] * y) / c[2]]

    q = np.zeros((1, 6))
    node = [at(dtv * c[2] + 3e-4, px=org[0] + 7.0 * h)]
    res = O.decision_band(multi_point_hand(node), ob, q, 0.0, prm)
    br = res["branches"][0]
    assert not res["flag"].any() and res["comparable"][0] and len(br["L"]) == 2
    # equal up to the float32 rounding of the stored grid values (the field is not exactly linear)
    assert np.abs(br["L"] - br["L"][0]).max() < 1e-12
    assert np.abs(br["grad"] - br["grad"][0]).max() < 1e-6 * np.abs(br["grad"][0]).max()
    assert not O.clean_candidates(multi_point_hand(node), ob, q, 0.0, prm)[0]
    tie = [at(dtv * c[2] + 5e-7), at(dtv * c[2] + 3e-3, px=x + 0.011)]
    res = O.decision_band(multi_point_hand(tie), ob, q, 0.0, prm)
    expect = np.zeros((1, 2, 7), dtype=bool)
    expect[0, 0, 5] = True                               # +z is simulation 5
    assert np.array_equal(res["flag"], expect) and np.array_equal(res["masked"], expect)
    # both flags of the tie are branches: with the contact (N = 1, a push of ~0.5 um) and without
    br = res["branches"][0]
    assert res["comparable"][0] and len(br["L"]) == 2
    ref = O.loss_and_grad(multi_point_hand(tie), ob, q, 0.0, prm)
    assert br["L"][0] == float(ref["L"].detach()[0]) and br["L"][1] != br["L"][0]


def test_decision_band_cell_choice_on_a_curved_field():
    """On a grid-sampled sphere the normal jumps across a node plane.  A flag is
    ambiguous exactly when phi_m taken just on either side of the plane (the lookup at
    p -+ 1e-7 voxel along the axis, where the cell choice is each side's own) has
    different signs or lies within the band.  Checked on points placed on node planes
    in a shell around the dilated surface, where both outcomes occur."""
    R = 0.04
    ob = obj_from(synth.sphere_grid(R, 64, 0.002), 1.0)
    hgrid = ob.pitch                                      # the float32 pitch of the grid
    prm = O.Params()
    rng = np.random.default_rng(4)
    org = ob.origin.numpy()
    V = np.array(O.TEST_DIRECTIONS, dtype=np.float64) * prm.v_test
    seen = {True: 0, False: 0}
    for _ in range(300):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        p = u * (R + rng.uniform(-2e-4, 2e-3))
        ax = rng.integers(3)
        k = np.round((p[ax] - org[ax]) / hgrid)
        p[ax] = org[ax] + k * hgrid                       # on a node plane
        res = O.decision_band(one_point_hand(p), ob, np.zeros((1, 6)), 0.0, prm)
        side = []
        for s in (-1.0, 1.0):
            ps = p.copy()
            ps[ax] += s * 1e-7 * hgrid
            phi, g = O.sdf_query(ob, torch.tensor(ps[None]), 0.0)
            n = g[0].numpy() / np.linalg.norm(g[0].numpy())
            side.append(float(phi[0]) - prm.dt * V @ n)
        side = np.array(side)                             # [2, 7]
        slack = 1e-6 + 2e-7 * hgrid
        if (np.abs(side) <= slack).any() or (np.abs(np.abs(side) - 1e-6) < 1e-8).any():
            continue                                      # on the band's edge: either answer is right
        want = (np.sign(side[0]) != np.sign(side[1]))
        assert np.array_equal(res["flag"][0, 0], want), (p, side)
        seen[bool(want.any())] += 1
    assert seen[True] >= 5 and seen[False] >= 50


def test_decision_band_friction_regime():
    """A single contact 0.5 micrometres from the friction boundary sigma = mu C of the
    +x simulation: the force is continuous there (sigma / w_t on both sides) but its
    derivative is not (d sigma against mu dC).  With a rotational inertia the static
    regime does not cancel the tangential velocity of the object's centre, so the two
    derivatives reach the loss: the flag is fixed, the two branches have nearly the
    same loss and different gradients; 0.2 mm from the boundary there is one branch."""
    c, ob = _tilted()
    ob.inv_inertia = 1.0 / (0.4 * 0.05 ** 2)
    prm = O.Params(mu=0.5)
    dtv = prm.dt * prm.v_test
    h = ob.pitch
    org = ob.origin.numpy()
    x, y = org[0] + 7.31 * h, org[1] + 9.47 * h
    boundary = dtv * c[0] - dtv * np.sqrt(1.0 - c[0] ** 2) / prm.mu

    def pt(phi):
        return [x, y, (phi - c[0] * x - c[1] * y) / c[2]]

    q = np.zeros((1, 6))
    near = O.decision_band(one_point_hand(pt(boundary + 5e-7)), ob, q, 0.0, prm)
    br = near["branches"][0]
    assert not near["flag"].any() and near["comparable"][0] and len(br["L"]) == 2
    assert abs(br["L"][1] - br["L"][0]) < 2e-5 * abs(br["L"][0])     # (sigma - mu C) / (w_t dt) apart
    assert np.linalg.norm(br["grad"][1] - br["grad"][0]) > 1e-3 * np.linalg.norm(br["grad"][0])
    far = O.decision_band(one_point_hand(pt(boundary + 2e-4)), ob, q, 0.0, prm)
    assert not far["flag"].any() and far["comparable"][0] and len(far["branches"][0]["L"]) == 1


def test_decision_band_gauss_seidel_masks_the_rest_of_a_chain():
    """Gauss-Seidel form: the state a point sees depends on every earlier projection
    of its simulation, so the comparison masks a chain from its first ambiguous
    decision on.  Three points in contact (depths 2, 3 and 4 mm, so that after each
    projection the next point is still clearly in contact): a near tie at the first
    point masks all three in that simulation; a tie at the last point, at the state
    the sweep reaches it with, masks only the last, and its flags are branches."""
    c, ob = _tilted()
    prm = O.Params(mu=0.5, gauss_seidel=1)
    h = ob.pitch
    org = ob.origin.numpy()
    x, y = org[0] + 7.31 * h, org[1] + 9.47 * h

    def pt(phi, dx=0.0):
        px = x + dx
        return [px, y, (phi - c[0] * px - c[1] * y) / c[2]]

    q = np.zeros((1, 6))
    m0 = 0                                               # the zero-velocity simulation
    deep = [pt(-2e-3, 0.0), pt(-3e-3, 0.004), pt(-4e-3, 0.008)]
    res = O.decision_band(multi_point_hand(deep), ob, q, 0.0, prm)
    assert not res["masked"][0, :, m0].any()
    # before any projection phi_m = phi: a tie at the first point
    first = [pt(5e-7, 0.0), deep[1], deep[2]]
    res = O.decision_band(multi_point_hand(first), ob, q, 0.0, prm)
    assert res["flag"][0, 0, m0] and res["masked"][0, :, m0].all()
    # the state before the last point (no rotation: inv_inertia = 0): phi_m = phi - n . D
    base = O.evaluate_gs(multi_point_hand(deep), ob, torch.zeros(1, 6, dtype=F64), 0.0, prm)
    st = base["dec"].state[0, 2, m0].numpy()
    assert np.all(st[3:] == 0)
    last = [deep[0], deep[1], pt(float(c @ st[:3]) + 5e-7, 0.008)]
    res = O.decision_band(multi_point_hand(last), ob, q, 0.0, prm)
    # static friction cancelled the tangential part of the state in every simulation, so
    # the last point ties in all seven: each flag is a branch (2^7 combinations)
    assert res["flag"][0, 2].all() and not res["flag"][0, :2].any()
    assert (res["masked"][0] == np.array([[False] * 7, [False] * 7, [True] * 7])).all()
    br = res["branches"][0]
    assert res["comparable"][0] and len(br["L"]) == 128 and len(np.unique(br["L"])) > 1
