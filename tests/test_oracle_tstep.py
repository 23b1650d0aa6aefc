"""Pins of the oracle's T-step form (evaluate_tstep): the object simulated for T
PBD steps per test velocity with the SDF re-queried at the predicted pose
(Sec. III-C, Sec. IV-A; the paper's experiments use T = 1).

  * closed forms: one hand point inside a half-space object (linear field, exact
    under trilinear interpolation), on the line of motion, so that there is no
    lever and no tangential displacement;
  * on a linear field the plane-linearised one-step form is exact, so T = 1 must
    reproduce it (value and gradient), which ties the new code to the pinned one;
  * free flight: a hand far from the object leaves every velocity unchanged;
  * the gradient against central differences of the branch-frozen loss (leaky
    surrogate anchored at the evaluation point) for T = 2 and 3."""

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O

F64 = torch.float64


def _halfspace(a: float, n: int = 16, pitch: float = 0.005):
    """phi(r) = r_x - a on a float64 grid centred on the origin (the object fills x < a)."""
    ax = (torch.arange(n, dtype=F64) - (n - 1) / 2.0) * pitch
    origin = torch.tensor([ax[0], ax[0], ax[0]], dtype=F64)
    X = ax[None, None, :].expand(n, n, n)
    return O.Obj(X - a, origin, pitch, (n, n, n), 1.0, 1.0 / 0.004)


def _one_point_hand(x: float):
    """A palm link with a single point at (x, 0, 0) and no joints (q = base pose only)."""
    T_fix = torch.zeros(1, 3, 4, dtype=F64)
    T_fix[0, :, :3] = torch.eye(3, dtype=F64)
    return O.Hand(L=1, J=0, D=6, P=1, parent=[-1], T_fix=T_fix, axis=torch.zeros(1, 3, dtype=F64),
                  q_low=torch.zeros(0, dtype=F64), q_up=torch.zeros(0, dtype=F64),
                  s=torch.tensor([[x, 0.0, 0.0]], dtype=F64), link=torch.zeros(1, dtype=torch.long))


@pytest.mark.parametrize("T", [1, 2, 3, 5])
def test_closed_form_single_point_in_a_halfspace(T):
    """Point at depth delta inside the half-space x < a, on the x axis.
    Simulation 0 (at rest): C = delta, the correction moves the object by -delta,
    so v = -delta/dt; the next predicted pose is 2 delta away and free: v stays.
    +x (moving into the point): C = delta + dt V, x+ = dt V - C = -delta, the same
    v = -delta/dt.  -x (moving away, dt V > delta): never in contact, v = -V.
    No lever (d is parallel to n) and no tangential displacement: no spin."""
    a, delta = 0.004, 0.0004
    prm = O.Params(alpha_leak=0.1, dt=1e-3, v_test=1.0, mu=0.5, w_range=0.0, w_limit=0.0)
    out = O.evaluate_tstep(_one_point_hand(a - delta), _halfspace(a), torch.zeros(1, 6, dtype=F64),
                           0.0, prm, T)
    v, w = out["xdot"][0], out["thdot"][0]
    exp = -delta / prm.dt
    for m in (0, 1):
        assert torch.allclose(v[m], torch.tensor([exp, 0.0, 0.0], dtype=F64), rtol=0, atol=1e-10), (m, v[m])
    assert torch.allclose(v[2], torch.tensor([-1.0, 0.0, 0.0], dtype=F64), rtol=0, atol=1e-12)
    assert torch.abs(w[:3]).max() < 1e-12
    assert float(out["N"][0, 0]) == 1 and float(out["N"][0, 1]) == 1 and float(out["N"][0, 2]) == 0


@pytest.fixture(scope="module")
def tiny():
    w = synth.tiny_sphere_workload(n_cand=16)
    return w, O.Setup(w.hand, w.objects, w.params)


@pytest.fixture(scope="module")
def linear_setup(tiny):
    """The tiny workload's hand over a linear field: phi = n0 . x + c with a unit
    normal, so the object is a half-space whose boundary crosses the hand."""
    w, S = tiny
    n0 = torch.tensor([0.48, -0.6, 0.64], dtype=F64)
    n0 = n0 / n0.norm()
    N, pitch = 80, 0.008                              # +-0.32 m: the whole hand inside the grid
    ax = (torch.arange(N, dtype=F64) - (N - 1) / 2.0) * pitch
    Z, Y, X = torch.meshgrid(ax, ax, ax, indexing="ij")
    grid = n0[0] * X + n0[1] * Y + n0[2] * Z - 0.07
    obj = O.Obj(grid, torch.tensor([ax[0]] * 3, dtype=F64), pitch, (N, N, N), 1.0, 1.0 / 0.004)
    return S, obj, w.q0.astype(np.float64)


def test_one_step_equals_plane_linearised_form_on_a_linear_field(linear_setup):
    S, obj, q = linear_setup
    prm = S.prm
    lin = O.evaluate(S.hand, obj, torch.tensor(q), 0.004, prm)
    ex = O.evaluate_tstep(S.hand, obj, torch.tensor(q), 0.004, prm, 1)
    assert int(lin["N"].sum()) > 50, "the workload must have contacts"
    assert torch.equal(lin["dec"].kappa, ex["dec"].steps[0].kappa)
    assert torch.allclose(ex["L"], lin["L"], rtol=1e-9, atol=1e-12)
    g_lin = O.loss_and_grad(S.hand, obj, q, 0.004, prm)["grad"]
    prm1 = O.Params(**{**prm.__dict__, "sim_steps": 1})
    g_ex = O.loss_and_grad(S.hand, obj, q, 0.004, prm1)["grad"]
    assert torch.allclose(g_ex, g_lin, rtol=1e-7, atol=1e-9 * float(g_lin.abs().max()))


def test_free_flight_keeps_the_test_velocities(tiny):
    w, S = tiny
    q = w.q0.astype(np.float64).copy()
    q[:, 0:3] += 5.0                                  # hand 5 m away from the object
    for T in (1, 2, 4):
        out = O.evaluate_tstep(S.hand, S.objs[0], torch.tensor(q), 0.004, S.prm, T)
        V = torch.tensor(O.TEST_DIRECTIONS, dtype=F64) * S.prm.v_test
        assert torch.equal(out["xdot"], V[None].expand_as(out["xdot"]))
        assert float(out["thdot"].abs().max()) == 0.0
        assert torch.allclose(out["L_stable"], torch.full_like(out["L_stable"], 6.0 / 7.0), rtol=1e-15)


def _fd_frozen_tstep(S, obj, q, r, prm, T, dec, h):
    B, D = q.shape
    g = np.zeros((B, D))
    for k in range(D):
        e = np.zeros(D)
        e[k] = h
        lp = O.evaluate_tstep(S.hand, obj, torch.tensor(q + e), r, prm, T, dec=dec, anchor_mode=True)["L"]
        lm = O.evaluate_tstep(S.hand, obj, torch.tensor(q - e), r, prm, T, dec=dec, anchor_mode=True)["L"]
        g[:, k] = ((lp - lm) / (2 * h)).detach().numpy()
    return g


@pytest.mark.parametrize("T,alpha", [(2, 0.1), (3, 0.1), (2, 0.0)])
def test_tstep_gradient_matches_frozen_branch_differences(tiny, T, alpha):
    w, S = tiny
    prm = O.Params(**{**S.prm.__dict__, "alpha_leak": alpha, "sim_steps": T})
    q = w.q0.astype(np.float64)[:8]
    out = O.loss_and_grad(S.hand, S.objs[0], q, 0.004, prm)
    assert int(out["N"].sum()) > 0
    # Every simulated step multiplies the higher derivatives by ~1/dt: the central
    # difference's h^2 error is 2e-3 at h = 1e-8 and 2e-5 at 1e-9 for T = 2, and
    # 2e-4 at 1e-10 for T = 3.  Richardson extrapolation of h = 2e-10 and 1e-10
    # cancels the h^2 term; what is left is round-off (~1e-5 relative at worst).
    h = 2e-10
    d1 = _fd_frozen_tstep(S, S.objs[0], q, 0.004, prm, T, out["dec"], h)
    d2 = _fd_frozen_tstep(S, S.objs[0], q, 0.004, prm, T, out["dec"], h / 2)
    fd = (4.0 * d2 - d1) / 3.0
    g = out["grad"].numpy()
    rel = np.linalg.norm(fd - g, axis=1) / np.maximum(np.linalg.norm(g, axis=1), 1e-12)
    assert rel.max() < 2e-5, rel


def test_frozen_tstep_decisions_reproduce_the_method(tiny):
    w, S = tiny
    q = torch.tensor(w.q0.astype(np.float64))
    a = O.evaluate_tstep(S.hand, S.objs[0], q, 0.004, S.prm, 3)
    b = O.evaluate_tstep(S.hand, S.objs[0], q, 0.004, S.prm, 3, dec=a["dec"], anchor_mode=True)
    assert torch.equal(a["L"], b["L"])
