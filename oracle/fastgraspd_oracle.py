"""FP64 CPU oracle of the Fast-Grasp'D grasp-search step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import or call this module.
The product (the CUDA library and its Python binding) never does, and shares no
code with it: the two meet only through the seeded inputs of ``synth``.

What it computes, step by step, in the paper's order (Sec. III-C, Sec. IV-A):

  FK        p = FK(q_h): base pose (t, w) with R_b = Exp(w), then for every link
            T_l = T_parent(l) * T_fix_l * Rot(a_l, theta_j(l)); points p_i = R_l s_i + t_l.
  SDF       trilinear interpolation of a voxel grid (the Grasp'D representation of
            Sec. III-A), with the analytic gradient of the interpolant, an excess
            distance outside the grid, and dilation phi_hat = phi - r (Sec. III-B).
  PBD       M = 7 one-step simulations with test velocities 0, +-x, +-y, +-z (Sec. IV-A);
            object at its canonical pose; each hand point gives the constraint
            C = max(0, -phi) (Sec. III-C) on the plane through the query, and the
            single-constraint projection of Eq. (1) with J = [n^T, (d x n)^T];
            Coulomb friction at position level; corrections averaged over the
            active contacts (Jacobi reading of the Gauss-Seidel step; ``evaluate_gs``
            projects them one after another in point order instead).
  Loss      L_stable of Eq. (2), L_range (Eq. 3), L_limit (Eq. 4) and an optional
            penetration sum; L = L_stable + w_r L_range + w_l L_limit + w_pen L_pen.
  Gradient  reverse mode (torch autograd in float64) with the paper's leaky rule:
            dC/dphi = -1 in contact and -alpha outside (Sec. III-C, "Leaky gradient").
  Update    q <- q - lr * dL/dq (Sec. IV-A); dilation r decreases linearly to 0.

Every branch the method takes (clamp side, voxel cell, contact flag, friction
regime, zero norms, active joint limits) is a recorded *decision*.  ``evaluate``
either takes decisions from the current values (the method itself) or is handed a
frozen set, which turns the loss into one smooth piece; finite differences of that
piece pin the autograd gradient, including the leaky part (see ``tests``).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import mesh_sdf as _mesh

F64 = torch.float64

# Sec. IV-A: zero velocity plus positive and negative velocity along each axis.
TEST_DIRECTIONS = ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))
M_SIMS = len(TEST_DIRECTIONS)


# ----------------------------------------------------------------------------- inputs

@dataclass
class Hand:
    L: int
    J: int
    D: int
    P: int
    parent: list
    T_fix: torch.Tensor        # [L,3,4]
    axis: torch.Tensor         # [L,3]
    q_low: torch.Tensor        # [J]
    q_up: torch.Tensor         # [J]
    s: torch.Tensor            # [P,3] link-local points
    link: torch.Tensor         # [P] long

    @staticmethod
    def from_synth(h: dict) -> "Hand":
        t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64))
        return Hand(h["L"], h["J"], h["D"], h["P"], [int(v) for v in h["parent"]],
                    t(h["T_fix"]), t(h["axis"]), t(h["q_low"]), t(h["q_up"]),
                    t(h["pts_local"]), torch.as_tensor(h["link_of_point"]).long())


@dataclass
class Obj:
    grid: torch.Tensor         # [nz,ny,nx] float64
    origin: torch.Tensor       # [3]
    pitch: float
    dims: tuple                # (nx, ny, nz)
    inv_mass: float
    inv_inertia: float

    @staticmethod
    def from_synth(o: dict) -> "Obj":
        g = o["grid"].detach().to("cpu", F64)
        nz, ny, nx = g.shape
        return Obj(g, torch.as_tensor(np.asarray(o["origin"], dtype=np.float64)),
                   float(o["pitch"]), (nx, ny, nz), 1.0 / float(o["mass"]), 1.0 / float(o["inertia"]))


@dataclass
class Params:
    alpha_leak: float = 0.1
    dt: float = 1e-3
    v_test: float = 1.0
    mu: float = 0.5
    lr: float = 1e-3
    r0: float = 0.004
    w_range: float = 0.1
    w_limit: float = 1.0
    w_pen: float = 0.0
    schedule: str = "fixed"
    sim_steps: int = 0          # 0: one step, plane-linearised query; T >= 1: T steps, re-queried
    gauss_seidel: int = 0       # 0: Jacobi-averaged corrections; 1: Gauss-Seidel in point order (one step)

    @staticmethod
    def from_dict(d: dict) -> "Params":
        keys = Params.__dataclass_fields__.keys()
        return Params(**{k: d[k] for k in keys if k in d})


def dilation_radius(p: Params, step: int, total_steps: int) -> float:
    """Sec. III-B: the surface is the r-level set and r decreases linearly to 0.
    Reading: r_k = r0 * max(0, 1 - k / (K - 1)) over a K-step run ("linear"), or a
    constant r0 ("fixed")."""
    if p.schedule == "fixed":
        return p.r0
    return p.r0 * max(0.0, 1.0 - step / max(total_steps - 1, 1))


# ----------------------------------------------------------------------------- FK

def skew(w: torch.Tensor) -> torch.Tensor:
    z = torch.zeros_like(w[..., 0])
    return torch.stack([torch.stack([z, -w[..., 2], w[..., 1]], -1),
                        torch.stack([w[..., 2], z, -w[..., 0]], -1),
                        torch.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def so3_exp(w: torch.Tensor) -> torch.Tensor:
    """Rodrigues: Exp(w) = I + sin(a)/a [w]x + (1 - cos a)/a^2 [w]x^2, a = |w|;
    the series I + [w]x + [w]x^2/2 below |w| = 1e-8."""
    a2 = (w * w).sum(-1)
    small = a2 < 1e-16
    a = torch.sqrt(torch.where(small, torch.ones_like(a2), a2))
    c1 = torch.where(small, 1.0 - a2 / 6.0, torch.sin(a) / a)
    c2 = torch.where(small, 0.5 - a2 / 24.0, (1.0 - torch.cos(a)) / (a * a))
    K = skew(w)
    eye = torch.eye(3, dtype=w.dtype).expand(K.shape)
    return eye + c1[..., None, None] * K + c2[..., None, None] * (K @ K)


def axis_rotation(axis: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
    """Rotation by theta about the unit axis (Rodrigues with a unit axis)."""
    K = skew(axis).expand(theta.shape + (3, 3))
    eye = torch.eye(3, dtype=theta.dtype).expand(K.shape)
    return eye + torch.sin(theta)[..., None, None] * K + (1.0 - torch.cos(theta))[..., None, None] * (K @ K)


def forward_kinematics(hand: Hand, q: torch.Tensor):
    """Link frames for q = (t, w, theta): returns R [B,L,3,3], o [B,L,3] (Sec. III-C, p = FK(q_h))."""
    t, w, th = q[:, 0:3], q[:, 3:6], q[:, 6:]
    Rs, os_ = [so3_exp(w)], [t]
    for l in range(1, hand.L):
        par = hand.parent[l]
        Rf, tf = hand.T_fix[l, :, :3], hand.T_fix[l, :, 3]
        Rj = axis_rotation(hand.axis[l], th[:, l - 1])
        Rs.append(Rs[par] @ Rf @ Rj)
        os_.append(os_[par] + (Rs[par] @ tf[:, None])[..., 0])
    return torch.stack(Rs, 1), torch.stack(os_, 1)


def hand_points(hand: Hand, R: torch.Tensor, o: torch.Tensor) -> torch.Tensor:
    """p_i = R_l(i) s_i + o_l(i) for all points: [B,P,3]."""
    Rl, ol = R[:, hand.link], o[:, hand.link]
    return (Rl @ hand.s[None, :, :, None])[..., 0] + ol


# ----------------------------------------------------------------------------- SDF

def _safe_norm(x: torch.Tensor, nonzero: torch.Tensor):
    sq = (x * x).sum(-1)
    return torch.where(nonzero, torch.sqrt(torch.where(nonzero, sq, torch.ones_like(sq))),
                       torch.zeros_like(sq))


def sdf_decisions(obj: Obj, p: torch.Tensor) -> dict:
    """Branches of the grid lookup: per axis clamped below/above, and the cell index
    i0 = min(floor(clamp(u, 0, n-1)), n-2).  For a mesh object, the mesh query's
    (closest face, sign, Phong point; oracle/mesh_sdf.py)."""
    if isinstance(obj, _mesh.MeshObj):
        return _mesh.mesh_decisions(obj, p)
    with torch.no_grad():
        n = torch.tensor(obj.dims, dtype=F64)
        u = (p - obj.origin) / obj.pitch
        lo, hi = u < 0, u > n - 1
        uc = torch.minimum(torch.maximum(u, torch.zeros_like(u)), n - 1)
        i0 = torch.minimum(torch.floor(uc), n - 2).long()
    return {"lo": lo, "hi": hi, "i0": i0}


def sdf_eval(obj: Obj, p: torch.Tensor, dec: dict):
    """phi and its gradient for given branch decisions (Sec. III-A grid + trilinear).

    u = (p - origin)/h; u_c = u clamped into [0, n-1] (per the decisions);
    f = u_c - i0; phi = trilinear(G, i0, f) + h |u - u_c|;
    grad = (1/h) d trilinear/d f on unclamped axes + (u - u_c)/|u - u_c| outside.
    For a mesh object: the Phong SDF rho and its gradient (oracle/mesh_sdf.py)."""
    if isinstance(obj, _mesh.MeshObj):
        return _mesh.mesh_eval(obj, p, dec)
    n = torch.tensor(obj.dims, dtype=F64)
    h = obj.pitch
    u = (p - obj.origin) / h
    lo, hi, i0 = dec["lo"], dec["hi"], dec["i0"]
    uc = torch.where(lo, torch.zeros_like(u), torch.where(hi, (n - 1).expand_as(u), u))
    du = u - uc
    outside = lo.any(-1) | hi.any(-1)
    e = h * _safe_norm(du, outside)
    f = uc - i0.to(F64)
    ix, iy, iz = i0[..., 0], i0[..., 1], i0[..., 2]
    G = obj.grid
    val = torch.zeros_like(f[..., 0])
    dval = [torch.zeros_like(val) for _ in range(3)]
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                corner = G[iz + c, iy + b, ix + a]
                wx = f[..., 0] if a else 1.0 - f[..., 0]
                wy = f[..., 1] if b else 1.0 - f[..., 1]
                wz = f[..., 2] if c else 1.0 - f[..., 2]
                sx, sy, sz = (1.0 if a else -1.0), (1.0 if b else -1.0), (1.0 if c else -1.0)
                val = val + wx * wy * wz * corner
                dval[0] = dval[0] + sx * wy * wz * corner
                dval[1] = dval[1] + wx * sy * wz * corner
                dval[2] = dval[2] + wx * wy * sz * corner
    interior = ~(lo | hi)
    g_tri = torch.stack(dval, -1) / h * interior.to(F64)
    den = _safe_norm(du, outside)[..., None]
    g_out = torch.where(outside[..., None], du / torch.where(outside[..., None], den, torch.ones_like(den)),
                        torch.zeros_like(du))
    return val + e, g_tri + g_out


def sdf_query(obj: Obj, p: torch.Tensor, r: float):
    """Dilated SDF phi_hat = phi - r (Sec. III-B) and the gradient of phi, for points p [...,3]."""
    phi, grad = sdf_eval(obj, p, sdf_decisions(obj, p))
    return phi - r, grad


# ----------------------------------------------------------------------------- step

def _forced(taken: torch.Tensor, force: dict | None, key: str, i: int | None = None) -> torch.Tensor:
    """A decision taken from the values, except where ``force[key] = (mask, value)``
    sets it ([B,P,M] tables; ``i`` selects point i of them)."""
    if force is None or key not in force:
        return taken
    mask, value = force[key]
    if i is not None:
        mask, value = mask[:, i], value[:, i]
    return torch.where(mask, value, taken)


def _forced_cells(sdf_dec: dict, force: dict | None) -> dict:
    """Grid lookup decisions, except at the points where ``force["sdf"] = (mask [B,P],
    decisions)`` gives them."""
    if force is None or "sdf" not in force:
        return sdf_dec
    mask, alt = force["sdf"]
    return {k: torch.where(mask[..., None], alt[k], v) for k, v in sdf_dec.items()}


@dataclass
class Decisions:
    sdf: dict = None
    grad_nz: torch.Tensor = None     # [B,P]   |grad phi| > 0
    kappa: torch.Tensor = None       # [B,P,M] contact flag phi_m < 0
    has_t: torch.Tensor = None       # [B,P,M] tangential displacement sigma > 0
    static: torch.Tensor = None      # [B,P,M] sigma <= mu C
    anchor: torch.Tensor = None      # [B,P,M] phi_m at the decision state (leak surrogate)
    v_nz: torch.Tensor = None        # [B,M]   |x_dot+| > 0
    w_nz: torch.Tensor = None        # [B,M]   |theta_dot+| > 0
    range_nz: torch.Tensor = None    # [B]     |theta - mid| > 0
    above: torch.Tensor = None       # [B,J]   theta > q_up
    below: torch.Tensor = None       # [B,J]   theta < q_low
    ncontact: torch.Tensor = None    # [B,M]   N_m (a constant in the gradient)


def _cross(a, b):
    return torch.linalg.cross(a, b, dim=-1)


def _dot(a, b):
    return (a * b).sum(-1)


def evaluate(hand: Hand, obj: Obj, q: torch.Tensor, r: float, prm: Params,
             dec: Decisions | None = None, anchor_mode: bool = False, force: dict | None = None) -> dict:
    """One grasp-metric evaluation for a batch of candidates on one object.

    With ``dec=None`` every decision is taken from the current values (the method).
    With a frozen ``dec`` the same arithmetic is evaluated on that branch; with
    ``anchor_mode`` non-contact constraints use C = -alpha (phi_m - anchor), whose
    value is 0 at the anchor state and whose slope is the leaky -alpha.
    ``force`` (with ``dec=None``) sets some decisions while the others are taken
    from the values (see ``_forced``).
    Returns a dict of per-candidate tensors and the decisions used."""
    take = dec is None
    if take:
        dec = Decisions()
    B = q.shape[0]
    R, o = forward_kinematics(hand, q)
    p = hand_points(hand, R, o)                                      # [B,P,3]
    if take:
        dec.sdf = _forced_cells(sdf_decisions(obj, p), force)
    phi, grad = sdf_eval(obj, p, dec.sdf)
    phi_hat = phi - r
    if take:
        dec.grad_nz = (grad.detach() * grad.detach()).sum(-1) > 0
    gnorm = _safe_norm(grad, dec.grad_nz)
    nrm = grad / torch.where(dec.grad_nz, gnorm, torch.ones_like(gnorm))[..., None]

    V = torch.tensor(TEST_DIRECTIONS, dtype=F64) * prm.v_test         # [M,3]
    v = V[None, None]                                                 # [1,1,M,3]
    x_pred = prm.dt * v                                               # symplectic Euler, x^- = 0
    n_ = nrm[:, :, None, :]                                           # [B,P,1,3]
    p_ = p[:, :, None, :]
    # constraint on the plane through the query: phi(p - x_pred) ~ phi_hat - n . x_pred
    phi_m = phi_hat[..., None] - _dot(n_, x_pred)                     # [B,P,M]
    if take:
        dec.kappa = _forced(phi_m.detach() < 0, force, "kappa")
    if anchor_mode:
        anchor = dec.anchor
    else:
        anchor = phi_m.detach()
        if take:
            dec.anchor = anchor
    alpha = prm.alpha_leak
    # C = max(0, -phi_m); outside contact the value is 0 and the slope is -alpha
    C = torch.where(dec.kappa, -phi_m, -alpha * (phi_m - anchor))
    d = p_ - x_pred                                                   # lever arm from the object centre
    u_n = _cross(d, n_.expand_as(d))
    w_n = obj.inv_mass + obj.inv_inertia * _dot(u_n, u_n)        # J M^-1 J^T, Eq. (1)
    lam_n = C / w_n
    s = prm.dt * (v - _dot(v, n_)[..., None] * n_)                    # tangential displacement
    if take:
        dec.has_t = (s.detach() * s.detach()).sum(-1) > 0
    sig = _safe_norm(s, dec.has_t)
    t_hat = s / torch.where(dec.has_t, sig, torch.ones_like(sig))[..., None]
    u_t = _cross(d, t_hat)
    w_t = obj.inv_mass + obj.inv_inertia * _dot(u_t, u_t)
    if take:
        dec.static = _forced(sig.detach() <= prm.mu * C.detach(), force, "static")
    lam_t = torch.where(dec.has_t, torch.where(dec.static, sig, prm.mu * C) / w_t, torch.zeros_like(sig))
    f = -(lam_n[..., None] * n_ + lam_t[..., None] * t_hat)          # [B,P,M,3]
    W_lin = f.sum(1)                                                  # [B,M,3]
    W_ang = _cross(d, f).sum(1)
    if take:
        dec.ncontact = dec.kappa.sum(1).to(F64)                       # [B,M]
    Nc = torch.clamp(dec.ncontact, min=1.0)
    dx = W_lin * obj.inv_mass / Nc[..., None]                         # averaged position correction
    dth = W_ang * obj.inv_inertia / Nc[..., None]
    xdot = V[None] + dx / prm.dt                                      # x_dot+ = (x+ - x-)/dt
    thdot = dth / prm.dt
    if take:
        dec.v_nz = (xdot.detach() ** 2).sum(-1) > 0
        dec.w_nz = (thdot.detach() ** 2).sum(-1) > 0
    L_stable = (_safe_norm(xdot, dec.v_nz) + _safe_norm(thdot, dec.w_nz)).sum(-1) / M_SIMS   # Eq. (2)

    th = q[:, 6:]
    mid = 0.5 * (hand.q_up + hand.q_low)
    if take:
        dec.range_nz = ((th.detach() - mid) ** 2).sum(-1) > 0
        dec.above = th.detach() > hand.q_up
        dec.below = th.detach() < hand.q_low
    L_range = _safe_norm(th - mid, dec.range_nz)                                             # Eq. (3)
    L_limit = (torch.where(dec.above, th - hand.q_up, torch.zeros_like(th)) +
               torch.where(dec.below, hand.q_low - th, torch.zeros_like(th))).sum(-1)        # Eq. (4)
    L_pen = C[..., 0].sum(-1)
    L = L_stable + prm.w_range * L_range + prm.w_limit * L_limit + prm.w_pen * L_pen
    return {"L": L, "L_stable": L_stable, "L_range": L_range, "L_limit": L_limit, "L_pen": L_pen,
            "W": torch.cat([W_lin, W_ang], -1), "N": dec.ncontact, "kappa": dec.kappa,
            "points": p, "phi_hat": phi_hat, "grad_phi": grad, "phi_m": phi_m, "C": C,
            "sigma": sig, "dec": dec}


@dataclass
class StepDecisions:
    """Branches of one simulation step of the T-step form (per point and simulation)."""
    sdf: dict = None
    grad_nz: torch.Tensor = None     # [B,P,M]
    kappa: torch.Tensor = None       # [B,P,M]
    has_t: torch.Tensor = None       # [B,P,M]
    static: torch.Tensor = None      # [B,P,M]
    anchor: torch.Tensor = None      # [B,P,M]
    ncontact: torch.Tensor = None    # [B,M]


@dataclass
class TStepDecisions:
    steps: list = field(default_factory=list)
    v_nz: torch.Tensor = None
    w_nz: torch.Tensor = None
    range_nz: torch.Tensor = None
    above: torch.Tensor = None
    below: torch.Tensor = None


def _joint_losses(hand: Hand, q: torch.Tensor, dec):
    th = q[:, 6:]
    mid = 0.5 * (hand.q_up + hand.q_low)
    if dec.range_nz is None:
        dec.range_nz = ((th.detach() - mid) ** 2).sum(-1) > 0
        dec.above = th.detach() > hand.q_up
        dec.below = th.detach() < hand.q_low
    L_range = _safe_norm(th - mid, dec.range_nz)                                             # Eq. (3)
    L_limit = (torch.where(dec.above, th - hand.q_up, torch.zeros_like(th)) +
               torch.where(dec.below, hand.q_low - th, torch.zeros_like(th))).sum(-1)        # Eq. (4)
    return L_range, L_limit


def evaluate_tstep(hand: Hand, obj: Obj, q: torch.Tensor, r: float, prm: Params, T: int,
                   dec: TStepDecisions | None = None, anchor_mode: bool = False) -> dict:
    """The grasp metric with T simulation steps per test velocity (Sec. IV-A: the
    object's velocity after T steps; the paper's experiments take T = 1).

    Each simulation starts at the canonical pose with velocity V e_m and no spin.
    One step (Sec. III-C):
      predict (symplectic Euler, no external force)  x~ = x + dt v,  R~ = Exp(dt w) R;
      every hand point in the object frame at the predicted pose, r = R~^T (p - x~),
      re-queried in the SDF: phi_hat = phi(r) - r_dil, world normal n = R~ grad/|grad|;
      C = max(0, -phi_hat) with the leaky rule; the projection of Eq. (1) with lever
      d = p - x~; Coulomb friction on the tangential part of the displacement of the
      object's material point at the contact, s = p - (x + R r);
      corrections averaged over the N active contacts (Jacobi reading):
      x+ = x~ + dx,  R+ = Exp(dtheta) R~,  v+ = (x+ - x)/dt,  w+ = w + dtheta/dt.
    L_stable (Eq. 2) on (v, w) after T steps.  At T = 1 this is the one-step metric
    with the SDF evaluated at the moved pose instead of on the plane through the
    query; on a linear field the two coincide."""
    take = dec is None
    if take:
        dec = TStepDecisions()
    B = q.shape[0]
    M = M_SIMS
    Rh, oh = forward_kinematics(hand, q)
    p = hand_points(hand, Rh, oh)                                     # [B,P,3], the hand is static
    P = p.shape[1]
    V = torch.tensor(TEST_DIRECTIONS, dtype=F64) * prm.v_test         # [M,3]
    x = torch.zeros(B, M, 3, dtype=F64)
    Rb = torch.eye(3, dtype=F64).expand(B, M, 3, 3)
    v = V[None].expand(B, M, 3)
    w = torch.zeros(B, M, 3, dtype=F64)
    alpha = prm.alpha_leak
    pe = p[:, :, None, :]                                             # [B,P,1,3]
    C_first = None
    trace = []
    for t in range(T):
        sd = StepDecisions() if take else dec.steps[t]
        x_t = x + prm.dt * v                                          # [B,M,3]
        R_t = so3_exp(prm.dt * w) @ Rb                                # [B,M,3,3]
        d = pe - x_t[:, None]                                         # [B,P,M,3]
        rr = (R_t.transpose(-1, -2)[:, None] @ d[..., None])[..., 0]  # object frame
        if take:
            sd.sdf = sdf_decisions(obj, rr)
        phi, g_obj = sdf_eval(obj, rr, sd.sdf)
        phi_hat = phi - r
        if take:
            sd.grad_nz = (g_obj.detach() * g_obj.detach()).sum(-1) > 0
        gn = _safe_norm(g_obj, sd.grad_nz)
        n_obj = g_obj / torch.where(sd.grad_nz, gn, torch.ones_like(gn))[..., None]
        n = (R_t[:, None] @ n_obj[..., None])[..., 0]                 # world normal
        if take:
            sd.kappa = phi_hat.detach() < 0
        if anchor_mode:
            anchor = sd.anchor
        else:
            anchor = phi_hat.detach()
            if take:
                sd.anchor = anchor
        C = torch.where(sd.kappa, -phi_hat, -alpha * (phi_hat - anchor))
        if t == 0:
            C_first = C
        u_n = _cross(d, n)
        w_n = obj.inv_mass + obj.inv_inertia * _dot(u_n, u_n)
        lam_n = C / w_n
        s_raw = pe - x[:, None] - (Rb[:, None] @ rr[..., None])[..., 0]
        s = s_raw - _dot(s_raw, n)[..., None] * n
        if take:
            sd.has_t = (s.detach() * s.detach()).sum(-1) > 0
        sig = _safe_norm(s, sd.has_t)
        t_hat = s / torch.where(sd.has_t, sig, torch.ones_like(sig))[..., None]
        u_t = _cross(d, t_hat)
        w_t = obj.inv_mass + obj.inv_inertia * _dot(u_t, u_t)
        if take:
            sd.static = sig.detach() <= prm.mu * C.detach()
        lam_t = torch.where(sd.has_t, torch.where(sd.static, sig, prm.mu * C) / w_t, torch.zeros_like(sig))
        f = -(lam_n[..., None] * n + lam_t[..., None] * t_hat)
        W_lin = f.sum(1)
        W_ang = _cross(d, f).sum(1)
        if t == 0:
            W_first = torch.cat([W_lin, W_ang], -1)
        trace.append({"r": rr.detach(), "phi_hat": phi_hat.detach(), "C": C.detach(), "sigma": sig.detach(),
                      "s_raw": _safe_norm(s_raw.detach(), torch.ones_like(sd.kappa)), "kappa": sd.kappa,
                      "has_t": sd.has_t})
        if take:
            sd.ncontact = sd.kappa.sum(1).to(F64)
        Nc = torch.clamp(sd.ncontact, min=1.0)
        dx = W_lin * obj.inv_mass / Nc[..., None]
        dth = W_ang * obj.inv_inertia / Nc[..., None]
        x_new = x_t + dx
        R_new = so3_exp(dth) @ R_t
        v = (x_new - x) / prm.dt
        w = w + dth / prm.dt
        x, Rb = x_new, R_new
        if take:
            dec.steps.append(sd)
    if take:
        dec.v_nz = (v.detach() ** 2).sum(-1) > 0
        dec.w_nz = (w.detach() ** 2).sum(-1) > 0
    L_stable = (_safe_norm(v, dec.v_nz) + _safe_norm(w, dec.w_nz)).sum(-1) / M_SIMS       # Eq. (2)
    L_range, L_limit = _joint_losses(hand, q, dec)
    L_pen = C_first[..., 0].sum(-1)
    L = L_stable + prm.w_range * L_range + prm.w_limit * L_limit + prm.w_pen * L_pen
    return {"L": L, "L_stable": L_stable, "L_range": L_range, "L_limit": L_limit, "L_pen": L_pen,
            "xdot": v, "thdot": w, "W": W_first, "N": dec.steps[0].ncontact, "kappa": dec.steps[0].kappa,
            "points": p, "dec": dec, "trace": trace}


@dataclass
class GSDecisions:
    """Branches of the Gauss-Seidel form (per point and simulation unless noted)."""
    sdf: dict = None
    grad_nz: torch.Tensor = None     # [B,P]
    kappa: torch.Tensor = None       # [B,P,M]
    has_t: torch.Tensor = None       # [B,P,M]
    static: torch.Tensor = None      # [B,P,M]
    anchor: torch.Tensor = None      # [B,P,M] leak surrogate: phi_m at the decision state
    state: torch.Tensor = None       # [B,P,M,6] (dx, dth) before each point at the decision state
    v_nz: torch.Tensor = None
    w_nz: torch.Tensor = None
    range_nz: torch.Tensor = None
    above: torch.Tensor = None
    below: torch.Tensor = None


def evaluate_gs(hand: Hand, obj: Obj, q: torch.Tensor, r: float, prm: Params,
                dec: GSDecisions | None = None, anchor_mode: bool = False, force: dict | None = None) -> dict:
    """The one-step grasp metric with the constraints projected by a Gauss-Seidel
    sweep (Sec. III-C: the update of Eq. (1) for each constraint, applied in turn).

    Everything up to the constraint is the one-step form of ``evaluate``: FK, one SDF
    query per point, the plane through it, the 7 test velocities.  Each simulation
    keeps a correction state (dx, dth), zero at the predicted pose x~ = dt v_m, and
    visits the hand points in index order.  Point i sees the object's material
    point at p_i displaced by D = dt v_m + dx + dth x d (d = p_i - x~, the lever
    held at the predicted pose), so
        phi_m  = phi_hat_i - n_i . D,         C = max(0, -phi_m),
        lambda_n = C / w_n (Eq. 1),           Coulomb friction on s = D - (D . n) n,
    exactly the per-point correction of the Jacobi form evaluated at the current
    state, and the correction M^-1 [f; d x f] is added to the state in full (no
    averaging).  x_dot+ = v_m + dx / dt, theta_dot+ = dth / dt and the loss follow
    Eqs. (2)-(4).

    Leaky rule (Sec. III-C states the biased derivative of C with respect to the hand
    point): outside contact C = -alpha (phi_m - anchor) is taken through the hand
    point only; the state that earlier projections left is held constant in it, so a
    non-contact constraint neither moves the state nor passes gradient between
    states (its exact derivative with respect to the state is 0).  With a frozen
    ``dec`` and ``anchor_mode`` that state is the one recorded at the decision point,
    which makes the leaky gradient the exact gradient of the frozen surrogate.
    ``force`` (with ``dec=None``) sets some decisions while the others, later ones
    of the sweep included, are taken from the values (see ``_forced``)."""
    take = dec is None
    if take:
        dec = GSDecisions()
    B = q.shape[0]
    P = hand.P
    R, o = forward_kinematics(hand, q)
    p = hand_points(hand, R, o)                                      # [B,P,3]
    if take:
        dec.sdf = _forced_cells(sdf_decisions(obj, p), force)
    phi, grad = sdf_eval(obj, p, dec.sdf)
    phi_hat = phi - r
    if take:
        dec.grad_nz = (grad.detach() * grad.detach()).sum(-1) > 0
    gnorm = _safe_norm(grad, dec.grad_nz)
    nrm = grad / torch.where(dec.grad_nz, gnorm, torch.ones_like(gnorm))[..., None]

    V = torch.tensor(TEST_DIRECTIONS, dtype=F64) * prm.v_test         # [M,3]
    x_pred = (prm.dt * V)[None]                                       # [1,M,3]
    alpha = prm.alpha_leak
    if take:
        dec.kappa = torch.zeros(B, P, M_SIMS, dtype=torch.bool)
        dec.has_t = torch.zeros(B, P, M_SIMS, dtype=torch.bool)
        dec.static = torch.zeros(B, P, M_SIMS, dtype=torch.bool)
        dec.anchor = torch.zeros(B, P, M_SIMS, dtype=F64)
        dec.state = torch.zeros(B, P, M_SIMS, 6, dtype=F64)
    dx = torch.zeros(B, M_SIMS, 3, dtype=F64)
    dth = torch.zeros(B, M_SIMS, 3, dtype=F64)
    Wsum = torch.zeros(B, M_SIMS, 6, dtype=F64)
    phi_ms, Cs, sigs = [], [], []
    # per-point views (unbind: the reverse pass gathers their gradients once)
    p_i, n_i, ph_i = p.unbind(1), nrm.unbind(1), phi_hat.unbind(1)
    for i in range(P):
        n_ = n_i[i][:, None, :].expand(B, M_SIMS, 3)
        d = p_i[i][:, None, :] - x_pred                               # [B,M,3]
        Dsp = x_pred + dx + _cross(dth, d)                            # material point's displacement
        phi_m = ph_i[i][:, None] - _dot(n_, Dsp)                      # [B,M]
        if take:
            dec.state[:, i] = torch.cat([dx, dth], -1).detach()
            dec.kappa[:, i] = _forced(phi_m.detach() < 0, force, "kappa", i)
        if anchor_mode:
            st = dec.state[:, i].clone()
            dx_c, dth_c = st[..., :3], st[..., 3:]
        else:
            dx_c, dth_c = dx.detach(), dth.detach()
        phi_p = ph_i[i][:, None] - _dot(n_, x_pred + dx_c + _cross(dth_c, d))
        if take:
            dec.anchor[:, i] = phi_p.detach()
        anchor = dec.anchor[:, i].clone() if anchor_mode else phi_p.detach()
        kap = dec.kappa[:, i].clone()           # copies: the decision tables are filled in place
        C = torch.where(kap, -phi_m, -alpha * (phi_p - anchor))
        u_n = _cross(d, n_)
        w_n = obj.inv_mass + obj.inv_inertia * _dot(u_n, u_n)
        lam_n = C / w_n
        s = Dsp - _dot(Dsp, n_)[..., None] * n_                       # tangential displacement
        if take:
            dec.has_t[:, i] = (s.detach() * s.detach()).sum(-1) > 0
        ht = dec.has_t[:, i].clone()
        sig = _safe_norm(s, ht)
        t_hat = s / torch.where(ht, sig, torch.ones_like(sig))[..., None]
        u_t = _cross(d, t_hat)
        w_t = obj.inv_mass + obj.inv_inertia * _dot(u_t, u_t)
        if take:
            dec.static[:, i] = _forced(sig.detach() <= prm.mu * C.detach(), force, "static", i)
        stat = dec.static[:, i].clone()
        lam_t = torch.where(ht, torch.where(stat, sig, prm.mu * C) / w_t, torch.zeros_like(sig))
        f = -(lam_n[..., None] * n_ + lam_t[..., None] * t_hat)       # [B,M,3]
        tq = _cross(d, f)
        dx = dx + obj.inv_mass * f
        dth = dth + obj.inv_inertia * tq
        Wsum = Wsum + torch.cat([f, tq], -1)
        phi_ms.append(phi_m)
        Cs.append(C)
        sigs.append(sig)
    xdot = V[None] + dx / prm.dt
    thdot = dth / prm.dt
    if take:
        dec.v_nz = (xdot.detach() ** 2).sum(-1) > 0
        dec.w_nz = (thdot.detach() ** 2).sum(-1) > 0
    L_stable = (_safe_norm(xdot, dec.v_nz) + _safe_norm(thdot, dec.w_nz)).sum(-1) / M_SIMS   # Eq. (2)
    L_range, L_limit = _joint_losses(hand, q, dec)
    C = torch.stack(Cs, 1)                                            # [B,P,M]
    L_pen = C[..., 0].sum(-1)
    L = L_stable + prm.w_range * L_range + prm.w_limit * L_limit + prm.w_pen * L_pen
    return {"L": L, "L_stable": L_stable, "L_range": L_range, "L_limit": L_limit, "L_pen": L_pen,
            "W": Wsum, "N": dec.kappa.sum(1).to(F64), "kappa": dec.kappa, "dx": dx, "dth": dth,
            "points": p, "phi_hat": phi_hat, "grad_phi": grad, "phi_m": torch.stack(phi_ms, 1), "C": C,
            "sigma": torch.stack(sigs, 1), "dec": dec}


def evaluate_any(hand: Hand, obj: Obj, q: torch.Tensor, r: float, prm: Params, dec=None,
                 anchor_mode: bool = False, force: dict | None = None) -> dict:
    """evaluate (sim_steps = 0), evaluate_gs (sim_steps = 0, gauss_seidel = 1) or
    evaluate_tstep (sim_steps = T >= 1)."""
    if prm.sim_steps >= 1:
        return evaluate_tstep(hand, obj, q, r, prm, prm.sim_steps, dec=dec, anchor_mode=anchor_mode)
    if prm.gauss_seidel:
        return evaluate_gs(hand, obj, q, r, prm, dec=dec, anchor_mode=anchor_mode, force=force)
    return evaluate(hand, obj, q, r, prm, dec=dec, anchor_mode=anchor_mode, force=force)


def loss_and_grad(hand: Hand, obj: Obj, q32, r: float, prm: Params, alpha=None):
    """Loss, gradient dL/dq (leaky rule) and the forward outputs for candidates q [B,D]."""
    if alpha is not None:
        prm = Params(**{**prm.__dict__, "alpha_leak": alpha})
    q = torch.as_tensor(np.asarray(q32, dtype=np.float64)).clone().requires_grad_(True)
    out = evaluate_any(hand, obj, q, r, prm)
    (g,) = torch.autograd.grad(out["L"].sum(), q)
    out["grad"] = g
    return out


# ----------------------------------------------------------------------------- driver

class Setup:
    """Hand, objects and parameters of one workload, converted for the oracle."""

    def __init__(self, hand: dict, objects: list, params: dict):
        self.hand = Hand.from_synth(hand)
        self.objs = [_mesh.MeshObj.from_synth(o) if "faces" in o else Obj.from_synth(o) for o in objects]
        self.prm = Params.from_dict(params)


def batch_loss_and_grad(setup: Setup, q32: np.ndarray, obj_of_cand: np.ndarray, r: float,
                        chunk: int = 8) -> dict:
    """loss_and_grad over a mixed-object batch, processed per object in small chunks."""
    B = q32.shape[0]
    res = {"L": np.zeros(B), "grad": np.zeros((B, setup.hand.D)), "W": np.zeros((B, M_SIMS, 6)),
           "N": np.zeros((B, M_SIMS)), "kappa": np.zeros((B, setup.hand.P, M_SIMS), dtype=bool),
           "L_stable": np.zeros(B)}
    for k in np.unique(obj_of_cand):
        idx = np.nonzero(obj_of_cand == k)[0]
        for s in range(0, len(idx), chunk):
            sel = idx[s:s + chunk]
            out = loss_and_grad(setup.hand, setup.objs[int(k)], q32[sel], r, setup.prm)
            res["L"][sel] = out["L"].detach().numpy()
            res["L_stable"][sel] = out["L_stable"].detach().numpy()
            res["grad"][sel] = out["grad"].numpy()
            res["W"][sel] = out["W"].detach().numpy()
            res["N"][sel] = out["N"].numpy()
            res["kappa"][sel] = out["kappa"].numpy()
    return res


def optimize(setup: Setup, q32: np.ndarray, obj_of_cand: np.ndarray, step0: int, nsteps: int,
             total_steps: int, round_to_f32: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """nsteps of gradient descent q <- q - lr dL/dq (Sec. IV-A).  Returns (q, loss at
    the last step before its update)."""
    q = np.asarray(q32, dtype=np.float64).copy()
    last = None
    for k in range(step0, step0 + nsteps):
        r = dilation_radius(setup.prm, k, total_steps)
        res = batch_loss_and_grad(setup, q, obj_of_cand, r)
        q = q - setup.prm.lr * res["grad"]
        if round_to_f32:
            q = q.astype(np.float32).astype(np.float64)
        last = res["L"]
    return q, last


# ----------------------------------------------------------------------------- guard band

def _face_margin(obj: Obj, pts: torch.Tensor) -> torch.Tensor:
    """Per point and axis, the distance (in voxels) of the lookup's decision from its
    threshold: inside the grid range the cell choice (distance to the nearest
    node plane), outside it the clamp (distance to the clamp plane).  For a mesh,
    ten times (in metres) the smallest of: the gap to the next distinct closest
    point (the face choice); the distance to the flat surface (the sign); the gap to
    a face whose closest point lies elsewhere (gap_dir), scaled so that float32's
    resolution of distances, 5e-8 m + 3e-7 of the distance, counts as 1
    micrometre; and the distance to the Phong point scaled by 1e-2, so that 1e-4 m
    counts as 1 micrometre (the Phong SDF's gradient field turns at the rate
    1/|p - r*_rho|, and float32 positions, good to ~1e-8 m, leave the adjoint's
    second-order term of a closer point uncertain by more than 1e-4 of itself).
    The default tolerance of 1e-5 is 1 micrometre."""
    if isinstance(obj, _mesh.MeshObj):
        with torch.no_grad():
            dec = _mesh.mesh_decisions(obj, pts)
            res32 = 5e-8 + 3e-7 * dec["dist"]
            d_rho = torch.linalg.norm(pts - dec["q_rho"], dim=-1)
            m = torch.minimum(torch.minimum(dec["gap"], dec["dist"]),
                              torch.minimum(dec["gap_dir"] * (1e-6 / res32), 1e-2 * d_rho))
            return (10.0 * m)[..., None]
    n = torch.tensor(obj.dims, dtype=F64)
    u = (pts - obj.origin) / obj.pitch
    uc = torch.minimum(torch.maximum(u, torch.zeros_like(u)), n - 1)
    inside = u == uc
    return torch.where(inside, (u - torch.round(u)).abs(), (u - uc).abs())


def guard_margins_tstep(hand: Hand, obj: Obj, q32, r: float, prm: Params) -> dict:
    """guard_margins for the T-step form: the same distances over every step and
    simulation (object-frame query points r, phi_hat, friction regime), and the
    sine of the angle between the normal and the material point's displacement."""
    with torch.no_grad():
        q = torch.as_tensor(np.asarray(q32, dtype=np.float64))
        out = evaluate_tstep(hand, obj, q, r, prm, prm.sim_steps)
        inf = float("inf")
        B = q.shape[0]
        face = torch.full((B,), inf, dtype=F64)
        phim = torch.full((B,), inf, dtype=F64)
        fr = torch.full((B,), inf, dtype=F64)
        par = torch.full((B,), inf, dtype=F64)
        for tr in out["trace"]:
            face = torch.minimum(face, _face_margin(obj, tr["r"]).amin(dim=(1, 2, 3)))
            phim = torch.minimum(phim, tr["phi_hat"].abs().amin(dim=(1, 2)))
            f = (tr["sigma"] - prm.mu * tr["C"]).abs()
            f = torch.where(tr["kappa"] & tr["has_t"], f, torch.full_like(f, inf)).amin(dim=(1, 2))
            fr = torch.minimum(fr, f)
            moving = tr["s_raw"] > 0
            ratio = torch.where(moving, tr["sigma"] / torch.where(moving, tr["s_raw"], torch.ones_like(tr["s_raw"])),
                                torch.full_like(tr["sigma"], inf))
            par = torch.minimum(par, ratio.amin(dim=(1, 2)))
    return {"face": face.numpy(), "phi": phim.numpy(), "friction": fr.numpy(), "parallel": par.numpy()}


def guard_margins(hand: Hand, obj: Obj, q32, r: float, prm: Params) -> dict:
    """Distances of every decision from its threshold, per candidate (minimum over
    points): voxel faces / clamp planes (in voxels), |phi_m| for the contact flag
    (metres), |sigma - mu C| for the friction regime of contact points (metres) and
    sigma / (dt V) = sin(angle between n and v_m) for the moving simulations, where a
    normal nearly parallel to the test velocity leaves the friction direction
    ill-conditioned."""
    with torch.no_grad():
        q = torch.as_tensor(np.asarray(q32, dtype=np.float64))
        out = evaluate(hand, obj, q, r, prm)
        face = _face_margin(obj, out["points"]).amin(dim=(-1, -2))
        phim = out["phi_m"].abs().amin(dim=(-1, -2))
        kap = out["kappa"]
        fr = (out["sigma"] - prm.mu * out["C"]).abs()
        fr = torch.where(kap & out["dec"].has_t, fr, torch.full_like(fr, float("inf"))).amin(dim=(-1, -2))
        par = (out["sigma"][..., 1:] / (prm.dt * prm.v_test)).amin(dim=(-1, -2))
    return {"face": face.numpy(), "phi": phim.numpy(), "friction": fr.numpy(), "parallel": par.numpy()}


def guard_margins_gs(hand: Hand, obj: Obj, q32, r: float, prm: Params) -> dict:
    """guard_margins for the Gauss-Seidel form: the same distances, with each point's
    constraint value, friction regime and tangential direction taken at the state
    the sweep reaches it with."""
    with torch.no_grad():
        q = torch.as_tensor(np.asarray(q32, dtype=np.float64))
        out = evaluate_gs(hand, obj, q, r, prm)
        face = _face_margin(obj, out["points"]).amin(dim=(-1, -2))
        phim = out["phi_m"].abs().amin(dim=(-1, -2))
        dec = out["dec"]
        fr = (out["sigma"] - prm.mu * out["C"]).abs()
        fr = torch.where(dec.kappa & dec.has_t, fr, torch.full_like(fr, float("inf"))).amin(dim=(-1, -2))
        par = (out["sigma"][..., 1:] / (prm.dt * prm.v_test)).amin(dim=(-1, -2))
    return {"face": face.numpy(), "phi": phim.numpy(), "friction": fr.numpy(), "parallel": par.numpy()}


def clean_candidates(hand: Hand, obj: Obj, q32, r: float, prm: Params, face_tol: float = 1e-5,
                     phi_tol: float = 1e-6, fr_tol: float = 1e-6, par_tol: float = 1e-3) -> np.ndarray:
    """Candidates whose decisions all sit outside the guard band, so that a float32
    evaluation takes the same branches as this float64 one."""
    if prm.sim_steps >= 1:
        m = guard_margins_tstep(hand, obj, q32, r, prm)
    elif prm.gauss_seidel:
        m = guard_margins_gs(hand, obj, q32, r, prm)
    else:
        m = guard_margins(hand, obj, q32, r, prm)
    return ((m["face"] > face_tol) & (m["phi"] > phi_tol) & (m["friction"] > fr_tol)
            & (m["parallel"] > par_tol))


# ----------------------------------------------------------------------------- guard band per decision

def _alternative_cells(obj: Obj, sdf_dec: dict, pts: torch.Tensor, face_tol: float):
    """The other side of every cell choice within face_tol voxel of its threshold.

    Per point and axis: inside the grid near an interior node plane k the cell is
    k - 1 or k, so the other one is 2k - 1 - i0; near the clamp planes u = 0 and
    u = n - 1 the clamp decision flips (the cell stays 0 or n - 2).  Returns the
    decisions with every such choice flipped and the per-point, per-axis mask of
    flipped choices [..., 3].  Mesh objects have no alternative (None)."""
    if isinstance(obj, _mesh.MeshObj):
        return None, None
    n = torch.tensor(obj.dims, dtype=F64)
    u = (pts - obj.origin) / obj.pitch
    k = torch.round(u)
    near = (u - k).abs() <= face_tol
    near_lo = near & (k == 0)
    near_hi = near & (k == n - 1)
    near_node = near & (k >= 1) & (k <= n - 2) & ~sdf_dec["lo"] & ~sdf_dec["hi"]
    alt = {"lo": torch.where(near_lo, ~sdf_dec["lo"], sdf_dec["lo"]),
           "hi": torch.where(near_hi, ~sdf_dec["hi"], sdf_dec["hi"]),
           "i0": torch.where(near_node, 2 * k.long() - 1 - sdf_dec["i0"], sdf_dec["i0"])}
    return alt, near_lo | near_hi | near_node


def _one_candidate(dec, b: int):
    """Decisions of candidate b alone (every tensor field sliced to [b:b+1])."""
    out = type(dec)()
    for name in dec.__dataclass_fields__:
        v = getattr(dec, name)
        if isinstance(v, dict):
            v = {k: t[b:b + 1].clone() for k, t in v.items()}
        elif isinstance(v, torch.Tensor):
            v = v[b:b + 1].clone()
        setattr(out, name, v)
    return out


def _stack_decisions(decs: list):
    """One decision set holding the candidates of several (concatenated along the batch)."""
    out = type(decs[0])()
    for name in out.__dataclass_fields__:
        v = getattr(decs[0], name)
        if isinstance(v, dict):
            v = {k: torch.cat([d_.__dict__[name][k] for d_ in decs]) for k in v}
        elif isinstance(v, torch.Tensor):
            v = torch.cat([getattr(d_, name) for d_ in decs])
        setattr(out, name, v)
    return out


def decision_band(hand: Hand, obj: Obj, q32, r: float, prm: Params, face_tol: float = 1e-5,
                  phi_tol: float = 1e-6, fr_tol: float = 1e-6, par_tol: float = 1e-3,
                  max_alternatives: int = 8, chunk: int = 64) -> dict:
    """Which decisions float32 may take differently from this float64 evaluation, pair
    by pair, and the oracle's result on every branch they allow.

    The decisions are those of ``clean_candidates`` (the cell choice and clamp within
    face_tol voxel of a node or clamp plane, the contact flag within phi_tol metres of
    phi_m = 0, the friction regime within fr_tol of sigma = mu C, the friction
    direction of a contact with sigma / (dt V) < par_tol), located per (point,
    simulation) instead of per candidate, and the last only for kinetic contacts (a
    static contact's friction force is -s / w_t, smooth in s).  For the Jacobi form (Sec. III-C, read as
    averaged corrections) and the Gauss-Seidel form (point order):

    ``flag`` [B,P,M]: contact flags that are not fixed: |phi_m| <= phi_tol, or on the
        other side of an ambiguous cell choice phi_m changes sign or comes within
        phi_tol of 0.  phi_m of the Gauss-Seidel form is taken at the state the sweep
        reaches the point with.
    ``masked`` [B,P,M]: the flags a comparison leaves out.  Jacobi: ``flag`` (each
        flag depends on its own point only).  Gauss-Seidel: in each simulation every
        pair from the first ambiguous decision of the chain on (an ambiguous flag, the
        regime or direction of a contact's friction, or an ambiguous cell of a point
        in contact on either side), since the state that later points see depends on it.
    ``branches``: per candidate, the loss "L" [K], gradient "grad" [K,D] and wrench
        "W" [K,M,6] on each of the K branches its ambiguous decisions allow (index 0:
        the method's own decisions; then every combination of the alternatives).  An
        alternative sets one decision to its other side: a cell choice, a contact
        flag within phi_tol of its threshold, or a friction regime; every other
        decision is taken from the values as the method takes it (the flags and
        counts of a point looked up in its other cell, and in the Gauss-Seidel form
        the rest of the sweep from the changed state on).  Where several branches
        are correct a float32 result must match one of them.
    ``comparable`` [B]: candidates whose branches are all enumerated: at most
        max_alternatives ambiguous decisions, no contact with an ill-conditioned
        friction direction (a conditioning question, not a branch), and for mesh
        objects no decision in the face band (no alternative is enumerated for them).
    ``ref``: the float64 forward outputs at the method's own decisions."""
    if prm.sim_steps >= 1:
        raise ValueError("decision_band covers the one-step forms (Jacobi, Gauss-Seidel)")
    gs = bool(prm.gauss_seidel)
    ref = loss_and_grad(hand, obj, q32, r, prm)
    dec = ref["dec"]
    with torch.no_grad():
        p = ref["points"].detach()
        phi_m = ref["phi_m"].detach()
        kap = ref["kappa"]
        B, P = p.shape[0], p.shape[1]
        alt, near = _alternative_cells(obj, dec.sdf, p, face_tol)
        if near is None:
            face_band = (_face_margin(obj, p)[..., 0] <= face_tol)
            has_alt = torch.zeros(B, P, dtype=torch.bool)
        else:
            has_alt = near.any(-1)
            face_band = torch.zeros(B, P, dtype=torch.bool)
        tie = phi_m.abs() <= phi_tol
        flag = tie.clone()
        flip_contact = torch.zeros_like(flag)
        phi_ma = None
        if has_alt.any():
            phi_a, g_a = sdf_eval(obj, p, alt)
            gn = _safe_norm(g_a, (g_a * g_a).sum(-1) > 0)
            n_a = g_a / torch.where(gn > 0, gn, torch.ones_like(gn))[..., None]
            V = torch.tensor(TEST_DIRECTIONS, dtype=F64) * prm.v_test
            x_pred = prm.dt * V                                       # [M,3]
            if gs:
                st = dec.state                                        # [B,P,M,6]
                d = p[:, :, None, :] - x_pred[None, None]
                D = x_pred[None, None] + st[..., :3] + _cross(st[..., 3:], d)
            else:
                D = x_pred[None, None].expand(B, P, M_SIMS, 3)
            phi_ma = (phi_a - r)[..., None] - _dot(n_a[:, :, None, :], D)
            alt_pair = has_alt[..., None].expand_as(flag)
            flag = flag | (alt_pair & (((phi_ma < 0) != kap) | (phi_ma.abs() <= phi_tol)))
            flip_contact = alt_pair & (kap | (phi_ma < 0))
        flag = flag | (face_band[..., None] & (phi_m.abs() <= 2.0 * prm.dt * prm.v_test + phi_tol))
        sig = ref["sigma"].detach()
        C = ref["C"].detach()
        fr_band = kap & dec.has_t & ((sig - prm.mu * C).abs() <= fr_tol)
        # a static contact's friction is -s / w_t, smooth in s; a kinetic one's direction
        # s / sigma is ill-conditioned when sigma is small against dt V
        par_band = torch.zeros_like(flag)
        par_band[..., 1:] = (kap & ~dec.static)[..., 1:] & (sig[..., 1:] / (prm.dt * prm.v_test) <= par_tol)
        if gs:
            amb = flag | fr_band | par_band | flip_contact | (face_band[..., None] & kap)
            masked = torch.cummax(amb.to(torch.int8), dim=1).values.bool()
        else:
            masked = flag.clone()
        comparable = ~(par_band.any(-1).any(-1) | face_band.any(-1))
        L = ref["L"].detach()
        G = ref["grad"]
        W = ref["W"].detach()
        q64 = np.asarray(q32, dtype=np.float64)
        static = dec.static

    # the alternatives of each comparable candidate: (table, point, simulation)
    owner, picks = [], []
    for b in torch.nonzero(comparable).flatten().tolist():
        changes = [("sdf", i, -1) for i in torch.nonzero(has_alt[b]).flatten().tolist()]
        changes += [("kappa", i, m) for i, m in torch.nonzero(tie[b] & ~has_alt[b][:, None]).tolist()]
        changes += [("static", i, m) for i, m in torch.nonzero(fr_band[b]).tolist()]
        if len(changes) > max_alternatives:
            comparable[b] = False
            continue
        for subset in range(1, 1 << len(changes)):
            owner.append(b)
            picks.append([c_ for j, c_ in enumerate(changes) if subset >> j & 1])
    branches = [{"L": L[b:b + 1].numpy(), "grad": G[b:b + 1].numpy(), "W": W[b:b + 1].numpy()} for b in range(B)]
    for s0 in range(0, len(picks), chunk):
        own = owner[s0:s0 + chunk]
        n_ = len(own)
        idx = torch.as_tensor(own)
        cell_mask = torch.zeros(n_, P, dtype=torch.bool)
        k_mask = torch.zeros(n_, P, M_SIMS, dtype=torch.bool)
        s_mask = torch.zeros_like(k_mask)
        for j, pick in enumerate(picks[s0:s0 + chunk]):
            for table, i, m in pick:
                if table == "sdf":
                    cell_mask[j, i] = True
                elif table == "kappa":
                    k_mask[j, i, m] = True
                else:
                    s_mask[j, i, m] = True
        force = {"kappa": (k_mask, ~kap[idx]), "static": (s_mask, ~static[idx])}
        if alt is not None:
            force["sdf"] = (cell_mask, {k: v[idx] for k, v in alt.items()})
        qa = torch.as_tensor(q64[own]).clone().requires_grad_(True)
        out = evaluate_any(hand, obj, qa, r, prm, force=force)
        (ga,) = torch.autograd.grad(out["L"].sum(), qa)
        La, Wa = out["L"].detach().numpy(), out["W"].detach().numpy()
        for j, b in enumerate(own):
            br = branches[b]
            br["L"] = np.concatenate([br["L"], La[j:j + 1]])
            br["grad"] = np.concatenate([br["grad"], ga[j:j + 1].numpy()])
            br["W"] = np.concatenate([br["W"], Wa[j:j + 1]])
    return {"flag": flag.numpy(), "masked": masked.numpy(), "comparable": comparable.numpy(),
            "branches": branches,
            "ref": {"L": L.numpy(), "grad": G.numpy(), "W": W.numpy(), "N": ref["N"].numpy(),
                    "kappa": kap.numpy()}}
