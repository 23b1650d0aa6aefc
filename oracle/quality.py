"""FP64 oracle of the grasp-quality metrics of Sec. V ("Metrics").

TEST INFRASTRUCTURE ONLY, like ``fastgraspd_oracle``: only ``tests/``, the smoke
check and the benchmark's CPU legs may use it.

The paper names the metrics and says that contact area, epsilon and the wrench-
space volume depend on the distance threshold used to generate contacts (5 mm in
its Table II); it prints no formulas.  The definitions written out here are the
standard ones of the grasp-analysis works it compares with:

  contacts   hand surface points p_i with phi(p_i) < tau (undilated SDF of the
             object at its canonical pose), outward unit normal n = grad phi/|grad phi|
  CA         contact area: sum over contacts of the area a_i each surface sample
             stands for
  IV         intersection volume: sum of the volumes v_j of hand interior samples
             with phi < 0
  cone       at each contact, k unit-normal-force edges of the Coulomb cone
             f_e = -n + mu (cos(2 pi e / k) t1 + sin(2 pi e / k) t2), with (t1, t2) the
             tangent basis of n by the branch-free construction of Duff et al.
             ("Building an orthonormal basis, revisited", 2017)
  wrench     w = (f, (p - c) x f / rho): c the object's centre of mass (the origin
             of its frame), rho the torque scale (the object's bounding radius)
  GWS        the convex hull of all wrenches (the L1 grasp wrench space)
  eps        signed distance from the origin to the GWS boundary, the minimum over
             the hull's facets of -offset (negative: the origin is outside, no
             force closure; 0 for fewer than 7 affinely independent wrenches)
  Vol        the 6-D volume of the GWS
  eps_U      for a set of unit directions u_k: min_k h(u_k) with the support
             function h(u) = max over wrenches of u . w.  eps_U >= eps, with
             equality when the set holds the normal of the facet nearest the origin.

The hull is qhull (scipy.spatial.ConvexHull), a library routine used as one step.
"""

from __future__ import annotations

import math

import numpy as np
import torch

from . import fastgraspd_oracle as O

F64 = torch.float64


def contacts(hand: O.Hand, obj, q: np.ndarray, tau: float):
    """Contact points of candidate q [D] at threshold tau: (p [n,3], normal [n,3], phi [n], index [n])."""
    qt = torch.as_tensor(np.asarray(q, dtype=np.float64))[None]
    R, o = O.forward_kinematics(hand, qt)
    p = O.hand_points(hand, R, o)[0]
    phi, g = O.sdf_query(obj, p, 0.0)
    sel = phi < tau
    gn = g[sel].norm(dim=-1, keepdim=True)
    n = g[sel] / torch.where(gn > 0, gn, torch.ones_like(gn))
    idx = torch.nonzero(sel)[:, 0]
    return p[sel].numpy(), n.numpy(), phi[sel].numpy(), idx.numpy()


def tangent_basis(n: np.ndarray):
    """Duff et al. (2017): for unit n, s = sign(n_z) (+1 at 0), a = -1/(s + n_z),
    b = n_x n_y a, t1 = (1 + s n_x^2 a, s b, -s n_x), t2 = (b, s + n_y^2 a, -n_y)."""
    n = np.atleast_2d(n)
    s = np.where(n[:, 2] >= 0.0, 1.0, -1.0)
    a = -1.0 / (s + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    t1 = np.stack([1.0 + s * n[:, 0] ** 2 * a, s * b, -s * n[:, 0]], -1)
    t2 = np.stack([b, s + n[:, 1] ** 2 * a, -n[:, 1]], -1)
    return t1, t2


def cone_wrenches(p: np.ndarray, n: np.ndarray, mu: float, k: int, rho: float) -> np.ndarray:
    """All k cone-edge wrenches of every contact: [n_contacts * k, 6], contact-major."""
    t1, t2 = tangent_basis(n)
    out = []
    for e in range(k):
        ang = 2.0 * math.pi * e / k
        f = -n + mu * (math.cos(ang) * t1 + math.sin(ang) * t2)
        out.append(np.concatenate([f, np.cross(p, f) / rho], -1))
    return np.stack(out, 1).reshape(-1, 6)


def support_min(W: np.ndarray, U: np.ndarray) -> float:
    """eps_U = min over directions u of max over wrenches of u . w (-inf without wrenches)."""
    if len(W) == 0:
        return -math.inf
    return float((U @ W.T).max(axis=1).min())


def hull_metrics(W: np.ndarray):
    """(eps, Vol, facet normals) of the convex hull of the wrenches W [m, 6]."""
    from scipy.spatial import ConvexHull
    from scipy.spatial import QhullError
    if len(W) < 7:
        return 0.0, 0.0, np.zeros((0, 6))
    try:
        h = ConvexHull(W)
    except QhullError:                 # lower-dimensional set
        return 0.0, 0.0, np.zeros((0, 6))
    off = -h.equations[:, -1]          # facet planes n . x + d = 0, n unit, inside n . x + d <= 0
    return float(off.min()), float(h.volume), h.equations[:, :-1]


def measure(hand: O.Hand, obj, q: np.ndarray, weights: np.ndarray, tau: float) -> float:
    """sum of weights[i] over the points of candidate q with phi < tau (CA with area weights and
    tau the contact threshold; IV with interior samples, volume weights and tau = 0)."""
    qt = torch.as_tensor(np.asarray(q, dtype=np.float64))[None]
    R, o = O.forward_kinematics(hand, qt)
    p = O.hand_points(hand, R, o)[0]
    phi, _ = O.sdf_query(obj, p, 0.0)
    return float(np.asarray(weights, dtype=np.float64)[(phi < tau).numpy()].sum())


def grasp_metrics(hand: O.Hand, obj, q: np.ndarray, tau: float, mu: float, k: int, rho: float,
                  U: np.ndarray | None = None) -> dict:
    """Contacts, eps, Vol (and eps_U for directions U) of candidate q."""
    p, n, phi, idx = contacts(hand, obj, q, tau)
    W = cone_wrenches(p, n, mu, k, rho)
    eps, vol, normals = hull_metrics(W)
    out = {"n_contacts": len(p), "eps": eps, "vol": vol, "W": W, "facet_normals": normals, "index": idx,
           "p": p, "n": n, "phi": phi}
    if U is not None:
        out["eps_U"] = support_min(W, U)
    return out


def guard_ok(hand: O.Hand, obj, q: np.ndarray, tau: float, phi_tol: float = 1e-6, nz_tol: float = 1e-5,
             face_tol: float = 1e-5) -> bool:
    """The float32 evaluation takes the same decisions: no point within phi_tol of the
    threshold, no contact normal with |n_z| < nz_tol (the tangent basis switches sign),
    no point within face_tol voxels of a cell face."""
    qt = torch.as_tensor(np.asarray(q, dtype=np.float64))[None]
    R, o = O.forward_kinematics(hand, qt)
    p = O.hand_points(hand, R, o)[0]
    phi, g = O.sdf_query(obj, p, 0.0)
    if (phi - tau).abs().min() <= phi_tol:
        return False
    sel = phi < tau
    if sel.any():
        n = g[sel] / g[sel].norm(dim=-1, keepdim=True)
        if n[:, 2].abs().min() <= nz_tol:
            return False
    return bool(O._face_margin(obj, p[None]).min() > face_tol)
