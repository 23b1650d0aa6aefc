"""Pins of the oracle's grasp-quality metrics (Sec. V "Metrics": contact area,
intersection volume, epsilon, wrench-space volume) against closed forms,
library routines and invariants (no GPU)."""

import math

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O
from oracle import quality as Q

from test_oracle_pins import multi_point_hand, obj_from


def test_tangent_basis_is_a_right_handed_orthonormal_frame():
    """Duff et al.'s basis: (t1, t2, n) orthonormal and right-handed for every unit n,
    including the poles and the equator where the branch switches."""
    rng = np.random.default_rng(1)
    n = rng.normal(size=(2000, 3))
    n = np.concatenate([n, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0.6, 0.8, 0.0]]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    t1, t2 = Q.tangent_basis(n)
    for a, b in ((t1, t2), (t1, n), (t2, n)):
        assert np.abs((a * b).sum(1)).max() < 1e-14
    assert np.abs(np.linalg.norm(t1, axis=1) - 1).max() < 1e-14
    assert np.abs(np.linalg.norm(t2, axis=1) - 1).max() < 1e-14
    assert np.abs(np.cross(t1, t2) - n).max() < 1e-14


def test_cone_edges_and_torques():
    """Every edge pushes into the object with unit normal force and tangential part mu,
    the k edges are evenly spaced around the normal, and each torque is perpendicular
    to the lever and the force with magnitude |p| |f| sin(angle) / rho."""
    rng = np.random.default_rng(2)
    p = rng.normal(size=(5, 3)) * 0.05
    n = rng.normal(size=(5, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    mu, k, rho = 0.4, 8, 0.07
    W = Q.cone_wrenches(p, n, mu, k, rho).reshape(5, k, 6)
    f, t = W[..., :3], W[..., 3:]
    assert np.abs((f * n[:, None]).sum(-1) + 1).max() < 1e-14
    tang = f + n[:, None]
    assert np.abs(np.linalg.norm(tang, axis=-1) - mu).max() < 1e-14
    cosang = (tang[:, 0] * tang[:, 1]).sum(-1) / mu ** 2
    assert np.abs(cosang - math.cos(2 * math.pi / k)).max() < 1e-12
    assert np.abs((t * p[:, None]).sum(-1)).max() < 1e-15
    assert np.abs((t * f).sum(-1)).max() < 1e-15
    pn, fn = np.linalg.norm(p, axis=-1)[:, None], np.linalg.norm(f, axis=-1)
    sin = np.sqrt(1 - ((p[:, None] * f).sum(-1) / (pn * fn)) ** 2)
    assert np.abs(np.linalg.norm(t, axis=-1) - pn * fn * sin / rho).max() < 1e-12


def test_hull_of_the_cross_polytope():
    """W = {+-e_i} in R^6: the cross-polytope, inradius 1/sqrt(6) and volume 2^6/6!; moved
    so that the origin is outside, eps turns negative."""
    W = np.concatenate([np.eye(6), -np.eye(6)])
    eps, vol, normals = Q.hull_metrics(W)
    assert abs(eps - 1 / math.sqrt(6)) < 1e-12
    assert abs(vol - 64 / 720) < 1e-12
    eps2, _, _ = Q.hull_metrics(W + 2.0 * np.eye(6)[0])
    assert eps2 < 0
    # fewer than 7 points, or a flat set: no interior, eps = Vol = 0
    assert Q.hull_metrics(W[:6])[:2] == (0.0, 0.0)
    flat = W.copy()
    flat[:, 5] = 0.0
    assert Q.hull_metrics(flat)[:2] == (0.0, 0.0)


def test_support_minimum_bounds_epsilon_and_meets_it_at_the_facet_normals():
    """eps_U >= eps for any direction set, and eps_U = eps when U holds the hull's
    facet normals (the support function along a facet normal is the facet's offset)."""
    rng = np.random.default_rng(3)
    W = rng.normal(size=(60, 6)) + 0.1
    eps, _, normals = Q.hull_metrics(W)
    assert eps > 0
    U = synth.unit_directions(2000).astype(np.float64)
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    assert Q.support_min(W, U) >= eps - 1e-12
    assert abs(Q.support_min(W, normals) - eps) < 1e-12


@pytest.fixture(scope="module")
def sphere():
    return obj_from(synth.sphere_grid(0.04, 64, 0.002, shift=(0.0, 0.0, 0.0)))


def test_contacts_follow_the_threshold(sphere):
    """Points at 1, 3 and 6 mm from a 4 cm sphere: contacts at tau = 5 mm are the first two,
    with outward normals along the radius."""
    dirs = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, -1.0]])
    pts = dirs * np.array([0.041, 0.043, 0.046])[:, None]
    hand = multi_point_hand(pts)
    p, n, phi, idx = Q.contacts(hand, sphere, np.zeros(6), 0.005)
    assert list(idx) == [0, 1]
    assert np.abs(phi - [0.001, 0.003]).max() < 5e-5          # trilinear error on a 2 mm grid
    assert np.abs(n - dirs[:2]).max() < 1e-3


def test_force_closure_grows_with_friction(sphere):
    """Four contacts at the vertices of a tetrahedron on the sphere: frictionless forces all
    pass through the centre (no torque), so there is no force closure (eps <= 0, a flat
    wrench set); with friction eps > 0 and both eps and Vol grow with mu."""
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) / math.sqrt(3)
    hand = multi_point_hand(tet * 0.0405)
    m0 = Q.grasp_metrics(hand, sphere, np.zeros(6), 0.005, 0.0, 8, 0.04)
    assert m0["n_contacts"] == 4 and m0["eps"] <= 1e-9 and m0["vol"] < 1e-12
    prev_e, prev_v = 0.0, 0.0
    for mu in (0.2, 0.5, 1.0):
        m = Q.grasp_metrics(hand, sphere, np.zeros(6), 0.005, mu, 8, 0.04)
        assert m["eps"] > prev_e and m["vol"] > prev_v
        prev_e, prev_v = m["eps"], m["vol"]


def test_contact_area_of_the_palm_on_a_plane():
    """The palm box (9 x 9 x 2.5 cm) resting 1 mm above a plane, weights on its samples only:
    below a 0.5 mm threshold nothing touches; at 1.5 mm exactly the samples on the box's
    bottom plane do (the bottom face and the side faces' samples on its edges; every other
    sample is more than 1.5 mm up), so CA is their area, at least the face's 81 cm^2; far
    from the plane the whole palm counts."""
    plane = obj_from(synth.linear_grid((0.0, 0.0, 1.0), 0.0, 48, 0.005))
    h = synth.make_hand(3, 64)
    hand = O.Hand.from_synth(h)
    q = np.zeros(hand.D)
    q[2] = 0.0125 + 0.001                                      # palm half-thickness + 1 mm
    palm = h["link_of_point"] == 0
    w = np.where(palm, h["point_area"].astype(np.float64), 0.0)
    z = h["pts_local"][:, 2].astype(np.float64)
    bottom = palm & (np.abs(z + 0.0125) < 1e-7)
    assert (z[palm & ~bottom] + 0.0125).min() > 0.0006         # the next samples up are clear of 1.5 mm
    assert Q.measure(hand, plane, q, w, 0.0005) == 0.0
    ca = Q.measure(hand, plane, q, w, 0.0015)
    assert abs(ca - w[bottom].sum()) < 1e-15
    assert ca >= 0.09 * 0.09 - 1e-12
    assert abs(Q.measure(hand, plane, q, w, 1.0) - w.sum()) < 1e-15


def test_intersection_volume_of_a_capsule_cut_by_a_plane():
    """A finger capsule (length 45 mm, radius 9 mm) whose axis lies in the plane z = 0 of a
    half-space object: by the lattice's symmetry about the axis exactly half its samples
    are inside, and the sampled volume approaches the capsule's pi r^2 L + 4/3 pi r^3."""
    plane = obj_from(synth.linear_grid((0.0, 0.0, 1.0), 0.0, 64, 0.004))
    v = synth.interior_hand(3, 0.001)
    hand = O.Hand.from_synth(v)
    link = 1                                                   # the 45 mm proximal flexion link of finger 0
    w = np.where(v["link_of_point"] == link, v["point_volume"].astype(np.float64), 0.0)
    # put the link's frame at the origin with its axis along +y in the plane: R = I, o = 0
    R_rest, o_rest = v["rest_R"][link], v["rest_o"][link]
    q = np.zeros(hand.D)
    q[:3] = -o_rest                                            # palm moves so that the link sits at the origin
    total = w.sum()
    assert abs(total - (math.pi * 0.009 ** 2 * 0.045 + 4 / 3 * math.pi * 0.009 ** 3)) < 0.03 * total
    iv = Q.measure(hand, plane, q, w, 0.0)
    assert abs(iv - 0.5 * total) < 1e-12 * total + 1e-15
    assert np.allclose(R_rest, np.eye(3))
