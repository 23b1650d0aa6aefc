"""Mesh objects on the GPU (fg_sdf_create_mesh: the mesh queried through a BVH,
Phong SDF) against the FP64 oracle (oracle/mesh_sdf.py, brute-force closest
points), through the C ABI: point queries, loss and gradient in mesh and mixed
grid + mesh scenes, optimisation steps, every fused configuration, and the
entry points that refuse mesh scenes.

Tolerances: SDF values 2e-6 m + 1e-4 of the distance and gradient directions 5e-4 (the float32 limit
of choosing between nearly coplanar neighbouring faces by distance) on points
whose closest-face choice and sign sit outside the guard band (gap to a
non-adjacent face and distance to the surface above 1 micrometre); loss 1e-4
and gradient 1e-3 relative on clean candidates, as for grids."""

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O
from oracle import mesh_sdf as MS
from synth import meshes as SM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as m
    return m


def _dev():
    return torch.device("cuda:0")


MESHES = {
    "box_flat": (SM.box_mesh((0.03, 0.02, 0.05)), 0.0),
    "icosphere": (SM.icosphere(0.04, 3), MS.PHONG_ALPHA),
    "superquadric": (SM.superquadric_mesh((0.05, 0.03, 0.04), 0.7, 1.3, 20, 40), MS.PHONG_ALPHA),
    "hull": (SM.hull_mesh(np.random.default_rng(7).normal(size=(40, 3)) * 0.04), MS.PHONG_ALPHA),
    # non-convex, genus 1: saddle-shaped inner half, concave edges and vertices
    "torus_smooth": (SM.torus_mesh(0.04, 0.015, 24, 12), MS.PHONG_ALPHA),
    "torus_coarse": (SM.torus_mesh(0.04, 0.015, 6, 3), MS.PHONG_ALPHA),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_mesh_query_matches_oracle(fg, name):
    m, alpha = MESHES[name]
    sdf = fg.Sdf.from_mesh(m["vertices"], m["faces"], m["mass"], m["inertia"], phong_alpha=alpha)
    ref_mesh = MS.MeshObj.from_synth(m, alpha=alpha)
    rng = np.random.default_rng(11)
    for n in (1, 37, 3000):
        p = rng.uniform(-0.09, 0.09, size=(n, 3))
        p32 = p.astype(np.float32)
        phi, g = fg.sdf_query(sdf, torch.tensor(p32.T.copy(), device=_dev()), 0.002)
        res = MS.mesh_query(ref_mesh, p32.astype(np.float64))
        diff = p32.astype(np.float64) - res["q_rho"]
        d = np.linalg.norm(diff, axis=1)
        rho = res["sign"] * d
        grad = res["sign"][:, None] * diff / d[:, None]
        clean = (res["gap"] > 1e-6) & (res["dist"] > 1e-6) & (d > 1e-6)
        assert clean.sum() >= 0.9 * n
        # with Phong smoothing the sideways slack of the face choice (below) moves the
        # value at first order, by up to ~1e-4 of the distance
        err = np.abs(phi.cpu().numpy().astype(np.float64) - (rho - 0.002))[clean]
        assert (err < 2e-6 + 1e-4 * d[clean]).all(), (name, n, err.max())
        assert np.median(err) < 1e-7
        # The direction (p - r*_rho)/|p - r*_rho| carries the float32 error of the closest
        # point divided by the distance.  Between two nearly coplanar faces whose
        # closest points lie close together, float32 squared distances (relative
        # rounding ~1.2e-7) cannot tell apart points up to ~sqrt(2.4e-7) d apart, so the
        # chosen point may move sideways by that much: a direction error <= 5e-4.
        gerr = np.abs(g.cpu().numpy().T.astype(np.float64) - grad).max(axis=1)[clean]
        assert (gerr < 5e-4 + 2e-8 / d[clean]).all(), (name, n, gerr.max())
        assert np.median(gerr) < 1e-5


def _cone_mesh(n=200, r=0.04, h=0.06):
    """A cone of n side faces and n base faces: its apex and base centre have valence n."""
    V = [(0.0, 0.0, 2 * h / 3), (0.0, 0.0, -h / 3)]
    V += [(r * np.cos(2 * np.pi * i / n), r * np.sin(2 * np.pi * i / n), -h / 3) for i in range(n)]
    F = []
    for i in range(n):
        a, b = 2 + i, 2 + (i + 1) % n
        F += [(0, a, b), (1, b, a)]
    return {"vertices": np.asarray(V, np.float32), "faces": np.asarray(F, np.int32), "mass": 1.0,
            "inertia": 0.4 * r * r}


def _bowtie_mesh(s=0.03):
    """Two tetrahedra that share one vertex and no edge: the shared vertex's faces form
    two fans (a vertex that is not manifold)."""
    V = np.array([(0, 0, 0), (s, 0, s), (s, s, -s), (s, -s, -s),
                  (-s, 0, s), (-s, -s, -s), (-s, s, -s)], dtype=np.float64)
    F = [(0, 1, 2), (0, 2, 3), (0, 3, 1), (1, 3, 2), (0, 4, 5), (0, 5, 6), (0, 6, 4), (4, 6, 5)]
    F = np.asarray(F)
    for t in range(len(F)):                      # orient each face away from its tetrahedron's centroid
        A, B, C = V[F[t]]
        cen = V[[1, 2, 3]].mean(0) if F[t][1] in (1, 2, 3) or F[t][0] in (1, 2, 3) else V[[4, 5, 6]].mean(0)
        if np.cross(B - A, C - A) @ ((A + B + C) / 3 - cen) < 0:
            F[t] = F[t][[0, 2, 1]]
    return {"vertices": V.astype(np.float32), "faces": F.astype(np.int32), "mass": 1.0, "inertia": 4e-4}


@pytest.mark.parametrize("name", ["cone200", "bowtie"])
def test_mesh_query_high_valence_and_non_manifold_vertices(fg, name):
    """The local search scans a vertex's whole ring (valence 200 at the cone's apex and base
    centre) and leaves a vertex whose faces form two fans (the bow-tie's shared vertex) to
    the BVH walk: values and signs match the oracle as in the query test, and so do the
    bow-tie's directions.  On the flat meshes (alpha = 0), and without the cone's
    directions: its side faces are long and thin near the apex, where float32 rounding of
    the closest point on the right face already exceeds the query tolerances (the Phong
    value by 1.5x, the direction at 37 of these 2,000 points, both computed in float32
    on the oracle's own face choice), which says nothing about the search."""
    m = _cone_mesh() if name == "cone200" else _bowtie_mesh()
    sdf = fg.Sdf.from_mesh(m["vertices"], m["faces"], m["mass"], m["inertia"], phong_alpha=0.0)
    ref_mesh = MS.MeshObj.from_synth(m, alpha=0.0)
    rng = np.random.default_rng(5)
    V = m["vertices"].astype(np.float64)
    # far points, points around the vertices of highest valence, and points near every vertex
    far = rng.normal(size=(800, 3)) * 0.08
    hub = V[[0, 1]] if name == "cone200" else V[[0]]
    near_hub = hub[rng.integers(0, len(hub), 800)] + rng.normal(size=(800, 3)) * 0.01
    near_v = V[rng.integers(0, len(V), 400)] + rng.normal(size=(400, 3)) * 0.004
    p32 = np.concatenate([far, near_hub, near_v]).astype(np.float32)
    phi, g = fg.sdf_query(sdf, torch.tensor(p32.T.copy(), device=_dev()), 0.0)
    res = MS.mesh_query(ref_mesh, p32.astype(np.float64))
    diff = p32.astype(np.float64) - res["q_rho"]
    d = np.linalg.norm(diff, axis=1)
    rho = res["sign"] * d
    grad = res["sign"][:, None] * diff / d[:, None]
    clean = (res["gap"] > 1e-6) & (res["dist"] > 1e-6) & (d > 1e-6)
    assert clean.sum() >= 0.8 * len(p32)
    got = phi.cpu().numpy().astype(np.float64)
    err = np.abs(got - rho)[clean]
    assert (err < 2e-6 + 1e-4 * d[clean]).all(), (name, err.max())
    assert np.array_equal((got < 0)[clean], (rho < 0)[clean]), name
    if name == "bowtie":
        cdir = clean & ~_direction_ambiguous(ref_mesh, p32.astype(np.float64), res)
        gerr = np.abs(g.cpu().numpy().T.astype(np.float64) - grad).max(axis=1)[cdir]
        assert (gerr < 5e-4 + 2e-8 / d[cdir]).all(), (name, gerr.max())


def _torus_points(m, rng, n=600):
    """Points that probe a torus's sign: the bounding box (the hole included), within
    0.2-3 mm of the smooth torus on both sides, and around the mesh's vertices and
    edges (where the sharp convex and concave features are)."""
    R, r = 0.04, 0.015
    V = m["vertices"].astype(np.float64)
    F = np.asarray(m["faces"])
    box = rng.uniform(-1.0, 1.0, size=(n, 3)) * np.array([R + 1.5 * r, R + 1.5 * r, 1.5 * r])
    th, ph = rng.uniform(0, 2 * np.pi, size=(2, n))
    nrm = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], -1)
    srf = np.stack([(R + r * np.cos(ph)) * np.cos(th), (R + r * np.cos(ph)) * np.sin(th), r * np.sin(ph)], -1)
    near = srf + nrm * (rng.choice([-1.0, 1.0], size=n) * rng.uniform(0.0002, 0.003, size=n))[:, None]
    at_v = V[rng.integers(0, len(V), n)] + rng.normal(size=(n, 3)) * 0.003
    e = rng.integers(0, len(F), n)
    t = rng.uniform(size=(n, 1))
    at_e = V[F[e, 0]] * t + V[F[e, 1]] * (1 - t) + rng.normal(size=(n, 3)) * 0.003
    return np.concatenate([box, near, at_v, at_e])


def _direction_ambiguous(mesh, p, res, sep=4e-4, tol_abs=5e-8, tol_rel=3e-7):
    """Points whose closest point float32 cannot pin down to the direction tolerance:
    another face (adjacent or not) has its own closest point further than sep times
    the distance from the oracle's, at a distance within float32 resolution of the
    best (tol_abs + tol_rel d).  At a concave edge two neighbouring faces can both be
    closest at interior points, which the guard band's gap (non-adjacent faces)
    does not see."""
    V, F = mesh.V, mesh.F
    q, _, _ = MS.closest_on_triangles(p, V[F[:, 0]], V[F[:, 1]], V[F[:, 2]])
    dist = np.linalg.norm(p[:, None, :] - q, axis=-1)
    best = res["dist"]
    far = np.linalg.norm(q - res["q"][:, None, :], axis=-1) > sep * best[:, None]
    near = dist - best[:, None] <= tol_abs + tol_rel * best[:, None]
    return (far & near).any(axis=1)


@pytest.mark.parametrize("n_major,n_minor", [(24, 12), (8, 4), (6, 3)])
@pytest.mark.parametrize("alpha", [0.0, MS.PHONG_ALPHA])
def test_torus_sign_and_value_match_oracle(fg, n_major, n_minor, alpha):
    """Non-convex meshes on the GPU (Sec. III-B: inside or outside by the closest
    feature, then the Phong point): tori whose inner half is saddle-shaped; the coarse
    ones (tubes of 3 or 4 faces) have sharp concave edges and vertices, where the sign
    needs the edge or vertex pseudonormal.  Against the oracle's brute-force query
    (whose sign is pinned on these tori by the winding number): the sign exactly, the
    value and gradient within the query tolerances, on points outside the guard band
    (the gradient also away from concave-edge ties, _direction_ambiguous)."""
    m = SM.torus_mesh(0.04, 0.015, n_major, n_minor)
    sdf = fg.Sdf.from_mesh(m["vertices"], m["faces"], m["mass"], m["inertia"], phong_alpha=alpha)
    ref_mesh = MS.MeshObj.from_synth(m, alpha=alpha)
    p32 = _torus_points(m, np.random.default_rng(n_major)).astype(np.float32)
    phi, g = fg.sdf_query(sdf, torch.tensor(p32.T.copy(), device=_dev()), 0.0)
    res = MS.mesh_query(ref_mesh, p32.astype(np.float64))
    diff = p32.astype(np.float64) - res["q_rho"]
    d = np.linalg.norm(diff, axis=1)
    clean = (res["gap"] > 1e-6) & (res["dist"] > 1e-6) & (d > 1e-6)
    assert clean.sum() >= 0.9 * len(p32)
    got = phi.cpu().numpy().astype(np.float64)
    inside = res["sign"] < 0
    assert inside[clean].sum() > 300 and (~inside[clean]).sum() > 300
    assert np.array_equal((got < 0)[clean], inside[clean])
    err = np.abs(got - res["sign"] * d)[clean]
    assert (err < 2e-6 + 1e-4 * d[clean]).all(), err.max()
    grad = res["sign"][:, None] * diff / d[:, None]
    # the direction where float32 can pick a closest point elsewhere is left out
    cdir = clean & ~_direction_ambiguous(ref_mesh, p32.astype(np.float64), res)
    assert cdir.sum() >= 0.9 * clean.sum()
    gerr = np.abs(g.cpu().numpy().T.astype(np.float64) - grad).max(axis=1)[cdir]
    assert (gerr < 5e-4 + 2e-8 / d[cdir]).all(), gerr.max()


@pytest.mark.parametrize("n_major,n_minor", [(24, 12), (6, 3)])
def test_torus_loss_and_grad_match_oracle(fg, n_major, n_minor):
    """The 3-finger hand's candidates around a torus (tube radius 1.5 cm, ring 4 cm):
    loss and leaky gradient of the fused kernel (BVH walk, pseudonormal sign, Phong
    SDF, contacts) against the oracle on clean candidates."""
    w = synth.tiny_sphere_workload(n_cand=48)
    c = Case(fg, w.hand, [SM.torus_mesh(0.04, 0.015, n_major, n_minor)], w.obj_of_cand, w.q0, w.params)
    loss, grad = fg.loss_and_grad(c.hand, c.scene, torch.tensor(w.q0, device=_dev()), w.params, 0.004,
                                  obj_of_cand=c.oc)
    ref = O.batch_loss_and_grad(c.S, w.q0, w.obj_of_cand, 0.004)
    clean = c.clean(w.q0, 0.004)
    assert clean.sum() >= 0.6 * len(clean)
    assert (ref["N"].sum(axis=1) > 0).sum() >= 5, "workload must exercise contacts"
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)
    q1 = torch.tensor(w.q0, device=_dev())
    l1 = fg.optimize_step(c.hand, c.scene, q1, w.params, 0, w.steps, 1, obj_of_cand=c.oc)
    step = (q1 - torch.tensor(w.q0, device=_dev())).cpu().numpy().astype(np.float64) / -w.params["lr"]
    _compare(l1.cpu().numpy(), step, ref, clean)


class Case:
    def __init__(self, fg, hand, objects, obj_of_cand, q0, params):
        self.hand_d, self.objects, self.oc_np, self.q0, self.params = hand, objects, obj_of_cand, q0, params
        self.S = O.Setup(hand, objects, params)
        self.hand = fg.Hand.from_synth(hand)
        self.sdfs = [fg.Sdf.from_synth(o) for o in objects]
        self.scene = fg.Scene(self.sdfs)
        self.oc = torch.tensor(obj_of_cand, device=_dev(), dtype=torch.int32)

    def clean(self, q, r):
        mask = np.zeros(len(q), dtype=bool)
        for k in np.unique(self.oc_np):
            idx = np.nonzero(self.oc_np == k)[0]
            mask[idx] = O.clean_candidates(self.S.hand, self.S.objs[int(k)], q[idx], r, self.S.prm)
        return mask


def _compare(loss, grad, ref, clean):
    idx = np.nonzero(clean)[0]
    L = loss.astype(np.float64)[idx]
    lrel = np.abs(L - ref["L"][idx]) / np.maximum(np.abs(ref["L"][idx]), 1e-6)
    G = grad.astype(np.float64)[idx]
    grel = np.linalg.norm(G - ref["grad"][idx], axis=1) / np.maximum(np.linalg.norm(ref["grad"][idx], axis=1), 1e-6)
    assert lrel.max() < 1e-4, (idx[np.argmax(lrel)], lrel.max())
    assert grel.max() < 1e-3, (idx[np.argmax(grel)], grel.max())


@pytest.fixture(scope="module")
def sphere_case(fg):
    w = synth.tiny_sphere_workload(n_cand=48)
    return Case(fg, w.hand, [SM.icosphere(0.04, 3)], w.obj_of_cand, w.q0, w.params)


@pytest.mark.parametrize("alpha", [0.1, 0.0])
def test_mesh_loss_and_grad_match_oracle(fg, sphere_case, alpha):
    c = sphere_case
    params = dict(c.params, alpha_leak=alpha)
    S = O.Setup(c.hand_d, c.objects, params)
    loss, grad = fg.loss_and_grad(c.hand, c.scene, torch.tensor(c.q0, device=_dev()), params, 0.004,
                                  obj_of_cand=c.oc)
    ref = O.batch_loss_and_grad(S, c.q0, c.oc_np, 0.004)
    clean = c.clean(c.q0, 0.004)
    assert clean.sum() >= 0.6 * len(clean)
    assert (ref["N"].sum(axis=1) > 0).sum() >= 5, "workload must exercise contacts"
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_mixed_grid_and_mesh_scene_four_finger(fg):
    """Superquadric grids and superquadric meshes in one batch, 4-finger hand."""
    w = synth.batched_superquadric_workload(n_obj=2, per_obj=10, grid_n=48, points_per_link=32, steps=50,
                                            device="cuda")
    rng = np.random.default_rng(5)
    objects = list(w.objects) + [SM.random_superquadric_mesh(rng, 16, 32), SM.random_superquadric_mesh(rng, 16, 32)]
    oc = np.concatenate([w.obj_of_cand, w.obj_of_cand + 2])
    q0 = np.concatenate([w.q0, w.q0])
    c = Case(fg, w.hand, objects, oc, q0, w.params)
    r = O.dilation_radius(c.S.prm, 5, w.steps)
    loss, grad = fg.loss_and_grad(c.hand, c.scene, torch.tensor(q0, device=_dev()), w.params, r, obj_of_cand=c.oc)
    ref = O.batch_loss_and_grad(c.S, q0, oc, r)
    clean = c.clean(q0, r)
    assert clean.sum() >= 0.5 * len(clean)
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_mesh_optimize_step_every_configuration(fg, sphere_case):
    c = sphere_case
    K = 20
    r = O.dilation_radius(c.S.prm, 0, K)
    ref = O.batch_loss_and_grad(c.S, c.q0, c.oc_np, r)
    clean = c.clean(c.q0, r)
    q0 = torch.tensor(c.q0, device=_dev())
    try:
        for i in range(len(fg.fused_configs())):
            fg.fused_config_select(i)
            q1 = q0.clone()
            loss = fg.optimize_step(c.hand, c.scene, q1, c.params, 0, K, 1, obj_of_cand=c.oc)
            step = (q1 - q0).cpu().numpy().astype(np.float64) / -c.params["lr"]
            _compare(loss.cpu().numpy(), step, ref, clean)
    finally:
        fg.fused_config_select(-1)
    # contact wrench on a mesh scene runs (counts match the oracle's flags on clean candidates)
    W, N, _ = fg.contact_wrench(c.hand, c.scene, q0, c.params, r, obj_of_cand=c.oc)
    Nn = N.cpu().numpy()
    for b in np.nonzero(clean)[0]:
        assert np.array_equal(Nn[b], ref["N"][b].astype(np.int32)), b


def test_mesh_scenes_refused_where_unsupported(fg, sphere_case):
    from paper_2306_08132_gb300 import _lib
    c = sphere_case
    q = torch.tensor(c.q0[:4], device=_dev())
    with pytest.raises(_lib.FgError):
        fg.optimize_step_plain(c.hand, c.scene, q.clone(), c.params, 0, 10, 1)


@pytest.mark.parametrize("T", [1, 2])
def test_mesh_tstep_matches_oracle(fg, T):
    """The T-step metric on a mesh object (an icosphere of 320 faces): every point
    re-queried (BVH, Phong SDF) at each simulation's predicted pose for T steps, against
    the oracle's evaluate_tstep."""
    w = synth.tiny_sphere_workload(n_cand=12)
    c = Case(fg, w.hand, [SM.icosphere(0.04, 2)], w.obj_of_cand, w.q0, w.params)
    params = dict(w.params, sim_steps=T)
    S = O.Setup(w.hand, c.objects, params)
    loss, grad = fg.loss_and_grad(c.hand, c.scene, torch.tensor(w.q0, device=_dev()), params, 0.004,
                                  obj_of_cand=c.oc)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, 0.004)
    clean = O.clean_candidates(S.hand, S.objs[0], w.q0, 0.004, S.prm)
    assert clean.sum() >= 8
    assert (ref["N"].sum(axis=1) > 0).sum() >= 3
    _compare(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_mesh_full_size_sampled_parity(fg):
    """The benchmark's mesh workload at full size (the 8 superquadrics as meshes of 2,208
    faces, 4-finger hand with 4,352 points, 8,192 candidates) in the launch the benchmark
    times: loss and update of 3 sampled candidates against the oracle."""
    w = synth.batched_superquadric_workload(device="cuda")
    meshes = []
    for o in w.objects:
        pr = o["params"]
        meshes.append(SM.superquadric_mesh(pr["semi_axes"], float(np.clip(pr["eps1"], 0.5, 1.5)),
                                           float(np.clip(pr["eps2"], 0.5, 1.5)), 24, 48))
    c = Case(fg, w.hand, meshes, w.obj_of_cand, w.q0, w.params)
    q = torch.tensor(w.q0, device=_dev())
    q1 = q.clone()
    loss = fg.optimize_step(c.hand, c.scene, q1, w.params, 0, w.steps, 1, obj_of_cand=c.oc)
    torch.cuda.synchronize()
    assert torch.isfinite(loss).all() and torch.isfinite(q1).all()
    r = O.dilation_radius(c.S.prm, 0, w.steps)
    sample = np.sort(np.random.default_rng(14).choice(w.B, size=8, replace=False))
    ref = O.batch_loss_and_grad(c.S, w.q0[sample], w.obj_of_cand[sample], r)
    clean = np.array([O.clean_candidates(c.S.hand, c.S.objs[int(w.obj_of_cand[b])], w.q0[b:b + 1], r, c.S.prm)[0]
                      for b in sample])
    assert clean.sum() >= 2
    step = ((q1 - q).cpu().numpy()[sample]).astype(np.float64) / -w.params["lr"]
    _compare(loss.cpu().numpy()[sample], step, ref, clean)
