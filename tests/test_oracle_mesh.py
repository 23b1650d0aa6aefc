"""Pins of the oracle's mesh SDF and Phong SDF (oracle/mesh_sdf.py):
closest points on one triangle in each Voronoi region by hand, against dense
sampling of the triangle, the flat mesh SDF of a box against the box's closed
form (inside and outside), the sign, the Phong point at vertices and across a
shared edge, and the Phong surface of an icosphere against the sphere."""

import numpy as np
import pytest
import torch

from oracle import mesh_sdf as MS
from synth import meshes as SM


def test_closest_point_regions_by_hand():
    a, b, c = np.array([[0.0, 0, 0]]), np.array([[1.0, 0, 0]]), np.array([[0.0, 1, 0]])
    cases = [((0.2, 0.2, 1.0), (0.2, 0.2, 0.0), MS.FACE), ((-1.0, -1.0, 0.5), (0, 0, 0), MS.VERT_A),
             ((2.0, -0.5, 0.0), (1, 0, 0), MS.VERT_B), ((-0.5, 2.0, 0.3), (0, 1, 0), MS.VERT_C),
             ((0.5, -1.0, 0.2), (0.5, 0, 0), MS.EDGE_AB), ((1.0, 1.0, -0.4), (0.5, 0.5, 0), MS.EDGE_BC),
             ((-1.0, 0.5, 0.0), (0, 0.5, 0), MS.EDGE_CA)]
    p = np.array([x for x, _, _ in cases])
    q, bary, region = MS.closest_on_triangles(p, a, b, c)
    for k, (_, qe, code) in enumerate(cases):
        assert np.allclose(q[k, 0], qe, atol=1e-15), (k, q[k, 0])
        assert region[k, 0] == code
        assert np.allclose(bary[k, 0] @ np.vstack([a, b, c]), q[k, 0], atol=1e-15)
        assert abs(bary[k, 0].sum() - 1.0) < 1e-15 and (bary[k, 0] >= -1e-15).all()


def test_closest_point_against_dense_sampling():
    rng = np.random.default_rng(1)
    tri = rng.normal(size=(3, 3))
    n = 400
    s, t = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    keep = s + t <= 1
    samples = tri[0] + s[keep, None] * (tri[1] - tri[0]) + t[keep, None] * (tri[2] - tri[0])
    p = rng.normal(size=(64, 3)) * 2.0
    q, _, _ = MS.closest_on_triangles(p, tri[0:1], tri[1:2], tri[2:3])
    d = np.linalg.norm(p - q[:, 0], axis=1)
    dense = np.linalg.norm(p[:, None] - samples[None], axis=-1).min(axis=1)
    spacing = np.linalg.norm(tri[1] - tri[0]) / n + np.linalg.norm(tri[2] - tri[0]) / n
    assert (d <= dense + 1e-12).all()                 # never farther than a sample
    assert (dense - d <= spacing).all()               # and within the sampling resolution


def _box_sdf(p, h):
    q = np.abs(p) - h
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=1)
    inside = np.minimum(q.max(axis=1), 0.0)
    return outside + inside


def test_flat_box_mesh_is_the_exact_box_sdf():
    h = np.array([0.03, 0.02, 0.05])
    mesh = MS.MeshObj.from_synth(SM.box_mesh(h), alpha=0.0)
    rng = np.random.default_rng(2)
    p = rng.uniform(-0.08, 0.08, size=(4000, 3))
    res = MS.mesh_query(mesh, p)
    rho = res["sign"] * np.linalg.norm(p - res["q_rho"], axis=1)
    h32 = h.astype(np.float32).astype(np.float64)          # the mesh stores float32 vertices
    assert np.abs(rho - _box_sdf(p, h32)).max() < 1e-15
    inside = (np.abs(p) < h32).all(axis=1)
    assert inside.sum() > 100 and (res["sign"][inside] < 0).all() and (res["sign"][~inside] > 0).all()


def test_phong_point_at_vertices_and_across_shared_edges():
    mesh = MS.MeshObj.from_synth(SM.icosphere(0.04, 1))
    # at a vertex the Phong point is the vertex (psi_x(v_x) = v_x)
    f = np.arange(len(mesh.F))
    for k in range(3):
        bary = np.zeros((len(f), 3))
        bary[:, k] = 1.0
        q = mesh.V[mesh.F[f, k]]
        assert np.abs(MS.phong_point(mesh, f, bary, q) - q).max() < 1e-15
    # a point of a shared edge gives the same Phong point from either face
    owner = {}
    for fi, (a, b, c) in enumerate(mesh.F):
        for e, (u, v) in enumerate(((a, b), (b, c), (c, a))):
            owner[(int(u), int(v))] = (fi, e)
    rng = np.random.default_rng(3)
    for _ in range(50):
        fi = int(rng.integers(len(mesh.F)))
        e = int(rng.integers(3))
        u, v = int(mesh.F[fi, e]), int(mesh.F[fi, (e + 1) % 3])
        g, _ = owner[(v, u)]
        t = rng.uniform(0.05, 0.95)
        q = ((1 - t) * mesh.V[u] + t * mesh.V[v])[None]

        def bary_in(face):
            bb = np.zeros((1, 3))
            idx = list(mesh.F[face])
            bb[0, idx.index(u)] = 1 - t
            bb[0, idx.index(v)] = t
            return bb
        pa = MS.phong_point(mesh, np.array([fi]), bary_in(fi), q)
        pb = MS.phong_point(mesh, np.array([g]), bary_in(g), q)
        assert np.abs(pa - pb).max() < 1e-15


def test_phong_surface_of_an_icosphere_approximates_the_sphere_better():
    R = 0.04
    flat = MS.MeshObj.from_synth(SM.icosphere(R, 1), alpha=0.0)
    phong = MS.MeshObj.from_synth(SM.icosphere(R, 1))
    # vertex normals of a sphere mesh are radial
    assert np.abs(np.abs((phong.vert_n * phong.V / R).sum(1)) - 1.0).max() < 2e-3
    rng = np.random.default_rng(4)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = d * rng.uniform(R + 0.004, R + 0.02, size=(2000, 1))     # outside, near the surface
    true = np.linalg.norm(p, axis=1) - R
    err = []
    for mesh in (flat, phong):
        res = MS.mesh_query(mesh, p)
        rho = res["sign"] * np.linalg.norm(p - res["q_rho"], axis=1)
        err.append(np.abs(rho - true).mean())
    assert err[1] < 0.5 * err[0], err


def test_mesh_eval_gradient_is_the_papers_formula():
    mesh = MS.MeshObj.from_synth(SM.icosphere(0.04, 2))
    rng = np.random.default_rng(5)
    p = torch.tensor(rng.uniform(-0.07, 0.07, size=(300, 3)), requires_grad=True)
    dec = MS.mesh_decisions(mesh, p)
    rho, grad = MS.mesh_eval(mesh, p, dec)
    (g,) = torch.autograd.grad(rho.sum(), p)
    assert torch.allclose(g, grad, atol=1e-12)
    assert torch.allclose(grad.norm(dim=-1), torch.ones(300, dtype=torch.float64), atol=1e-12)
    inside = p.detach().norm(dim=-1) < 0.035
    assert (rho.detach()[inside] < 0).all()


def test_mesh_object_in_the_grasp_metric():
    """A mesh object in the one-step metric: the gradient is the exact gradient of
    the branch-frozen loss (Phong points held fixed, the paper's gradient), and an
    icosphere behaves like the sphere grid of the same radius."""
    import synth
    from oracle import fastgraspd_oracle as O
    w = synth.tiny_sphere_workload(n_cand=8)
    S = O.Setup(w.hand, [SM.icosphere(0.04, 3)], w.params)
    q = w.q0.astype(np.float64)
    out = O.loss_and_grad(S.hand, S.objs[0], q, 0.004, S.prm)
    assert int(out["N"].sum()) > 0
    g = out["grad"].numpy()
    h = 1e-8
    fd = np.zeros_like(g)
    for k in range(S.hand.D):
        e = np.zeros(S.hand.D)
        e[k] = h
        lp = O.evaluate(S.hand, S.objs[0], torch.tensor(q + e), 0.004, S.prm, dec=out["dec"], anchor_mode=True)["L"]
        lm = O.evaluate(S.hand, S.objs[0], torch.tensor(q - e), 0.004, S.prm, dec=out["dec"], anchor_mode=True)["L"]
        fd[:, k] = ((lp - lm) / (2 * h)).detach().numpy()
    rel = np.linalg.norm(fd - g, axis=1) / np.maximum(np.linalg.norm(g, axis=1), 1e-12)
    assert rel.max() < 1e-6, rel
    grid = O.Setup(w.hand, w.objects, w.params)
    ref = O.evaluate(grid.hand, grid.objs[0], torch.tensor(q), 0.004, grid.prm)
    free = (ref["N"].sum(1) == 0).numpy()
    assert np.allclose(out["L"].detach().numpy()[free], ref["L"].numpy()[free], rtol=1e-3)


def _winding_number(V, F, p):
    """Generalised winding number of a closed triangle mesh at points p: the solid
    angles of its faces seen from p (Van Oosterom and Strackee, 1983) summed over the
    faces and divided by 4 pi; 1 inside a watertight outward-oriented mesh, 0 outside."""
    w = np.zeros(len(p))
    for f in F:
        a, b, c = V[f[0]] - p, V[f[1]] - p, V[f[2]] - p
        la, lb, lc = (np.linalg.norm(x, axis=1) for x in (a, b, c))
        num = (a * np.cross(b, c)).sum(-1)
        den = la * lb * lc + (a * b).sum(-1) * lc + (b * c).sum(-1) * la + (c * a).sum(-1) * lb
        w += 2.0 * np.arctan2(num, den)
    return w / (4.0 * np.pi)


@pytest.mark.parametrize("n_major,n_minor", [(24, 12), (8, 4), (6, 3)])
def test_sign_on_a_non_convex_mesh_matches_the_winding_number(n_major, n_minor):
    """The pseudonormal sign (the closest face, edge or vertex decides) on tori, whose
    inner half is saddle-shaped, against an independent inside test: the generalised
    winding number.  Points fill the bounding box (the hole included), lie within
    0.2-3 mm of the smooth torus on both sides, and cluster around the vertices and
    edges of the mesh.  The coarse tori (tubes of 3 or 4 faces, 60-90 degree bends
    along the ring) have sharp convex and concave features, where a sign taken from
    the closest face's normal alone, or from its vertices' normals, is wrong."""
    R, r = 0.04, 0.015
    m = SM.torus_mesh(R, r, n_major, n_minor)
    mesh = MS.MeshObj.from_synth(m, alpha=0.0)
    V = m["vertices"].astype(np.float64)
    F = mesh.F
    rng = np.random.default_rng(6)
    box = rng.uniform(-1.0, 1.0, size=(1500, 3)) * np.array([R + 1.5 * r, R + 1.5 * r, 1.5 * r])
    th, ph = rng.uniform(0, 2 * np.pi, size=(2, 1500))
    n = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], -1)
    s = np.stack([(R + r * np.cos(ph)) * np.cos(th), (R + r * np.cos(ph)) * np.sin(th), r * np.sin(ph)], -1)
    near = s + n * (rng.choice([-1.0, 1.0], size=1500) * rng.uniform(0.0002, 0.003, size=1500))[:, None]
    at_vertices = V[rng.integers(0, len(V), 1500)] + rng.normal(size=(1500, 3)) * 0.003
    e = rng.integers(0, len(F), 1500)
    t = rng.uniform(size=(1500, 1))
    at_edges = V[F[e, 0]] * t + V[F[e, 1]] * (1 - t) + rng.normal(size=(1500, 3)) * 0.003
    p = np.concatenate([box, near, at_vertices, at_edges])
    res = MS.mesh_query(mesh, p)
    w = _winding_number(V, F, p)
    assert np.abs(w - np.round(w)).max() < 1e-9            # closed and consistently oriented
    keep = res["dist"] > 1e-7
    inside = np.round(w[keep]) == 1
    assert inside.sum() > 500 and (~inside).sum() > 500
    assert np.array_equal(res["sign"][keep] < 0, inside)
    # the hole: points on the axis are outside
    axis = np.stack([np.zeros(20), np.zeros(20), np.linspace(-r, r, 20)], -1)
    assert (MS.mesh_query(mesh, axis)["sign"] > 0).all()


@pytest.mark.parametrize("eps", [(0.5, 0.5), (1.0, 1.0), (0.7, 1.3), (1.5, 1.5)])
def test_superquadric_meshes_of_convex_surfaces_are_convex(eps):
    """The generator splits each latitude/longitude quad along its outward-folding
    diagonal, so the mesh of a convex superquadric (exponents <= 2) is convex on its
    float32 coordinates: no vertex lies outside any face's plane beyond double
    rounding.  The library's certified local search relies on faces on the hull."""
    m = SM.superquadric_mesh((0.05, 0.03, 0.04), eps[0], eps[1], 24, 48)
    V = m["vertices"].astype(np.float64)
    F = np.asarray(m["faces"])
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    n /= np.linalg.norm(n, axis=1)[:, None]
    gap = (V @ n.T - (n * V[F[:, 0]]).sum(1)[None, :]).max(axis=0)
    assert gap.max() <= 1e-12 * np.abs(V).max(), gap.max()
    # the quads are not planar, so the diagonal matters: the first quad's fourth
    # vertex lies off the plane of its other three
    n_lon = 48
    a0, a1, b0, b1 = 1, 2, 1 + n_lon, 2 + n_lon
    t = np.cross(V[a1] - V[a0], V[b1] - V[a0])
    assert t @ (V[b0] - V[a0]) != 0
