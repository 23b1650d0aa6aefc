"""Synthetic watertight triangle meshes (stand-ins for the paper's object meshes).

A mesh is ``{"kind", "vertices" float32 [V,3], "faces" int32 [F,3], "mass",
"inertia", "bound_radius"}`` with faces counter-clockwise about the outward
normal, centred on the object's centre of mass (the world origin).  Mass and
inertia follow the grid objects' reading (m = 1, I = 0.4 m R_b^2).  Only
geometry is generated here; distances, normals and signs are computed by the
oracle and by the library, each on its own.
"""

from __future__ import annotations

import numpy as np


def _pack(kind, V, F, params):
    V = np.asarray(V, dtype=np.float64)
    rb = float(np.linalg.norm(V, axis=1).max())
    return {"kind": kind, "vertices": V.astype(np.float32), "faces": np.asarray(F, dtype=np.int32),
            "mass": 1.0, "inertia": float(np.float32(0.4 * rb * rb)), "bound_radius": rb, "params": params}


def _orient_outward(V, F):
    """Flip faces whose normal points towards the centre (valid for star-shaped meshes
    about the origin, which all generators here produce)."""
    F = np.asarray(F).copy()
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(B - A, C - A)
    flip = (n * (A + B + C)).sum(-1) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def box_mesh(half):
    """Axis-aligned box with half extents ``half``: 8 vertices, 12 triangles."""
    h = np.asarray(half, dtype=np.float64)
    V = np.array([[sx, sy, sz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], dtype=np.float64) * h
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    F = []
    for a, b, c, d in quads:
        F += [(a, b, c), (a, c, d)]
    return _pack("box", V, _orient_outward(V, F), {"half": h.tolist()})


def icosphere(radius: float, subdivisions: int):
    """Sphere of the given radius: a subdivided icosahedron (20 * 4^s triangles)."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    for _ in range(subdivisions):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                mid[key] = len(V) - 1
            return mid[key]
        nf = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    V = np.array(V) * radius
    return _pack("icosphere", V, _orient_outward(V, F), {"radius": radius, "subdivisions": subdivisions})


def superquadric_mesh(semi_axes, eps1: float, eps2: float, n_lat: int, n_lon: int):
    """Superquadric surface sampled on a latitude/longitude grid with two poles:
    x = a1 c(eta)^e1 c(om)^e2, y = a2 c(eta)^e1 s(om)^e2, z = a3 s(eta)^e1 with
    signed powers; (n_lat - 1) rings of n_lon vertices, 2 n_lon (n_lat - 1) faces."""
    a = np.asarray(semi_axes, dtype=np.float64)

    def spow(x, e):
        return np.sign(x) * np.abs(x) ** e
    V = [(0.0, 0.0, -a[2])]
    for i in range(1, n_lat):
        eta = -np.pi / 2 + np.pi * i / n_lat
        for j in range(n_lon):
            om = -np.pi + 2 * np.pi * j / n_lon
            V.append((a[0] * spow(np.cos(eta), eps1) * spow(np.cos(om), eps2),
                      a[1] * spow(np.cos(eta), eps1) * spow(np.sin(om), eps2),
                      a[2] * spow(np.sin(eta), eps1)))
    V.append((0.0, 0.0, a[2]))
    V = np.array(V)
    top = len(V) - 1
    ring = lambda i, j: 1 + (i - 1) * n_lon + (j % n_lon)
    F = []
    for j in range(n_lon):
        F.append((0, ring(1, j + 1), ring(1, j)))
        F.append((top, ring(n_lat - 1, j), ring(n_lat - 1, j + 1)))
    V32 = V.astype(np.float32).astype(np.float64)
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            a0, a1, b0, b1 = ring(i, j), ring(i, j + 1), ring(i + 1, j), ring(i + 1, j + 1)
            # a quad of four sampled points is rarely planar: split it along the diagonal
            # that folds outwards (the fourth vertex below the first triangle's plane, on
            # the float32 coordinates), so that the mesh of a convex surface is convex
            n = np.cross(V32[a1] - V32[a0], V32[b1] - V32[a0])
            if n @ (V32[a0] + V32[a1] + V32[b1]) < 0:
                n = -n
            if n @ (V32[b0] - V32[a0]) <= 0:
                F += [(a0, a1, b1), (a0, b1, b0)]
            else:
                F += [(a0, a1, b0), (a1, b1, b0)]
    return _pack("superquadric_mesh", V, _orient_outward(V, F),
                 {"semi_axes": a.tolist(), "eps1": eps1, "eps2": eps2, "n_lat": n_lat, "n_lon": n_lon})


def hull_mesh(points: np.ndarray):
    """Convex hull of ``points`` as an indexed mesh."""
    from scipy.spatial import ConvexHull
    P = np.asarray(points, dtype=np.float64)
    hull = ConvexHull(P)
    used = np.unique(hull.simplices)
    remap = -np.ones(len(P), dtype=np.int64)
    remap[used] = np.arange(len(used))
    V = P[used]
    F = remap[hull.simplices]
    return _pack("hull", V, _orient_outward(V, F), {"n_points": int(len(P))})



def torus_mesh(R: float, r: float, n_major: int, n_minor: int):
    """Torus about the z axis (tube centre radius R, tube radius r): a non-convex,
    genus-1 watertight mesh of 2 n_major n_minor triangles, each oriented by the
    torus's analytic outward normal at its centroid (the star-shaped orientation
    rule does not hold here)."""
    th = 2.0 * np.pi * np.arange(n_major) / n_major
    ph = 2.0 * np.pi * np.arange(n_minor) / n_minor
    T, P = np.meshgrid(th, ph, indexing="ij")
    V = np.stack([(R + r * np.cos(P)) * np.cos(T), (R + r * np.cos(P)) * np.sin(T), r * np.sin(P)], -1).reshape(-1, 3)
    idx = lambda i, j: (i % n_major) * n_minor + (j % n_minor)
    F = []
    for i in range(n_major):
        for j in range(n_minor):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            F += [(a, b, c), (a, c, d)]
    F = np.array(F)
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(B - A, C - A)
    g = (A + B + C) / 3.0
    ring = g[:, :2] * (R / np.linalg.norm(g[:, :2], axis=1))[:, None]     # nearest point of the tube's centre circle
    out = g - np.concatenate([ring, np.zeros((len(g), 1))], axis=1)
    flip = (n * out).sum(-1) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return _pack("torus", V, F, {"R": R, "r": r, "n_major": n_major, "n_minor": n_minor})

def random_superquadric_mesh(rng: np.random.Generator, n_lat: int = 24, n_lon: int = 48):
    """Superquadric mesh with exponents U(0.5, 1.5) (the grid objects use U(0.3, 2);
    sharper exponents fold the pole triangles of a latitude/longitude mesh) and
    semi-axes U(2, 8) cm."""
    eps1, eps2 = rng.uniform(0.5, 1.5, size=2)
    semi = rng.uniform(0.02, 0.08, size=3)
    return superquadric_mesh(semi, float(eps1), float(eps2), n_lat, n_lon)
