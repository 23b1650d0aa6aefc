"""Synthetic objects sampled onto voxel SDF grids (stand-ins for YCB/EGAD meshes).

Grids are float32 arrays indexed ``grid[z, y, x]`` (x fastest).  Node (i, j, k)
sits at ``origin + pitch * (i, j, k)`` for (x, y, z); grids are centred on the
object, whose centre of mass is the world origin.  Each object also carries the
rigid-body data the contact model needs: mass m = 1 and an isotropic inertia
I = (2/5) m R_b^2 with R_b the object's bounding radius (the paper gives no mass
model; this is the reading used throughout).

Signed distances are negative inside.  Builders run on any torch device so that
large grids can be made on the GPU; the arithmetic is float64 and the result is
rounded to float32 once.
"""

from __future__ import annotations

import math
import numpy as np
import torch

F64 = torch.float64


DEFAULT_SHIFT = (0.31, -0.17, 0.23)


def _centred_nodes(n: int, pitch: float, shift, device):
    """Node coordinates per axis: centred on the object, then moved by ``shift``
    voxels (|shift| < 1/2) so that no grid is mirror-symmetric about the object
    centre (a voxel-aligned symmetric grid has exactly zero interpolated slopes
    along its central cells, which real scans never have)."""
    origin = -0.5 * (n - 1) * pitch + pitch * np.asarray(shift, dtype=np.float64)
    axes = [origin[k] + pitch * torch.arange(n, dtype=F64, device=device) for k in range(3)]
    return origin, axes


def _pack(kind, grid64, origin, pitch, bound_radius, params):
    mass = 1.0
    return {
        "kind": kind,
        "grid": grid64.to(torch.float32).contiguous(),
        "origin": np.asarray(origin, dtype=np.float32),
        "pitch": float(np.float32(pitch)),
        "mass": mass,
        "inertia": float(np.float32(0.4 * mass * bound_radius * bound_radius)),
        "bound_radius": float(bound_radius),
        "params": params,
    }


def _field(n, pitch, fn, device, chunk=1 << 22, shift=DEFAULT_SHIFT):
    """Evaluate fn(xyz[M,3]) -> [M] over all nodes of an n^3 grid, in chunks."""
    origin, ax = _centred_nodes(n, pitch, shift, device)
    out = torch.empty(n * n * n, dtype=F64, device=device)
    total = n * n * n
    for s in range(0, total, chunk):
        idx = torch.arange(s, min(s + chunk, total), device=device)
        x = ax[0][idx % n]
        y = ax[1][(idx // n) % n]
        z = ax[2][idx // (n * n)]
        out[s:s + len(idx)] = fn(torch.stack([x, y, z], dim=-1))
    return out.view(n, n, n), origin


def sphere_grid(radius: float, n: int, pitch: float, device="cpu", shift=DEFAULT_SHIFT):
    g, origin = _field(n, pitch, lambda X: X.norm(dim=-1) - radius, device, shift=shift)
    return _pack("sphere", g, origin, pitch, radius, {"radius": radius})


def box_grid(half, n: int, pitch: float, device="cpu", shift=DEFAULT_SHIFT):
    hb = torch.tensor(half, dtype=F64, device=device)

    def fn(X):
        q = X.abs() - hb
        outside = q.clamp(min=0).norm(dim=-1)
        inside = q.max(dim=-1).values.clamp(max=0)
        return outside + inside
    g, origin = _field(n, pitch, fn, device, shift=shift)
    return _pack("box", g, origin, pitch, float(np.linalg.norm(half)), {"half": list(half)})


def linear_grid(coef, offset: float, n: int, pitch: float, device="cpu", shift=(0.0, 0.0, 0.0)):
    """A linear field coef . x + offset (not an SDF; used to check interpolation)."""
    c = torch.tensor(coef, dtype=F64, device=device)
    g, origin = _field(n, pitch, lambda X: X @ c + offset, device, shift=shift)
    return _pack("linear", g, origin, pitch, 0.05, {"coef": list(coef), "offset": offset})


def superquadric_grid(semi_axes, eps1: float, eps2: float, n: int, device="cpu", shift=DEFAULT_SHIFT):
    """Superquadric with inside-outside function
    F = (|x/a1|^(2/e2) + |y/a2|^(2/e2))^(e2/e1) + |z/a3|^(2/e1)  (surface F = 1),
    sampled with the radial distance phi(x) = |x| (1 - F(x)^(-e1/2)), which is the
    exact distance to the surface along the ray from the centre (exact for a sphere).
    The grid spans the largest semi-axis plus a 2 cm margin on each side."""
    a = [float(v) for v in semi_axes]
    amax = max(a)
    pitch = (2.0 * amax + 0.04) / (n - 1)
    A = torch.tensor(a, dtype=F64, device=device)

    def fn(X):
        r = (X / A).abs()
        F = (r[:, 0] ** (2.0 / eps2) + r[:, 1] ** (2.0 / eps2)) ** (eps2 / eps1) + r[:, 2] ** (2.0 / eps1)
        rad = X.norm(dim=-1)
        return rad * (1.0 - F.clamp(min=1e-300) ** (-eps1 / 2.0))
    g, origin = _field(n, pitch, fn, device, shift=shift)
    return _pack("superquadric", g, origin, pitch, amax,
                 {"semi_axes": a, "eps1": eps1, "eps2": eps2})


def _convex_hull(points: np.ndarray):
    from scipy.spatial import ConvexHull
    hull = ConvexHull(points)
    tris = points[hull.simplices]                    # [F,3,3]
    eq = hull.equations                              # outward n, offset: n.x + off <= 0 inside
    # orient each triangle counter-clockwise about its outward normal
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    flip = (nrm * eq[:, :3]).sum(-1) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris, eq


def polyhedron_grid(points: np.ndarray, n: int, device="cpu", shift=DEFAULT_SHIFT):
    """Convex hull of ``points`` sampled exactly: inside, the largest face-plane value
    (exact for a convex body); outside, the distance to the nearest face triangle."""
    tris, eq = _convex_hull(np.asarray(points, dtype=np.float64))
    rb = float(np.linalg.norm(points, axis=1).max())
    pitch = (2.0 * rb + 0.04) / (n - 1)
    T = torch.tensor(tris, dtype=F64, device=device)
    E = torch.tensor(eq, dtype=F64, device=device)
    A, B, C = T[:, 0], T[:, 1], T[:, 2]
    nrm = E[:, :3]

    def seg_dist(X, P0, P1):
        d = P1 - P0
        t = (((X[:, None, :] - P0) * d).sum(-1) / (d * d).sum(-1)).clamp(0.0, 1.0)
        return (X[:, None, :] - P0 - t[..., None] * d).norm(dim=-1)

    def fn_chunk(X):
        plane = X @ nrm.T + E[:, 3]                   # [M,F]
        inside_val = plane.max(dim=-1).values
        # projection inside the triangle: same side of all three edges
        proj = X[:, None, :] - plane[..., None] * nrm
        def side(P0, P1):
            return (torch.cross((P1 - P0).expand_as(proj), proj - P0, dim=-1) * nrm).sum(-1)
        inside_tri = (side(A, B) >= 0) & (side(B, C) >= 0) & (side(C, A) >= 0)
        edge = torch.minimum(torch.minimum(seg_dist(X, A, B), seg_dist(X, B, C)), seg_dist(X, C, A))
        dist = torch.where(inside_tri, plane.abs(), edge).min(dim=-1).values
        return torch.where(inside_val < 0, inside_val, dist)

    F = T.shape[0]
    chunk = max(1024, (1 << 22) // max(F, 1))

    def fn(X):
        return torch.cat([fn_chunk(X[s:s + chunk]) for s in range(0, X.shape[0], chunk)])
    g, origin = _field(n, pitch, fn, device, chunk=1 << 20, shift=shift)
    return _pack("polyhedron", g, origin, pitch, rb, {"n_faces": int(F), "points": np.asarray(points).tolist()})


def lazy_object(kind: str, bound_radius: float, make) -> dict:
    """An object whose grid is not built yet: ``realize`` builds it with make(device).
    The bound radius (all the candidate generator needs) is known from the draws."""
    return {"kind": kind, "lazy": make, "bound_radius": float(bound_radius)}


def realize(obj: dict, device="cpu") -> dict:
    """The built object (obj itself when it is not lazy)."""
    return obj["lazy"](device) if "lazy" in obj else obj


def random_superquadric(rng: np.random.Generator, n: int, device="cpu", build: bool = True):
    eps1, eps2 = rng.uniform(0.3, 2.0, size=2)
    semi = rng.uniform(0.02, 0.08, size=3)
    shift = rng.uniform(-0.5, 0.5, size=3)

    def make(dev):
        return superquadric_grid(semi, float(eps1), float(eps2), n, device=dev, shift=shift)
    return make(device) if build else lazy_object("superquadric", float(max(semi)), make)


def random_polyhedron(rng: np.random.Generator, n: int, device="cpu", n_pts=None, build: bool = True):
    """Hull of k ~ U{8..22} points on an ellipsoid (semi-axes U(2, 8) cm): all points
    are extreme, so the hull has 2k - 4 triangular faces (12..40)."""
    k = int(rng.integers(8, 23)) if n_pts is None else int(n_pts)
    semi = rng.uniform(0.02, 0.08, size=3)
    d = rng.normal(size=(k, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    shift = rng.uniform(-0.5, 0.5, size=3)
    pts = d * semi

    def make(dev):
        return polyhedron_grid(pts, n, device=dev, shift=shift)
    return make(device) if build else lazy_object("polyhedron", float(np.linalg.norm(pts, axis=1).max()), make)
