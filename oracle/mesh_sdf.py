"""FP64 oracle of the mesh SDF and the Phong SDF (Sec. III-B, "Signed distance
function" and "Phong SDF").

TEST INFRASTRUCTURE ONLY, like ``fastgraspd_oracle``.

For a watertight triangle mesh in canonical pose:

  closest point   r* = the closest point on the mesh surface to r, found here by
                  brute force over every triangle (the paper uses a BVH; a brute
                  force search is the plain definition);
  sign            negative inside the mesh volume.  The paper casts a ray; on a
                  watertight mesh the angle-weighted pseudonormal of the closest
                  feature (face, edge or vertex) gives the same answer without a
                  second search: s = sign((r - r*) . N_feature), s = +1 on the surface;
  phi(r)          s |r - r*|;
  Phong point     with barycentric coordinates (b_i, b_j, b_k) of r* on its face and
                  vertex normals n_i, n_j, n_k (angle-weighted averages of the
                  incident face normals), psi_x(q) = q - ((q - v_x) . n_x) n_x is the
                  projection of q onto the tangent plane at vertex x, and the point on
                  the Phong-tessellated surface is
                  r*_rho = (1 - a) r* + a (b_i psi_i(r*) + b_j psi_j(r*) + b_k psi_k(r*)),
                  with a the blend between the flat (a = 0) and curved triangle;
  Phong SDF       rho(r) = s |r - r*_rho|, with the gradient the paper gives,
                  grad rho = s (r - r*_rho) / |r - r*_rho|: r*_rho is held fixed when
                  differentiating (``mesh_eval`` treats it as a decision-like constant).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

F64 = torch.float64

# Phong tessellation blend: the paper leaves it unset; 3/4 is the value the
# Phong-tessellation technique recommends.
PHONG_ALPHA = 0.75


@dataclass
class MeshObj:
    V: np.ndarray              # [V,3] float64
    F: np.ndarray              # [F,3] int64
    face_n: np.ndarray         # [F,3] unit face normals
    vert_n: np.ndarray         # [V,3] angle-weighted vertex normals (Phong and vertex pseudonormals)
    edge_n: np.ndarray         # [F,3,3] pseudonormal of local edge e = (k, k+1 mod 3) of each face
    inv_mass: float
    inv_inertia: float
    alpha: float = PHONG_ALPHA

    @staticmethod
    def from_synth(m: dict, alpha: float = PHONG_ALPHA) -> "MeshObj":
        V = np.asarray(m["vertices"], dtype=np.float64)
        F = np.asarray(m["faces"], dtype=np.int64)
        fn, vn, en = mesh_normals(V, F)
        return MeshObj(V, F, fn, vn, en, 1.0 / float(m["mass"]), 1.0 / float(m["inertia"]), alpha)


def mesh_normals(V: np.ndarray, F: np.ndarray):
    """Unit face normals, angle-weighted vertex normals, and per face-edge
    pseudonormals (sum of the normals of the two faces sharing the edge)."""
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(B - A, C - A)
    fn = n / np.linalg.norm(n, axis=1, keepdims=True)
    vn = np.zeros_like(V)
    corners = (A, B, C)
    for k in range(3):
        p0, p1, p2 = corners[k], corners[(k + 1) % 3], corners[(k + 2) % 3]
        e1 = p1 - p0
        e2 = p2 - p0
        cosang = (e1 * e2).sum(1) / (np.linalg.norm(e1, axis=1) * np.linalg.norm(e2, axis=1))
        ang = np.arccos(np.clip(cosang, -1.0, 1.0))
        np.add.at(vn, F[:, k], ang[:, None] * fn)
    vn /= np.linalg.norm(vn, axis=1, keepdims=True)
    owner = {}
    for f, (a, b, c) in enumerate(F):
        for e, (u, v) in enumerate(((a, b), (b, c), (c, a))):
            owner[(int(u), int(v))] = (f, e)
    en = np.zeros((len(F), 3, 3))
    for f, (a, b, c) in enumerate(F):
        for e, (u, v) in enumerate(((a, b), (b, c), (c, a))):
            g, _ = owner[(int(v), int(u))]           # the face across the edge (watertight)
            s = fn[f] + fn[g]
            en[f, e] = s / np.linalg.norm(s)
    return fn, vn, en


# Region codes of the closest point on a triangle (a, b, c)
FACE, EDGE_AB, EDGE_BC, EDGE_CA, VERT_A, VERT_B, VERT_C = range(7)


def closest_on_triangles(p: np.ndarray, a: np.ndarray, b: np.ndarray, c: np.ndarray):
    """Closest points of p [N,3] on triangles (a, b, c) [F,3] by the Voronoi regions of
    the triangle's vertices, edges and face.  Returns q [N,F,3], barycentric
    coordinates [N,F,3] and region codes [N,F]."""
    p = p[:, None, :]
    ab, ac = (b - a)[None], (c - a)[None]
    ap, bp, cp = p - a[None], p - b[None], p - c[None]
    d1, d2 = (ab * ap).sum(-1), (ac * ap).sum(-1)
    d3, d4 = (ab * bp).sum(-1), (ac * bp).sum(-1)
    d5, d6 = (ab * cp).sum(-1), (ac * cp).sum(-1)
    vc = d1 * d4 - d3 * d2
    vb = d5 * d2 - d1 * d6
    va = d3 * d6 - d5 * d4
    N, Fn = d1.shape
    bary = np.zeros((N, Fn, 3))
    region = np.full((N, Fn), -1, dtype=np.int64)

    def assign(mask, code, u, v, w):
        m = mask & (region < 0)
        region[m] = code
        bary[m, 0] = u[m] if np.ndim(u) else u
        bary[m, 1] = v[m] if np.ndim(v) else v
        bary[m, 2] = w[m] if np.ndim(w) else w

    with np.errstate(divide="ignore", invalid="ignore"):
        assign((d1 <= 0) & (d2 <= 0), VERT_A, 1.0, 0.0, 0.0)
        assign((d3 >= 0) & (d4 <= d3), VERT_B, 0.0, 1.0, 0.0)
        t_ab = d1 / (d1 - d3)
        assign((vc <= 0) & (d1 >= 0) & (d3 <= 0), EDGE_AB, 1.0 - t_ab, t_ab, 0.0 * t_ab)
        assign((d6 >= 0) & (d5 <= d6), VERT_C, 0.0, 0.0, 1.0)
        t_ac = d2 / (d2 - d6)
        assign((vb <= 0) & (d2 >= 0) & (d6 <= 0), EDGE_CA, 1.0 - t_ac, 0.0 * t_ac, t_ac)
        t_bc = (d4 - d3) / ((d4 - d3) + (d5 - d6))
        assign((va <= 0) & ((d4 - d3) >= 0) & ((d5 - d6) >= 0), EDGE_BC, 0.0 * t_bc, 1.0 - t_bc, t_bc)
        den = va + vb + vc
        v_, w_ = vb / den, vc / den
        assign(np.ones_like(region, dtype=bool), FACE, 1.0 - v_ - w_, v_, w_)
    q = bary[..., 0:1] * a[None] + bary[..., 1:2] * b[None] + bary[..., 2:3] * c[None]
    return q, bary, region


# Closest points of two faces closer than this fraction of the distance count as the
# same point for gap_dir (their directions from p differ by less).
SAME_POINT = 1e-2


def mesh_query(mesh: MeshObj, p: np.ndarray, chunk: int = 2048) -> dict:
    """Closest face, point, barycentrics, region, sign and Phong point for p [N,3];
    also, for the guard band, two gaps:

    gap      the closest distance over faces that share no vertex with the closest
             face, minus the closest distance (a near tie with a face elsewhere is a
             medial-axis ambiguity; a choice between faces that share an edge or a
             vertex at the closest point does not matter: the point, its
             pseudonormal and the Phong point are the same from either);
    gap_dir  the same over every face, adjacent or not, whose own closest point lies
             further than SAME_POINT times the distance from the closest point: at a
             concave edge of a non-convex mesh (or inside a convex corner) two
             neighbouring faces can both be closest at interior points, and picking
             the other one turns the direction from the closest point."""
    V, F = mesh.V, mesh.F
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    N = p.shape[0]
    out = {k: [] for k in ("face", "q", "bary", "region", "dist", "gap", "gap_dir")}
    for s in range(0, N, chunk):
        ps = p[s:s + chunk]
        q, bary, region = closest_on_triangles(ps, a, b, c)
        d2 = ((ps[:, None, :] - q) ** 2).sum(-1)
        f = np.argmin(d2, axis=1)
        i = np.arange(len(ps))
        best = d2[i, f]
        qf = q[i, f]
        Ff = F[f]
        adjacent = (F[None, :, :, None] == Ff[:, None, None, :]).any(axis=(-1, -2))
        other = np.where(adjacent, np.inf, d2).min(axis=1)
        same_point = np.linalg.norm(q - qf[:, None, :], axis=-1) <= SAME_POINT * np.sqrt(best)[:, None]
        other_dir = np.where(same_point, np.inf, d2).min(axis=1)
        out["face"].append(f)
        out["q"].append(qf)
        out["bary"].append(bary[i, f])
        out["region"].append(region[i, f])
        out["dist"].append(np.sqrt(best))
        out["gap"].append(np.sqrt(other) - np.sqrt(best))
        out["gap_dir"].append(np.sqrt(other_dir) - np.sqrt(best))
    res = {k: np.concatenate(v) for k, v in out.items()}
    res["sign"] = mesh_sign(mesh, p, res)
    res["q_rho"] = phong_point(mesh, res["face"], res["bary"], res["q"])
    return res


def mesh_sign(mesh: MeshObj, p: np.ndarray, res: dict) -> np.ndarray:
    """+1 outside or on the surface, -1 inside, from the pseudonormal of the closest feature."""
    f, reg = res["face"], res["region"]
    Nf = np.empty((len(f), 3))
    face = reg == FACE
    Nf[face] = mesh.face_n[f[face]]
    for code, e in ((EDGE_AB, 0), (EDGE_BC, 1), (EDGE_CA, 2)):
        m = reg == code
        Nf[m] = mesh.edge_n[f[m], e]
    for code, k in ((VERT_A, 0), (VERT_B, 1), (VERT_C, 2)):
        m = reg == code
        Nf[m] = mesh.vert_n[mesh.F[f[m], k]]
    dot = ((p - res["q"]) * Nf).sum(-1)
    return np.where(dot < 0, -1.0, 1.0)


def phong_point(mesh: MeshObj, face: np.ndarray, bary: np.ndarray, q: np.ndarray) -> np.ndarray:
    """r*_rho = (1 - a) r* + a sum_x b_x psi_x(r*), psi_x(r*) = r* - ((r* - v_x) . n_x) n_x."""
    acc = np.zeros_like(q)
    for k in range(3):
        vk = mesh.V[mesh.F[face, k]]
        nk = mesh.vert_n[mesh.F[face, k]]
        psi = q - (((q - vk) * nk).sum(-1))[:, None] * nk
        acc += bary[:, k:k + 1] * psi
    return (1.0 - mesh.alpha) * q + mesh.alpha * acc


def mesh_decisions(mesh: MeshObj, p: torch.Tensor) -> dict:
    """The lookup's decisions at p [...,3]: closest face and region, sign, and the
    Phong point (constant under differentiation, as in the paper's gradient)."""
    shape = p.shape[:-1]
    flat = p.detach().reshape(-1, 3).cpu().numpy()
    res = mesh_query(mesh, flat)
    t = lambda x, dt=F64: torch.as_tensor(x, dtype=dt).reshape(shape + x.shape[1:])
    return {"face": t(res["face"], torch.long), "region": t(res["region"], torch.long),
            "sign": t(res["sign"]), "q_rho": t(res["q_rho"]), "gap": t(res["gap"]), "dist": t(res["dist"]),
            "gap_dir": t(res["gap_dir"])}


def mesh_eval(mesh: MeshObj, p: torch.Tensor, dec: dict):
    """rho(p) = s |p - r*_rho| and grad rho = s (p - r*_rho)/|p - r*_rho| (zero at the
    Phong point itself)."""
    diff = p - dec["q_rho"]
    d2 = (diff * diff).sum(-1)
    nz = d2 > 0
    d = torch.sqrt(torch.where(nz, d2, torch.ones_like(d2)))
    rho = dec["sign"] * torch.where(nz, d, torch.zeros_like(d))
    grad = torch.where(nz[..., None], dec["sign"][..., None] * diff / d[..., None], torch.zeros_like(diff))
    return rho, grad
