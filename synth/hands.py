"""Synthetic articulated capsule hands (stand-ins for the Barrett/Allegro/Shadow models).

The paper represents a hand by a mesh plus an articulation chain whose links carry
meshes, and every hand vertex imposes a contact constraint (Sec. III, Sec. III-C).
No hand model ships with the paper, so three synthetic hands are generated here:

* ``3``: palm + 3 fingers x 3 flexion links              -> 10 links,  9 joints
* ``4``: palm + 4 fingers x (abduction + 3 flexion)        -> 17 links, 16 joints
* ``5``: the 4-finger layout with the two ulnar fingers mounted on a palm-arch
  link, plus a 5-link thumb                                -> 23 links, 22 joints

Every non-root link carries exactly one revolute joint (joint j drives link j+1),
so the configuration vector is q = (t[3], w[3], theta[J]) with D = 6 + J.

Geometry (metres): capsule links of radius 9 mm with flexion lengths 45/30/25 mm,
10 mm abduction knuckles, and a 9 x 9 x 2.5 cm box palm.  Surface points are a
deterministic Fibonacci sampling of each capsule (area-uniform) and a stratified
golden-ratio lattice on the box faces, listed per link in Morton order so that
consecutive points are neighbours on the surface.

Each link is first placed by its REST world frame (rotation R_l, origin o_l).  The
fixed parent->child transforms are then derived as T_fix = T_rest(parent)^-1 T_rest(l),
so the rest pose stored here is an independent statement of where the points sit
at q = 0 with an identity base.
"""

from __future__ import annotations

import math
import numpy as np

HAND_KINDS = (3, 4, 5)

CAPSULE_RADIUS = 0.009
FLEX_LENGTHS = (0.045, 0.030, 0.025)
THUMB_FLEX_LENGTHS = (0.035, 0.030, 0.025)
KNUCKLE_LENGTH = 0.010
PALM_HALF = (0.045, 0.045, 0.0125)

FLEX_LIMITS = (0.0, 1.6)
ABD_LIMITS = (-0.35, 0.35)
ARCH_LIMITS = (0.0, 0.5)

_GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))
_INV_PHI = (math.sqrt(5.0) - 1.0) / 2.0


def _rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def capsule_points(length: float, radius: float, n: int) -> np.ndarray:
    """Area-uniform Fibonacci samples on a capsule whose axis runs along local +y
    from y=0 to y=length (hemispherical caps at both ends)."""
    area_cap = 2.0 * math.pi * radius * radius          # one hemisphere
    area_cyl = 2.0 * math.pi * radius * length
    total = 2.0 * area_cap + area_cyl
    fb, fc = area_cap / total, area_cyl / total
    out = np.empty((n, 3), dtype=np.float64)
    for i in range(n):
        a = (i + 0.5) / n
        az = (i * _GOLDEN_ANGLE) % (2.0 * math.pi)
        if a < fb:                                      # bottom cap, pole at y=-r
            zeta = (a / fb) * radius                    # height above the pole
            y = -radius + zeta
            rho = math.sqrt(max(radius * radius - y * y, 0.0))
        elif a < fb + fc:                               # cylinder
            y = ((a - fb) / fc) * length
            rho = radius
        else:                                           # top cap, pole at y=length+r
            zeta = ((a - fb - fc) / fb) * radius        # height above y=length
            y = length + zeta
            rho = math.sqrt(max(radius * radius - zeta * zeta, 0.0))
        out[i] = (rho * math.cos(az), y, rho * math.sin(az))
    return out


def box_points(half, n: int) -> np.ndarray:
    """Stratified golden-ratio lattice on the six faces of an axis-aligned box."""
    hx, hy, hz = half
    faces = []   # (area, fixed axis, sign)
    for axis, (u_half, v_half) in ((0, (hy, hz)), (1, (hx, hz)), (2, (hx, hy))):
        for sign in (-1.0, 1.0):
            faces.append((4.0 * u_half * v_half, axis, sign))
    areas = np.array([f[0] for f in faces])
    raw = areas / areas.sum() * n
    counts = np.floor(raw).astype(int)
    rem = n - counts.sum()
    for idx in np.argsort(-(raw - counts), kind="stable")[:rem]:
        counts[idx] += 1
    pts = []
    for (area, axis, sign), k in zip(faces, counts):
        others = [a for a in range(3) if a != axis]
        for i in range(k):
            u = (i + 0.5) / k
            v = (i * _INV_PHI) % 1.0
            p = [0.0, 0.0, 0.0]
            p[axis] = sign * half[axis]
            p[others[0]] = (2.0 * u - 1.0) * half[others[0]]
            p[others[1]] = (2.0 * v - 1.0) * half[others[1]]
            pts.append(p)
    return np.array(pts, dtype=np.float64)


def box_point_areas(half, n: int) -> np.ndarray:
    """Area each sample of ``box_points(half, n)`` stands for (its face's area over
    the face's sample count), in the same order."""
    hx, hy, hz = half
    areas = []
    for u_half, v_half in ((hy, hz), (hx, hz), (hx, hy)):
        areas += [4.0 * u_half * v_half] * 2
    areas = np.array(areas)
    raw = areas / areas.sum() * n
    counts = np.floor(raw).astype(int)
    rem = n - counts.sum()
    for idx in np.argsort(-(raw - counts), kind="stable")[:rem]:
        counts[idx] += 1
    return np.concatenate([np.full(k, a / k) for a, k in zip(areas, counts) if k > 0])


def capsule_area(length: float, radius: float) -> float:
    return 2.0 * math.pi * radius * length + 4.0 * math.pi * radius * radius


def _morton_order(pts: np.ndarray) -> np.ndarray:
    """Order of points along a Morton (Z-order) curve of their 10-bit quantised
    coordinates, so that consecutive points are spatially close."""
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    q = np.floor((pts - lo) / np.maximum(hi - lo, 1e-12) * 1023.0).astype(np.int64)
    code = np.zeros(len(pts), dtype=np.int64)
    for bit in range(10):
        for axis in range(3):
            code |= ((q[:, axis] >> bit) & 1) << (3 * bit + axis)
    return np.argsort(code, kind="stable")


def _layout(kind: int):
    """Return link specs: (name, parent_index, R_rest, o_rest, axis_local, shape, limits)."""
    eye = np.eye(3)
    links = [("palm", -1, eye, np.zeros(3), np.zeros(3), ("box", PALM_HALF), None)]

    def add(name, parent, R, o, axis, shape, limits):
        links.append((name, parent, R, np.asarray(o, dtype=np.float64),
                       np.asarray(axis, dtype=np.float64), shape, limits))
        return len(links) - 1

    def finger(tag, parent_idx, x, with_abd):
        y = PALM_HALF[1]
        par = parent_idx
        if with_abd:
            par = add(f"{tag}_abd", par, eye, (x, y, 0.0), (0, 0, 1),
                      ("capsule", KNUCKLE_LENGTH), ABD_LIMITS)
            y += KNUCKLE_LENGTH
        for k, ln in enumerate(FLEX_LENGTHS):
            par = add(f"{tag}_flex{k + 1}", par, eye, (x, y, 0.0), (1, 0, 0),
                      ("capsule", ln), FLEX_LIMITS)
            y += ln

    if kind == 3:
        for i, x in enumerate((-0.03, 0.0, 0.03)):
            finger(f"f{i}", 0, x, with_abd=False)
    elif kind == 4:
        for i, x in enumerate((-0.0375, -0.0125, 0.0125, 0.0375)):
            finger(f"f{i}", 0, x, with_abd=True)
    elif kind == 5:
        xs = (-0.0375, -0.0125, 0.0125, 0.0375)
        finger("f0", 0, xs[0], with_abd=True)
        finger("f1", 0, xs[1], with_abd=True)
        arch = add("arch", 0, eye, (0.025, 0.005, 0.0), (0, -1, 0),
                   ("capsule", 0.035), ARCH_LIMITS)
        finger("f2", arch, xs[2], with_abd=True)
        finger("f3", arch, xs[3], with_abd=True)
        R_th = _rot_z(math.radians(50.0)) @ _rot_x(math.radians(20.0))
        base = np.array([-PALM_HALF[0], -0.005, 0.0])
        along = 0.0
        par = 0
        specs = [("th_rot", (0, 1, 0), KNUCKLE_LENGTH, ABD_LIMITS),
                 ("th_abd", (0, 0, 1), KNUCKLE_LENGTH, ABD_LIMITS)]
        specs += [(f"th_flex{k + 1}", (1, 0, 0), ln, FLEX_LIMITS)
                  for k, ln in enumerate(THUMB_FLEX_LENGTHS)]
        for name, axis, ln, lim in specs:
            o = base + R_th @ np.array([0.0, along, 0.0])
            par = add(name, par, R_th, o, axis, ("capsule", ln), lim)
            along += ln
    else:
        raise ValueError(f"unknown hand kind {kind}")
    return links


def make_hand(kind: int, points_per_link: int) -> dict:
    """Build a synthetic hand.  Arrays are float32 for the compute paths; the rest
    pose (``rest_*``) is kept in float64 for checks."""
    specs = _layout(kind)
    L = len(specs)
    J = L - 1
    parent = np.array([s[1] for s in specs], dtype=np.int32)
    assert all(parent[l] < l for l in range(1, L))
    rest_R = np.stack([s[2] for s in specs])
    rest_o = np.stack([s[3] for s in specs])
    axis = np.stack([s[4] for s in specs]).astype(np.float32)
    T_fix = np.zeros((L, 3, 4), dtype=np.float64)
    T_fix[0, :, :3] = np.eye(3)
    for l in range(1, L):
        p = parent[l]
        T_fix[l, :, :3] = rest_R[p].T @ rest_R[l]
        T_fix[l, :, 3] = rest_R[p].T @ (rest_o[l] - rest_o[p])
    q_low = np.array([specs[l][6][0] for l in range(1, L)], dtype=np.float32)
    q_up = np.array([specs[l][6][1] for l in range(1, L)], dtype=np.float32)

    local, link_of_point, link_start, areas = [], [], [0], []
    for l, s in enumerate(specs):
        shape = s[5]
        if shape[0] == "box":
            pts = box_points(shape[1], points_per_link)
            w = box_point_areas(shape[1], points_per_link)
        else:
            pts = capsule_points(shape[1], CAPSULE_RADIUS, points_per_link)
            w = np.full(len(pts), capsule_area(shape[1], CAPSULE_RADIUS) / len(pts))
        order = _morton_order(pts)             # spatially coherent runs of 32 points
        pts = pts[order]
        areas.append(w[order])
        local.append(pts)
        link_of_point.extend([l] * len(pts))
        link_start.append(link_start[-1] + len(pts))
    pts_local64 = np.concatenate(local, axis=0)
    pts_local = pts_local64.astype(np.float32)
    lop = np.array(link_of_point, dtype=np.int32)
    # rest pose from the (float32-rounded) local samples, placed by the rest frames
    p32 = pts_local.astype(np.float64)
    rest_pts = np.einsum("pij,pj->pi", rest_R[lop], p32) + rest_o[lop]
    return {
        "kind": kind,
        "names": [s[0] for s in specs],
        "L": L, "J": J, "D": 6 + J, "P": int(len(lop)),
        "parent": parent,
        "T_fix": T_fix.astype(np.float32),
        "axis": axis,
        "q_low": q_low, "q_up": q_up,
        "pts_local": pts_local,
        "link_of_point": lop,
        "link_start": np.array(link_start, dtype=np.int32),
        "rest_R": rest_R, "rest_o": rest_o, "rest_pts": rest_pts,
        "point_area": np.concatenate(areas).astype(np.float32),     # m^2 each surface sample stands for
    }


def interior_hand(kind: int, spacing: float) -> dict:
    """The same hand with its links' interiors sampled instead of their surfaces: a
    cubic lattice of the given spacing (metres) in each link frame, the nodes inside
    the capsule (or palm box), each standing for spacing^3 of volume (``point_volume``).
    Links overlap at the joints; each link keeps its own samples."""
    base = make_hand(kind, 8)
    specs = _layout(kind)
    local, lop, vol = [], [], []
    for l, s in enumerate(specs):
        shape = s[5]
        if shape[0] == "box":
            h = np.asarray(shape[1])
            axes = [np.arange(-h[k] + 0.5 * spacing, h[k], spacing) for k in range(3)]
            X, Y, Z = np.meshgrid(*axes, indexing="ij")
            pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1)
        else:
            ln, r = shape[1], CAPSULE_RADIUS
            ax = np.arange(-r + 0.5 * spacing, r, spacing)
            ay = np.arange(-r + 0.5 * spacing, ln + r, spacing)
            X, Y, Z = np.meshgrid(ax, ay, ax, indexing="ij")
            pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1)
            yc = np.clip(pts[:, 1], 0.0, ln)
            inside = (pts[:, 0] ** 2 + (pts[:, 1] - yc) ** 2 + pts[:, 2] ** 2) <= r * r
            pts = pts[inside]
        pts = pts[_morton_order(pts)]
        local.append(pts)
        lop.extend([l] * len(pts))
        vol.append(np.full(len(pts), spacing ** 3))
    out = dict(base)
    pts_local = np.concatenate(local).astype(np.float32)
    out.update({"P": int(len(lop)), "pts_local": pts_local, "link_of_point": np.array(lop, dtype=np.int32),
                "point_volume": np.concatenate(vol).astype(np.float32)})
    for key in ("point_area", "rest_pts", "link_start"):
        out.pop(key, None)
    return out
