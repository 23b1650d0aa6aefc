"""The C-ABI library builds, loads and exports what include/fastgraspd.h declares
(no GPU: no compute calls, only host-side entry points)."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(inc, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(fg_[A-Za-z0-9_]+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    from paper_2306_08132_gb300 import _lib
    return _lib.load()


def test_header_declares_the_hot_path_calls():
    names = _declared_functions()
    for n in ("fg_fk", "fg_sdf_query", "fg_contact_wrench", "fg_loss_and_grad", "fg_optimize_step",
              "fg_hand_create", "fg_sdf_create", "fg_scene_create", "fg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2306_08132_gb300 import _lib
    assert _declared_functions() <= set(_lib.SIGNATURES)


def test_host_only_entry_points(lib):
    a, b = C.c_int(), C.c_int()
    assert lib.fg_version(C.byref(a), C.byref(b)) == 0 and a.value >= 1
    assert lib.fg_status_string(3) == b"FG_ERR_BUDGET"
    assert lib.fg_status_string(99) == b"FG_ERR_UNKNOWN"
    buf = C.create_string_buffer(8)
    assert lib.fg_last_error(buf, 8) == 0
    assert lib.fg_last_error(None, 8) == 1


def test_invalid_descriptors_are_rejected_before_any_device_work(lib):
    """Validation runs on the host and returns FG_ERR_INVALID with a message."""
    import numpy as np
    from paper_2306_08132_gb300 import _lib
    out = C.c_void_p()
    assert lib.fg_hand_create(None, C.byref(out)) == 1
    par = np.array([-1, 0, 0], dtype=np.int32)
    bad_par = np.array([-1, 2, 0], dtype=np.int32)          # not topological
    tf = np.zeros((3, 12), dtype=np.float32)
    ax = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0]], dtype=np.float32)   # non-unit axis
    lo = np.zeros(2, dtype=np.float32)
    up = np.ones(2, dtype=np.float32)
    pts = np.zeros((4, 3), dtype=np.float32)
    lop = np.array([0, 1, 2, 1], dtype=np.int32)            # not sorted
    P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
    d = _lib.HandDesc(3, 4, P(bad_par, C.c_int), P(tf, C.c_float), P(ax, C.c_float), P(lo, C.c_float),
                      P(up, C.c_float), P(pts, C.c_float), P(lop, C.c_int))
    assert lib.fg_hand_create(C.byref(d), C.byref(out)) == 1
    assert b"topological" in _last(lib)
    d.parent = P(par, C.c_int)
    assert lib.fg_hand_create(C.byref(d), C.byref(out)) == 1
    assert b"unit" in _last(lib)
    org = (C.c_float * 3)(0, 0, 0)
    assert lib.fg_sdf_create(None, 4, 4, 4, org, 0.1, 1.0, 1.0, C.byref(out)) == 1
    g = np.zeros(8, dtype=np.float32)
    assert lib.fg_sdf_create(g.ctypes.data_as(C.c_void_p), 1, 2, 2, org, 0.1, 1.0, 1.0, C.byref(out)) == 1
    assert lib.fg_scene_create(None, 0, C.byref(out)) == 1


def _last(lib):
    buf = C.create_string_buffer(512)
    lib.fg_last_error(buf, 512)
    return buf.value


def test_invalid_meshes_are_rejected_on_the_host(lib):
    """fg_sdf_create_mesh validates on the host: index range, repeated vertices,
    zero-area faces, orientation, watertightness; each with its reason."""
    import numpy as np
    from synth import meshes as SM
    m = SM.box_mesh((0.03, 0.02, 0.05))
    V, F = m["vertices"], m["faces"].copy()
    out = C.c_void_p()

    def create(Vx, Fx, alpha=0.75):
        Vx = np.ascontiguousarray(Vx, dtype=np.float32)
        Fx = np.ascontiguousarray(Fx, dtype=np.int32)
        return lib.fg_sdf_create_mesh(Vx.ctypes.data_as(C.POINTER(C.c_float)), len(Vx),
                                      Fx.ctypes.data_as(C.POINTER(C.c_int)), len(Fx), alpha, 1.0, 1.0,
                                      C.byref(out))
    bad = F.copy(); bad[3, 1] = 99
    assert create(V, bad) == 1 and b"out of range" in _last(lib)
    bad = F.copy(); bad[2, 2] = bad[2, 0]
    assert create(V, bad) == 1 and b"repeated" in _last(lib)
    assert create(V, F[:, ::-1]) == 1 and b"counter-clockwise" in _last(lib)
    assert create(V, F[:-1]) == 1 and b"watertight" in _last(lib)
    bad = F.copy(); bad[0] = bad[0][[0, 2, 1]]
    assert create(V, bad) == 1 and b"directed edge" in _last(lib)
    Vd = V.copy(); Vd[1] = Vd[0] + 1e-12
    assert create(Vd, F) == 1 and (b"zero-area" in _last(lib) or b"directed" in _last(lib))
    assert create(V, F, alpha=1.5) == 1 and b"phong_alpha" in _last(lib)


def test_valid_meshes_pass_host_validation(lib):
    """Convex and non-convex watertight meshes (box, icosphere, superquadric, hull, and
    tori whose tubes have 3 to 12 faces) pass fg_sdf_create_mesh's host validation and
    BVH build; without a GPU the call then stops at the device copy."""
    import numpy as np
    from synth import meshes as SM
    rng = np.random.default_rng(7)
    meshes = [SM.box_mesh((0.03, 0.02, 0.05)), SM.icosphere(0.04, 2),
              SM.superquadric_mesh((0.05, 0.03, 0.04), 0.7, 1.3, 12, 24), SM.hull_mesh(rng.normal(size=(30, 3)) * 0.04),
              SM.torus_mesh(0.04, 0.015, 24, 12), SM.torus_mesh(0.04, 0.015, 6, 3)]
    for m in meshes:
        V = np.ascontiguousarray(m["vertices"], dtype=np.float32)
        F = np.ascontiguousarray(m["faces"], dtype=np.int32)
        out = C.c_void_p()
        st = lib.fg_sdf_create_mesh(V.ctypes.data_as(C.POINTER(C.c_float)), len(V),
                                    F.ctypes.data_as(C.POINTER(C.c_int)), len(F), 0.75, 1.0, 1.0, C.byref(out))
        if st == 0:
            assert lib.fg_sdf_destroy(out) == 0
        else:
            assert st == 5 and b"device copy" in _last(lib), (m["kind"], st, _last(lib))


def test_mesh_description_on_the_host(lib):
    """fg_mesh_describe runs the mesh build on the host: on a convex superquadric mesh (outward-folding quad
    diagonals) and a convex hull every face is on the hull and every vertex's faces form one fan; on a torus
    the inner half is off the hull; on two tetrahedra sharing a vertex, that vertex has two fans; invalid
    meshes are refused with the creation call's messages."""
    import numpy as np
    from synth import meshes as SM
    import paper_2306_08132_gb300 as fg

    def desc(m):
        return fg.Sdf.describe_mesh(m["vertices"], m["faces"])

    sq = SM.superquadric_mesh((0.05, 0.03, 0.04), 0.7, 1.3, 24, 48)
    d = desc(sq)
    assert d["faces"] == len(sq["faces"]) == d["hull_faces"]
    assert d["fan_vertices"] == len(sq["vertices"])
    assert d["bvh_nodes"] >= 2 * (d["faces"] // 4) - 1 and 1 <= d["bvh_depth"] <= 48
    assert 2 <= d["start_nodes"] <= 32 ** 3
    hull = SM.hull_mesh(np.random.default_rng(3).normal(size=(60, 3)) * 0.04)
    assert desc(hull)["hull_faces"] == len(hull["faces"])
    torus = SM.torus_mesh(0.04, 0.015, 24, 12)
    dt = desc(torus)
    assert 0 < dt["hull_faces"] < len(torus["faces"]) // 2 + len(torus["faces"]) // 4
    assert dt["fan_vertices"] == len(torus["vertices"])
    s = 0.03
    V = np.array([(0, 0, 0), (s, 0, s), (s, s, -s), (s, -s, -s), (-s, 0, s), (-s, -s, -s), (-s, s, -s)], np.float32)
    F = np.array([(0, 1, 2), (0, 2, 3), (0, 3, 1), (1, 3, 2), (0, 4, 5), (0, 5, 6), (0, 6, 4), (4, 6, 5)])
    for t in range(len(F)):                       # each face away from its tetrahedron's centroid
        A, B, Cc = V[F[t]].astype(np.float64)
        cen = V[[1, 2, 3]].mean(0) if 1 in F[t] or 2 in F[t] or 3 in F[t] else V[[4, 5, 6]].mean(0)
        if np.cross(B - A, Cc - A) @ ((A + B + Cc) / 3 - cen) < 0:
            F[t] = F[t][[0, 2, 1]]
    db = fg.Sdf.describe_mesh(V, F)
    assert db["fan_vertices"] == len(V) - 1            # the shared vertex: two fans
    with pytest.raises(Exception, match="watertight"):
        fg.Sdf.describe_mesh(sq["vertices"], sq["faces"][:-1])
