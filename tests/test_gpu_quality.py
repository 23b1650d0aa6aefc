"""GPU grasp-quality metrics (fg_contact_measure, fg_grasp_epsilon) against the
FP64 oracle (oracle/quality.py), through the C ABI.

Tolerances: the contact set is compared exactly (counts) on candidates whose
points all sit more than 1 micrometre from the threshold and 1e-5 voxel from a
cell face and whose contact normals keep |n_z| > 1e-5 (the tangent basis
switches there); sums of weights to 1e-5 relative (float32 accumulation);
epsilon to 1e-5 + 1e-4 |eps| (float32 dot products of unit-scale wrenches)."""

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O
from oracle import quality as Q
from synth import meshes as SM

pytestmark = pytest.mark.gpu

TAU = 0.005
MU = 0.5
EDGES = 8


@pytest.fixture(scope="module")
def fg():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as m
    return m


def _dev():
    return torch.device("cuda:0")


def _eps_close(a, b):
    both_inf = np.isneginf(a) & np.isneginf(b)
    with np.errstate(invalid="ignore"):
        close = np.abs(a - b) <= 1e-5 + 1e-4 * np.abs(b)
    return both_inf | close


@pytest.fixture(scope="module")
def batch(fg):
    """Tiny sphere candidates and 4-finger superquadric candidates, each on its own scene."""
    out = []
    w1 = synth.tiny_sphere_workload(n_cand=24)
    w2 = synth.batched_superquadric_workload(n_obj=2, per_obj=12, grid_n=48, points_per_link=32, steps=50)
    for w in (w1, w2):
        hand = fg.Hand.from_synth(w.hand)
        scene = fg.Scene([fg.Sdf.from_synth(o) for o in w.objects])
        S = O.Setup(w.hand, w.objects, w.params)
        ok = np.array([Q.guard_ok(S.hand, S.objs[int(k)], q, TAU) for q, k in zip(w.q0, w.obj_of_cand)])
        out.append((w, hand, scene, S, ok))
    return out


def test_contact_area_matches_oracle(fg, batch):
    for w, hand, scene, S, ok in batch:
        weights = torch.tensor(w.hand["point_area"], device=_dev())
        q = torch.tensor(w.q0, device=_dev())
        oc = torch.tensor(w.obj_of_cand, device=_dev(), dtype=torch.int32)
        ca = fg.contact_measure(hand, scene, q, weights, TAU, obj_of_cand=oc).cpu().numpy().astype(np.float64)
        ref = np.array([Q.measure(S.hand, S.objs[int(k)], qq, w.hand["point_area"], TAU)
                        for qq, k in zip(w.q0, w.obj_of_cand)])
        assert ok.sum() >= 0.6 * len(ok)
        assert (ref[ok] > 0).sum() >= 3, "candidates must touch the objects"
        assert np.all(np.abs(ca - ref)[ok] <= 1e-5 * np.maximum(ref[ok], 1e-6)), np.abs(ca - ref)[ok].max()


def test_intersection_volume_matches_oracle(fg):
    w = synth.tiny_sphere_workload(n_cand=16)
    vh = synth.interior_hand(3, 0.003)
    hand = fg.Hand.from_synth(vh)
    scene = fg.Scene([fg.Sdf.from_synth(o) for o in w.objects])
    S = O.Setup(vh, w.objects, w.params)
    q = torch.tensor(w.q0, device=_dev())
    iv = fg.contact_measure(hand, scene, q, torch.tensor(vh["point_volume"], device=_dev()), 0.0)
    iv = iv.cpu().numpy().astype(np.float64)
    ref = np.array([Q.measure(S.hand, S.objs[0], qq, vh["point_volume"], 0.0) for qq in w.q0])
    ok = np.array([Q.guard_ok(S.hand, S.objs[0], qq, 0.0, nz_tol=-1.0) for qq in w.q0])
    assert ok.sum() >= 8 and (ref[ok] > 0).sum() >= 3
    assert np.all(np.abs(iv - ref)[ok] <= 1e-5 * np.maximum(ref[ok], 1e-12))


def test_epsilon_matches_oracle(fg, batch):
    U = synth.unit_directions(256)
    dirs = torch.tensor(U, device=_dev())
    U64 = U.astype(np.float64)
    for w, hand, scene, S, ok in batch:
        q = torch.tensor(w.q0, device=_dev())
        oc = torch.tensor(w.obj_of_cand, device=_dev(), dtype=torch.int32)
        rho = 0.05
        eps, nc = fg.grasp_epsilon(hand, scene, q, TAU, MU, EDGES, 1.0 / rho, dirs, obj_of_cand=oc)
        eps, nc = eps.cpu().numpy().astype(np.float64), nc.cpu().numpy()
        ref, ncr = [], []
        for qq, k in zip(w.q0, w.obj_of_cand):
            p, n, phi, idx = Q.contacts(S.hand, S.objs[int(k)], qq, TAU)
            ref.append(Q.support_min(Q.cone_wrenches(p, n, MU, EDGES, rho), U64))
            ncr.append(len(p))
        ref, ncr = np.array(ref), np.array(ncr)
        assert np.array_equal(nc[ok], ncr[ok])
        assert (ncr[ok] > 0).sum() >= 3 and (ncr[ok] == 0).sum() >= 1
        assert np.all(_eps_close(eps, ref)[ok]), np.abs(eps - ref)[ok & np.isfinite(ref)].max()


def test_epsilon_at_the_facet_normals_is_the_ferrari_canny_epsilon(fg, batch):
    """With the direction set made of the oracle hull's facet normals the GPU value is
    the exact epsilon of qhull (on candidates with a full-dimensional wrench set)."""
    w, hand, scene, S, ok = batch[0]
    rho = 0.05
    done = 0
    for b in np.nonzero(ok)[0]:
        m = Q.grasp_metrics(S.hand, S.objs[0], w.q0[b], TAU, MU, 4, rho)
        N = m["facet_normals"]
        if m["n_contacts"] < 3 or len(N) == 0 or len(N) > 8192:
            continue
        dirs = torch.tensor(N.astype(np.float32), device=_dev())
        eps, _ = fg.grasp_epsilon(hand, scene, torch.tensor(w.q0[b:b + 1], device=_dev()), TAU, MU, 4, 1.0 / rho,
                                  dirs)
        e = float(eps.cpu()[0])
        assert abs(e - m["eps"]) <= 1e-5 + 1e-4 * abs(m["eps"]), (b, e, m["eps"])
        done += 1
        if done == 4:
            break
    assert done >= 2


def test_quality_on_mesh_objects(fg):
    w = synth.tiny_sphere_workload(n_cand=12)
    mesh = SM.icosphere(0.04, 3)
    hand = fg.Hand.from_synth(w.hand)
    scene = fg.Scene([fg.Sdf.from_synth(mesh)])
    S = O.Setup(w.hand, [mesh], w.params)
    ok = np.array([Q.guard_ok(S.hand, S.objs[0], qq, TAU) for qq in w.q0])
    q = torch.tensor(w.q0, device=_dev())
    ca = fg.contact_measure(hand, scene, q, torch.tensor(w.hand["point_area"], device=_dev()), TAU)
    ref = np.array([Q.measure(S.hand, S.objs[0], qq, w.hand["point_area"], TAU) for qq in w.q0])
    ca = ca.cpu().numpy().astype(np.float64)
    assert ok.sum() >= 6
    assert np.all(np.abs(ca - ref)[ok] <= 1e-5 * np.maximum(ref[ok], 1e-6))
    U = synth.unit_directions(128)
    eps, nc = fg.grasp_epsilon(hand, scene, q, TAU, MU, EDGES, 20.0, torch.tensor(U, device=_dev()))
    for b in np.nonzero(ok)[0]:
        p, n, phi, idx = Q.contacts(S.hand, S.objs[0], w.q0[b], TAU)
        r = Q.support_min(Q.cone_wrenches(p, n, MU, EDGES, 0.05), U.astype(np.float64))
        assert int(nc[b]) == len(p)
        # mesh normals carry the float32 closest-point error (<= 5e-4 in direction)
        assert (np.isneginf(r) and np.isneginf(float(eps[b]))) or abs(float(eps[b]) - r) <= 2e-3 + 1e-3 * abs(r)


def test_quality_arguments_are_checked(fg, batch):
    from paper_2306_08132_gb300 import _lib
    w, hand, scene, S, ok = batch[0]
    q = torch.tensor(w.q0[:2], device=_dev())
    dirs = torch.tensor(synth.unit_directions(4), device=_dev())
    for kw in ({"cone_edges": 0}, {"cone_edges": 33}, {"mu": -1.0}):
        args = dict(tau=TAU, mu=MU, cone_edges=EDGES, torque_scale=20.0)
        args.update(kw)
        with pytest.raises(_lib.FgError):
            fg.grasp_epsilon(hand, scene, q, args["tau"], args["mu"], args["cone_edges"], args["torque_scale"], dirs)
    with pytest.raises(_lib.FgError):
        fg.contact_measure(hand, scene, q, torch.ones(hand.P, device=_dev()), float("nan"))


def test_quality_full_size_sampled(fg):
    """Contact area and epsilon over the benchmark workload's 8,192 candidates (8
    superquadrics on 128^3 grids, 4-finger hand) in one launch each; 12 sampled
    candidates against the oracle."""
    w = synth.batched_superquadric_workload(device="cuda")
    hand = fg.Hand.from_synth(w.hand)
    scene = fg.Scene([fg.Sdf.from_synth(o) for o in w.objects])
    S = O.Setup(w.hand, w.objects, w.params)
    q = torch.tensor(w.q0, device=_dev())
    oc = torch.tensor(w.obj_of_cand, device=_dev(), dtype=torch.int32)
    U = synth.unit_directions(1024)
    ca = fg.contact_measure(hand, scene, q, torch.tensor(w.hand["point_area"], device=_dev()), TAU, obj_of_cand=oc)
    eps, nc = fg.grasp_epsilon(hand, scene, q, TAU, MU, EDGES, 1.0 / 0.08, torch.tensor(U, device=_dev()),
                               obj_of_cand=oc)
    ca, eps, nc = ca.cpu().numpy().astype(np.float64), eps.cpu().numpy().astype(np.float64), nc.cpu().numpy()
    sample = np.sort(np.random.default_rng(13).choice(w.B, size=12, replace=False))
    checked = 0
    for b in sample:
        obj = S.objs[int(w.obj_of_cand[b])]
        if not Q.guard_ok(S.hand, obj, w.q0[b], TAU):
            continue
        p, n, phi, idx = Q.contacts(S.hand, obj, w.q0[b], TAU)
        assert nc[b] == len(p)
        ref_ca = Q.measure(S.hand, obj, w.q0[b], w.hand["point_area"], TAU)
        assert abs(ca[b] - ref_ca) <= 1e-5 * max(ref_ca, 1e-6)
        ref_e = Q.support_min(Q.cone_wrenches(p, n, MU, EDGES, 0.08), U.astype(np.float64))
        assert _eps_close(np.array([eps[b]]), np.array([ref_e]))[0], (b, eps[b], ref_e)
        checked += 1
    assert checked >= 8


def test_quality_ragged_hand(fg):
    """Links not 32-aligned (P = 210, a last chunk of 18 points): contact area, contact
    counts and epsilon against the oracle; an empty batch; a hand far from the object
    (no contact: CA = 0, eps = -inf); object indices outside the scene (NaN, -1)."""
    w = synth.tiny_sphere_workload(n_cand=20)
    h = synth.make_hand(3, 21)
    qs = synth.sample_candidates(np.random.default_rng(7), h, 20, 0.095)
    hand = fg.Hand.from_synth(h)
    scene = fg.Scene([fg.Sdf.from_synth(o) for o in w.objects])
    S = O.Setup(h, w.objects, w.params)
    q = torch.tensor(qs, device=_dev())
    U = synth.unit_directions(64)
    ca = fg.contact_measure(hand, scene, q, torch.tensor(h["point_area"], device=_dev()), TAU).cpu().numpy()
    eps, nc = fg.grasp_epsilon(hand, scene, q, TAU, MU, EDGES, 20.0, torch.tensor(U, device=_dev()))
    eps, nc = eps.cpu().numpy().astype(np.float64), nc.cpu().numpy()
    checked = 0
    for b in range(len(qs)):
        if not Q.guard_ok(S.hand, S.objs[0], qs[b], TAU):
            continue
        p, n, phi, idx = Q.contacts(S.hand, S.objs[0], qs[b], TAU)
        assert nc[b] == len(p)
        ref_ca = Q.measure(S.hand, S.objs[0], qs[b], h["point_area"], TAU)
        assert abs(float(ca[b]) - ref_ca) <= 1e-5 * max(ref_ca, 1e-6)
        ref_e = Q.support_min(Q.cone_wrenches(p, n, MU, EDGES, 0.05), U.astype(np.float64))
        assert _eps_close(np.array([eps[b]]), np.array([ref_e]))[0]
        checked += 1
    assert checked >= 10 and (nc > 0).sum() >= 3
    e0, n0 = fg.grasp_epsilon(hand, scene, q[:0], TAU, MU, EDGES, 20.0, torch.tensor(U, device=_dev()))
    assert e0.numel() == 0
    far = np.zeros((2, h["D"]), dtype=np.float32)
    far[:, 0] = [0.5, -0.4]
    qf = torch.tensor(far, device=_dev())
    assert float(fg.contact_measure(hand, scene, qf, torch.tensor(h["point_area"], device=_dev()), TAU).abs().max()) == 0
    ef, nf = fg.grasp_epsilon(hand, scene, qf, TAU, MU, EDGES, 20.0, torch.tensor(U, device=_dev()))
    assert np.isneginf(ef.cpu().numpy()).all() and (nf.cpu().numpy() == 0).all()
    bad = torch.tensor([0, 5], device=_dev(), dtype=torch.int32)
    eb, nb = fg.grasp_epsilon(hand, scene, q[:2], TAU, MU, EDGES, 20.0, torch.tensor(U, device=_dev()), obj_of_cand=bad)
    assert np.isnan(eb.cpu().numpy()[1]) and nb.cpu().numpy()[1] == -1
