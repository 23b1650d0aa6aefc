"""Workload recipes: hands, objects, candidates and parameters for each benchmark case.

Seeds are ``2306081320 + k`` for workload k.  The recipes stand in for the paper's
YCB/EGAD objects and robot hands, which are not available; sizes follow the five
benchmark cases (tiny sphere, batched superquadrics, convex polyhedra, serving
stream, throughput sweep).  Every recipe takes scale arguments so tests can build
reduced copies with the same structure.
"""

from __future__ import annotations

import dataclasses
import math
import numpy as np

from .hands import make_hand
from .objects import sphere_grid, random_superquadric, random_polyhedron
from .candidates import sample_candidates

SEED_BASE = 2306081320


def default_params(r0: float = 0.004, schedule: str = "fixed") -> dict:
    """Method constants.  alpha_leak, dt and lr are the paper's values (Sec. III-C,
    Sec. IV-A); v_test, mu, the loss weights and r0 are readings where it is silent."""
    return {
        "alpha_leak": 0.1,   # leaky-gradient factor (Sec. III-C)
        "dt": 1e-3,          # one PBD step of 1 ms (Sec. IV-A)
        "v_test": 1.0,       # test-velocity magnitude, m/s (reading)
        "mu": 0.5,           # Coulomb friction coefficient (reading)
        "lr": 1e-3,          # gradient-descent learning rate (Sec. IV-A)
        "r0": r0,            # SDF dilation radius at step 0, metres (reading)
        "w_range": 0.1,      # weight of L_range (reading)
        "w_limit": 1.0,      # weight of L_limit (reading)
        "w_pen": 0.0,        # weight of the explicit penetration sum (reading: off)
        "schedule": schedule,  # "fixed" r = r0, or "linear" r0 -> 0 over the run
        "sim_steps": 0,      # 0: one step on the plane through the query; T >= 1: T re-queried steps
    }


@dataclasses.dataclass
class Workload:
    name: str
    hand: dict
    objects: list
    q0: np.ndarray           # float32 [B, D]
    obj_of_cand: np.ndarray  # int32 [B]
    params: dict
    steps: int

    @property
    def B(self) -> int:
        return int(self.q0.shape[0])

    @property
    def points_per_step(self) -> int:
        return self.B * self.hand["P"]


def _cands_for_objects(rng, hand, objects, per_obj, radius_fn):
    qs, oc = [], []
    for k, ob in enumerate(objects):
        qs.append(sample_candidates(rng, hand, per_obj, radius_fn(ob)))
        oc.append(np.full(per_obj, k, dtype=np.int32))
    return np.concatenate(qs), np.concatenate(oc)


def tiny_sphere_workload(n_cand: int = 16, steps: int = 100, device="cpu") -> Workload:
    """Sphere R = 4 cm on a 64^3 grid with 2 mm pitch (12.6 cm span), 3-finger hand with
    64 points per link (P = 640), palm on a 10 cm sphere, fixed dilation r = 4 mm."""
    rng = np.random.default_rng(SEED_BASE + 1)
    hand = make_hand(3, 64)
    obj = sphere_grid(0.04, 64, 0.002, device=device)
    q0, oc = _cands_for_objects(rng, hand, [obj], n_cand, lambda ob: 0.10)
    return Workload("sphere64_hand3_B%d" % n_cand, hand, [obj], q0, oc,
                    default_params(r0=0.004, schedule="fixed"), steps)


def batched_superquadric_workload(n_obj: int = 8, per_obj: int = 1024, grid_n: int = 128,
                                  points_per_link: int = 256, steps: int = 500,
                                  device="cpu", build: bool = True) -> Workload:
    """Random superquadrics (exponents U(0.3, 2), semi-axes U(2, 8) cm) on grid_n^3
    grids, 4-finger hand (17 links x points_per_link), per_obj candidates per object
    with the palm at R_b + 6 cm, dilation 10 mm -> 0 over the run.  build=False leaves
    the grids unbuilt (``synth.realize`` builds one on demand)."""
    rng = np.random.default_rng(SEED_BASE + 2)
    hand = make_hand(4, points_per_link)
    objs = [random_superquadric(rng, grid_n, device=device, build=build) for _ in range(n_obj)]
    q0, oc = _cands_for_objects(rng, hand, objs, per_obj, lambda ob: ob["bound_radius"] + 0.06)
    return Workload("superquadric%d_%d^3_hand4_B%d" % (n_obj, grid_n, n_obj * per_obj), hand, objs,
                    q0, oc, default_params(r0=0.010, schedule="linear"), steps)


def polyhedra_workload(n_obj: int = 32, per_obj: int = 4096, grid_n: int = 128,
                       points_per_link: int = 256, steps: int = 100, device="cpu", build: bool = True) -> Workload:
    """Convex polyhedra (12-40 faces) on grid_n^3 grids, 5-finger hand (23 links).
    build=False leaves the grids unbuilt (``synth.realize`` builds one on demand)."""
    rng = np.random.default_rng(SEED_BASE + 3)
    hand = make_hand(5, points_per_link)
    objs = [random_polyhedron(rng, grid_n, device=device, build=build) for _ in range(n_obj)]
    q0, oc = _cands_for_objects(rng, hand, objs, per_obj, lambda ob: ob["bound_radius"] + 0.06)
    return Workload("polyhedra%d_%d^3_hand5_B%d" % (n_obj, grid_n, n_obj * per_obj), hand, objs,
                    q0, oc, default_params(r0=0.010, schedule="linear"), steps)


def sweep_workload(n_obj: int = 256, total_cand: int = 65536, grid_n: int = 192,
                   points_per_link: int = 256, steps: int = 1000, device="cpu", build: bool = True) -> Workload:
    """Half superquadrics, half polyhedra on grid_n^3 grids, 5-finger hand.
    build=False leaves the grids unbuilt (``synth.realize`` builds one on demand)."""
    rng = np.random.default_rng(SEED_BASE + 5)
    hand = make_hand(5, points_per_link)
    objs = []
    for k in range(n_obj):
        objs.append(random_superquadric(rng, grid_n, device=device, build=build) if k % 2 == 0
                    else random_polyhedron(rng, grid_n, device=device, build=build))
    per_obj = total_cand // n_obj
    q0, oc = _cands_for_objects(rng, hand, objs, per_obj, lambda ob: ob["bound_radius"] + 0.06)
    return Workload("sweep%d_%d^3_hand5_B%d" % (n_obj, grid_n, per_obj * n_obj), hand, objs,
                    q0, oc, default_params(r0=0.010, schedule="linear"), steps)


def serving_stream(n_requests: int = 2000, rate_hz: float = 200.0, grid_sizes=(32, 64, 128, 256),
                   cand_range=(64, 4096), step_range=(100, 1000), seed_offset: int = 4) -> list:
    """A fixed Poisson stream of grasp-search request specs (objects are built lazily
    from each spec's seed).  Each spec: arrival time (s), hand kind, object kind,
    grid size, candidate count (log-uniform), step count, object seed."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    out = []
    lo, hi = math.log(cand_range[0]), math.log(cand_range[1])
    for i in range(n_requests):
        out.append({
            "id": i,
            "arrival_s": float(t[i]),
            "hand_kind": int(rng.choice([3, 4, 5])),
            "object_kind": str(rng.choice(["superquadric", "polyhedron"])),
            "grid_n": int(rng.choice(grid_sizes)),
            "B": int(round(math.exp(rng.uniform(lo, hi)))),
            "steps": int(rng.integers(step_range[0], step_range[1] + 1)),
            "object_seed": int(rng.integers(0, 2**62)),
            "cand_seed": int(rng.integers(0, 2**62)),
        })
    return out


def hand_points_per_link(kind: int) -> int:
    return 64 if kind == 3 else 256


def build_request(spec: dict, device="cpu", hand_cache=None):
    """Materialise one serving request: (hand, object, q0, params, steps)."""
    kind = spec["hand_kind"]
    if hand_cache is not None and kind in hand_cache:
        hand = hand_cache[kind]
    else:
        hand = make_hand(kind, hand_points_per_link(kind))
        if hand_cache is not None:
            hand_cache[kind] = hand
    orng = np.random.default_rng(spec["object_seed"])
    if spec["object_kind"] == "superquadric":
        obj = random_superquadric(orng, spec["grid_n"], device=device)
    else:
        obj = random_polyhedron(orng, spec["grid_n"], device=device)
    crng = np.random.default_rng(spec["cand_seed"])
    q0 = sample_candidates(crng, hand, spec["B"], obj["bound_radius"] + 0.06)
    return hand, obj, q0, default_params(r0=0.010, schedule="linear"), spec["steps"]
