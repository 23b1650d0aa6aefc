"""Benchmark of the grasp-search step (candidate-steps per second).

Workload (default): the 256-object throughput sweep, 128 superquadrics and 128
convex polyhedra on 192^3 float32 SDF grids (7.1 GB), the 5-finger synthetic hand
(23 links, 5,888 points), 65,536 candidates (256 per object), paper constants
(alpha = 0.1, dt = 1 ms, lr = 1e-3), dilation 10 mm at step 0 of a 1,000-step
linear schedule.  One timed step = one fused forward + adjoint + update launch
over all candidates, starting from the initial candidates (q is reset by a device
copy inside the timed region, so every step sees the same contact state).  The
L2 is flushed (256 MiB write) between timed steps.  `--workload` selects the
8-superquadric batch (128^3, 4-finger hand, 8,192 candidates) or the 32 polyhedra
instead; the 8-superquadric batch is also measured beside the sweep as a
sub-record.

Lines: the fused path (value), the plain per-stage GPU form (plain), the same
step end to end through the library's host-buffer entry point (e2e), the
roofline of the fused kernel (ALU time at the measured FP32 peak against DRAM time
at the measured HBM bandwidth), sampled SM clocks, and the FP64 oracle on the
host cores (cpu_baseline).  `--impl reference` times the oracle alone on the same
workload.

Multi-GPU (`--gpus N` under torchrun): the workload's objects are split into N
contiguous blocks; each rank builds only its objects' grids and optimises only
their candidates, with no exchange in the step loop; the job time is the slowest
rank's, and one optimisation step's (q, loss) is gathered on rank 0 at the end.

Optional legs on the same candidates: --gs (Gauss-Seidel projection), --tstep T
(the T-step metric), --mesh (the objects as meshes with the Phong SDF; with --gs
also that combination), --quality (contact area and epsilon), --order-quality (the
grasps of a whole optimisation in the Jacobi and the Gauss-Seidel order, compared
by their quality metrics), --serving N and --serving-sweep (request latency
against offered load); --profile-kernel runs a few launches of the selected
kernel for ncu and exits.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic floating-point operations per point-step: the method as the FP64
# oracle computes it (forward pass + reverse mode, every branch evaluated), from
# the oracle's counting instantiation (oracle/flop_count.py); the same for the
# 4- and 5-finger hands.
FLOPS_PER_POINT_STEP = 2092
# The fused kernel's own minimal count for a point out of contact (forward once +
# leaky adjoint once, FMA = 2), reported beside it.
KERNEL_MIN_FLOPS_PER_POINT_STEP = 599
# The same count for the Gauss-Seidel form (oracle counting instantiation, this workload).
GS_FLOPS_PER_POINT_STEP = 2540
# The T-step form, by the number of simulation steps T (same counter, same workload).
TSTEP_FLOPS_PER_POINT_STEP = {1: 6228, 2: 13061, 4: 26729}
METRIC = "candidate-steps/sec fused fwd+bwd vs plain GPU form at 1e-3 grad tol; p50/p99 latency"
WORKLOADS = ("sweep256", "superquadric8", "polyhedra32")
# HBM copy bandwidth when the measured-peaks file is absent (the profiling recipe's fallback)
FALLBACK_HBM_GBS = 6800.0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def load_profile(kernel_tag: str, workload: str):
    """The committed ncu figures of one kernel on one workload (profiles/traffic.txt),
    if they were taken on the current kernel sources (matching source hash): DRAM
    bytes per launch and, where recorded, the FP32 operations the kernel executes per
    point-step (FADD, FMUL 1, FFMA 2, packed forms twice).  None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    from paper_2306_08132_gb300.build import source_hash, FUSED_SOURCES
    cur = source_hash(FUSED_SOURCES)
    for line in open(path):
        parts = line.split()
        if line.startswith("#") or len(parts) < 4:
            continue
        if parts[0] == kernel_tag and parts[1] == workload and parts[2] == cur:
            rec = {"traffic": float(parts[3]), "source_hash": cur}
            if len(parts) >= 5 and parts[4] != "-":
                rec["executed_fp32_flops_per_point_step"] = float(parts[4])
            return rec
    return None


def measured_hbm_gbs():
    """(HBM copy bandwidth in GB/s, its basis): the driver's measured-peaks file, else the
    profiling recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def build_workload(device, rank: int = 0, world: int = 1, kind: str = "sweep256", lazy: bool = False, **sizes):
    """Rank `rank`'s share of a benchmark workload and a description of the partition.

    Workloads: "sweep256" the 256 objects (192^3) with the 5-finger hand and 65,536
    candidates; "superquadric8" the 8 superquadrics (128^3) with the 4-finger hand and
    8,192 candidates; "polyhedra32" the 32 polyhedra (128^3) with the 5-finger hand and
    131,072 candidates (sizes adjustable for tests).  The objects are split into
    `world` contiguous blocks; rank k builds only the grids of block k and keeps the
    candidates of those objects (object indices renumbered within the block).  With
    lazy=True no grid is built (``synth.realize`` builds one when it is needed)."""
    import synth
    from paper_2306_08132_gb300 import shard
    if kind == "polyhedra32":
        full = synth.polyhedra_workload(device=device, build=False, **sizes)
    elif kind == "sweep256":
        full = synth.sweep_workload(device=device, build=False, **sizes)
    elif kind == "superquadric8":
        full = synth.batched_superquadric_workload(device=device, build=False, **sizes)
    else:
        raise ValueError("unknown workload %r" % kind)
    part = shard.shard_workload(len(full.objects), full.obj_of_cand, rank, world)
    objs = [full.objects[k] if lazy else synth.realize(full.objects[k], device) for k in part["objects"]]
    w = synth.Workload(full.name, full.hand, objs, full.q0[part["candidates"]], part["obj_of_cand"],
                       full.params, full.steps)
    grid_bytes = int(sum(o["grid"].numel() * o["grid"].element_size() for o in objs if "grid" in o))
    info = {"objects": part["objects"], "candidates": part["candidates"], "total_candidates": full.B,
            "total_objects": len(full.objects), "grid_bytes": grid_bytes}
    return w, info


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The slowest rank's time (the whole job is done when the last rank is)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device="cpu") -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_sample(w, n_objects: int = 2):
    """The FP64 oracle's set-up for the candidates of the workload's first n_objects
    objects (the sample the CPU legs time), on the host: (setup, q, object indices)."""
    import synth
    from oracle import fastgraspd_oracle as O
    objs = [synth.realize(o, "cpu") for o in w.objects[:n_objects]]
    keep = np.nonzero(np.asarray(w.obj_of_cand) < n_objects)[0]
    S = O.Setup(w.hand, objs, w.params)
    return S, w.q0[keep], np.asarray(w.obj_of_cand)[keep]


def oracle_rate(S, q, oc, budget_s: float, r: float, max_cands: int | None = None, offset: int = 0):
    """FP64 oracle on the host: candidate-steps/s over chunks of 8 candidates of the
    sample until the time budget (or max_cands) is used."""
    import torch
    from oracle import fastgraspd_oracle as O
    done, t0 = 0, time.perf_counter()
    B = len(q)
    order = np.random.default_rng(3).permutation(B)
    while time.perf_counter() - t0 < budget_s and (max_cands is None or done < max_cands):
        start = (offset + done) % B
        sel = order[start:start + 8]
        O.batch_loss_and_grad(S, q[sel], oc[sel], r, chunk=8)
        done += len(sel)
    dt = time.perf_counter() - t0
    return done / dt, done, dt, torch.get_num_threads()


def measure_fp32_peak(fg, device, gpu_index: int, seconds: float = 0.6):
    """FP32 fused multiply-add throughput of this GPU (the library's microbenchmark,
    scalar FFMA and packed f32x2 FMA, 8 independent chains per thread, 8 CTAs of 256
    threads per SM), timed with CUDA events, SM clocks sampled meanwhile.  The peak is
    the faster form's best launch."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    out = torch.empty(sms * 8 * 256, device=device)
    stream = torch.cuda.current_stream()
    res = {}
    sampler = ClockSampler(gpu_index)
    sampler.start()
    for packed in (False, True):
        fg.fp32_peak_launch(out, packed, 1000)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fg.fp32_peak_launch(out, packed, 20000)
        e1.record(stream)
        torch.cuda.synchronize()
        iters = max(1000, int(20000 * 150.0 / max(e0.elapsed_time(e1), 1e-3)))    # ~150 ms a launch
        best = 0.0
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            e0.record(stream)
            flops = fg.fp32_peak_launch(out, packed, iters)
            e1.record(stream)
            torch.cuda.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) / 1000.0) / 1e12)
        res["packed" if packed else "scalar"] = best
    clocks = sampler.stop()
    form = max(res, key=res.get)
    return {"tflops": res[form], "form": form, "scalar_tflops": res["scalar"], "packed_tflops": res["packed"],
            "sms": sms, "clocks": clocks,
            "basis": "FMA microbenchmark (fg_fp32_peak_launch): %d SMs x 8 CTAs x 256 threads, 8 chains each, "
                     "best of ~150 ms launches" % sms}


def run_serving(fg, n_requests: int, rates_hz, device, budget_bytes: int, steps_per_launch: int = 10):
    """Replays the first n_requests of the seeded Poisson request stream into a
    request queue in real time, once per arrival rate (the stream's arrival times
    scaled to the rate), and returns latency percentiles and throughput per rate."""
    import synth
    from synth.workloads import build_request
    base_rate = 200.0
    specs = synth.serving_stream(n_requests=n_requests, rate_hz=base_rate)
    cache = {}
    built = []
    for sp in specs:
        hand_d, obj, q0, params, steps = build_request(sp, device=device, hand_cache=cache)
        key = sp["hand_kind"]
        if ("h", key) not in cache:
            cache[("h", key)] = fg.Hand.from_synth(hand_d)
        built.append((cache[("h", key)], fg.Sdf.from_synth(obj), q0, params, steps, sp["arrival_s"]))
    cand_steps = sum(b[2].shape[0] * b[4] for b in built)
    out = []
    for rate in rates_hz:
        scale = base_rate / rate
        queue = fg.Queue(budget_bytes, steps_per_launch=steps_per_launch)
        ids, lat = [], []
        t0 = time.perf_counter()
        try:
            for hand, sdf, q0, params, steps, t_arr in built:
                while time.perf_counter() - t0 < t_arr * scale:
                    time.sleep(0.0005)
                ids.append(queue.submit(hand, sdf, q0, steps, params))
            for rid in ids:
                queue.wait(rid, 600000)
                lat.append(queue.result(rid)[2])
            makespan = time.perf_counter() - t0
            st = queue.stats()
        finally:
            queue.close()
        lat = np.array(lat)
        span = max(built[-1][5] * scale, 1e-9)
        offered = cand_steps / span
        served = cand_steps / makespan
        out.append({"requests": n_requests, "arrival_rate_hz": rate, "p50_s": float(np.percentile(lat, 50)),
                    "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()), "makespan_s": makespan,
                    "offered_candidate_steps_per_s": offered, "candidate_steps_per_s": served,
                    "rounds": st["rounds"], "steps_per_launch": steps_per_launch,
                    "mean_round_ms": 1000.0 * makespan / max(st["rounds"], 1),
                    "note": ("offered load exceeds capacity: latency includes queueing" if served < 0.9 * offered
                             else "offered load within capacity")})
    return out


def run_order_quality(fg, w, hand, scene, oc, q0, device, lrs, steps_per_launch: int = 10):
    """Jacobi against Gauss-Seidel projection, compared by the grasps they produce: the
    same initial candidates optimised over the workload's whole schedule (w.steps
    steps, dilation from r0 down to 0) in each order and at each learning rate of lrs
    (the paper's 1e-3 moves a candidate by decimetres per step in SI units, so smaller
    rates are swept beside it), then the quality metrics of the final grasps at the
    5 mm contact threshold: contact area (area-weighted surface samples), intersection
    volume (3 mm interior lattice, phi < 0), epsilon over 1,024 unit directions (8-edge
    cones, mu = 0.5, torque scaled by 1/rho of each object), contacts, and the loss of
    the last step."""
    import torch
    import synth as _synth
    areas = torch.tensor(w.hand["point_area"], device=device)
    ih = _synth.interior_hand(w.hand["kind"], 0.003)
    ihand = fg.Hand.from_synth(ih)
    vols = torch.tensor(ih["point_volume"], device=device)
    dirs = torch.tensor(_synth.unit_directions(1024), device=device)
    oc_np = np.asarray(w.obj_of_cand)
    groups = [torch.tensor(np.nonzero(oc_np == k)[0], device=device) for k in range(len(w.objects))]

    def med(x):
        return float(x.double().median())

    def mean(x):
        return float(x.double().mean())

    runs = []
    for lr in lrs:
        eps_of = {}
        for name, gs in (("jacobi", 0), ("gauss_seidel", 1)):
            prm = dict(w.params, gauss_seidel=gs, lr=lr)
            q = q0.clone()
            loss = torch.empty(w.B, device=device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k in range(0, w.steps, steps_per_launch):
                fg.optimize_step(hand, scene, q, prm, k, w.steps, min(steps_per_launch, w.steps - k),
                                 obj_of_cand=oc, loss=loss)
            e1.record()
            torch.cuda.synchronize()
            ca = fg.contact_measure(hand, scene, q, areas, 0.005, obj_of_cand=oc)
            iv = fg.contact_measure(ihand, scene, q, vols, 0.0, obj_of_cand=oc)
            eps = torch.empty(w.B, device=device)
            nc = torch.empty(w.B, device=device, dtype=torch.int32)
            for k, sel in enumerate(groups):
                e, n = fg.grasp_epsilon(hand, scene, q[sel].contiguous(), 0.005, 0.5, 8,
                                        1.0 / float(w.objects[k]["bound_radius"]), dirs,
                                        obj_of_cand=oc[sel].contiguous())
                eps[sel] = e
                nc[sel] = n
            torch.cuda.synchronize()
            eps_of[name] = eps
            touching = nc > 0
            runs.append({"lr": lr, "order": name, "optimise_s": e0.elapsed_time(e1) / 1000.0,
                         "loss_median": med(loss), "with_contact_frac": mean(touching),
                         "contacts_mean": mean(nc), "contact_area_cm2_mean": mean(ca * 1e4),
                         "intersection_volume_cm3_mean": mean(iv * 1e6),
                         "force_closure_frac": mean(eps > 0),
                         "epsilon_median_of_force_closure": med(eps[eps > 0]) if bool((eps > 0).any()) else None})
        runs.append({"lr": lr, "gs_epsilon_above_jacobi_frac": mean(eps_of["gauss_seidel"] > eps_of["jacobi"])})
    setup = ("%d candidates, %d steps (dilation %.0f mm -> 0), threshold 5 mm, 1,024 directions, 8-edge cones, "
             "mu 0.5, interior lattice 3 mm (%d samples)" % (w.B, w.steps, 1000.0 * w.params["r0"], ih["P"]))
    return {"setup": setup, "runs": runs}



def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores, on the same
    workload (each timed step a bounded sample of it: 16 candidates of its first two
    objects, one step each).  Under torchrun only rank 0 runs."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch
    from oracle import fastgraspd_oracle as O
    w, _ = build_workload("cpu", 0, 1, args.workload, lazy=True)
    S, qs, ocs = oracle_sample(w)
    r = O.dilation_radius(S.prm, 0, w.steps)
    per_step = 16
    for k in range(args.warmup):
        oracle_rate(S, qs, ocs, 0.0, r, max_cands=8, offset=8 * k)
    t0 = time.perf_counter()
    total = 0
    for k in range(args.steps):
        _, n, _, cores = oracle_rate(S, qs, ocs, 1e9, r, max_cands=per_step, offset=per_step * k)
        total += n
    dt = time.perf_counter() - t0
    value = total / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "candidate-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "candidates": w.B, "points_per_candidate": w.hand["P"],
                       "sample_per_step": "%d candidates x 1 step (FP64 oracle, host cores), drawn from the "
                                          "candidates of the workload's first two objects" % per_step},
            "cpu_baseline": {"value": value, "unit": "candidate-steps/s", "cores": torch.get_num_threads(),
                             "kind": "oracle", "sample": "%d candidates x %d steps" % (per_step, args.steps)},
            "e2e": {"value": value, "unit": "candidate-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))



def graphed(step_fn):
    """Capture one step (q reset + launches) in a CUDA graph; replaying it keeps host
    launch latency out of the per-step device time."""
    import torch
    for _ in range(2):
        step_fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step_fn()
    torch.cuda.synchronize()
    return g.replay


def prewarm(fn, seconds=0.5):
    import torch
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        fn()
        torch.cuda.synchronize()


def timed(step_fn, nsteps, warm, flush, world, pre=None, label="timed"):
    """Per-step device time (ms) with CUDA events on the launching stream; the L2 flush
    (and `pre`, e.g. a reset of q) run before each start event.  Barriers on both
    sides under torchrun.  The timed steps are an NVTX range named `label` (a
    profiler can select their launches with it)."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        if pre is not None:
            pre()
        step_fn()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    torch.cuda.nvtx.range_push(label)
    for i in range(nsteps):
        flush.fill_(i & 0xff)
        if pre is not None:
            pre()
        starts[i].record(stream)
        step_fn()
        ends[i].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    return ms


class Bound:
    """A workload bound to the library on one device."""

    def __init__(self, fg, w, device):
        import torch
        self.w = w
        self.hand = fg.Hand.from_synth(w.hand)
        self.sdfs = [fg.Sdf.from_synth(o) for o in w.objects]
        self.scene = fg.Scene(self.sdfs)
        self.oc = torch.tensor(w.obj_of_cand, device=device, dtype=torch.int32)
        self.q0 = torch.tensor(w.q0, device=device)
        self.q = self.q0.clone()
        self.loss = torch.empty(w.B, device=device)


def roofline_of(w, S_in, kern_ms, peak, hbm_gbs, hbm_basis, prof):
    """Roofline of one fused launch: the ALU time of the method's work at the measured
    FP32 peak against the DRAM time of the launch's measured traffic at the HBM
    bandwidth; the slower one bounds it.  Three fractions of the ALU peak, by the
    basis of the flop count."""
    units = w.B * w.hand["P"] * S_in
    kern_s = kern_ms / 1000.0
    P = peak["tflops"]
    flops = FLOPS_PER_POINT_STEP * units
    t_alu = flops / (P * 1e12)
    traffic = prof["traffic"] if prof else None
    t_hbm = traffic / (hbm_gbs * 1e9) if traffic else None
    bound = "alu" if t_hbm is None or t_alu >= t_hbm else "hbm"
    alu_tflops = flops / kern_s / 1e12
    fractions = {
        "oracle_count": {"flops_per_point_step": FLOPS_PER_POINT_STEP, "frac": alu_tflops / P,
                         "basis": "the method's work as the FP64 oracle computes it (oracle/flop_count.py: "
                                  "forward pass + reverse mode, both arms of every select)"},
        "kernel_minimal": {"flops_per_point_step": KERNEL_MIN_FLOPS_PER_POINT_STEP,
                           "frac": KERNEL_MIN_FLOPS_PER_POINT_STEP * units / kern_s / 1e12 / P,
                           "basis": "the fused kernel's own operation count for a point out of contact "
                                    "(forward once + leaky adjoint once, FMA = 2); contacts add work"},
        "executed_fp32": None,
    }
    if prof and "executed_fp32_flops_per_point_step" in prof:
        x = prof["executed_fp32_flops_per_point_step"]
        fractions["executed_fp32"] = {"flops_per_point_step": x, "frac": x * units / kern_s / 1e12 / P,
                                      "basis": "FP32 operations the kernel executes (ncu instruction counts of "
                                               "this workload: FADD, FMUL 1, FFMA 2, packed f32x2 forms twice)"}
    rec = {"bound": bound, "kernel_ms": kern_ms, "traffic": traffic,
           "alu_time_ms": 1000.0 * t_alu, "hbm_time_ms": None if t_hbm is None else 1000.0 * t_hbm,
           "flops_per_launch": flops, "flops_per_point_step": FLOPS_PER_POINT_STEP,
           "flops_basis": fractions["oracle_count"]["basis"], "fractions": fractions,
           "alu_peak_tflops": P, "alu_peak_basis": "of measured: " + peak["basis"],
           "alu_peak_derived_tflops": (peak["sms"] * 128 * 2 * peak["clocks"]["sm_mhz"] * 1e6 / 1e12
                                       if peak.get("clocks") and peak["clocks"].get("sm_mhz") else None),
           "hbm_peak_gbs": hbm_gbs, "hbm_basis": hbm_basis}
    if bound == "alu":
        rec.update({"achieved": alu_tflops, "peak": P, "unit": "TFLOP/s", "frac": alu_tflops / P})
    else:
        rec.update({"achieved": traffic / kern_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": traffic / kern_s / 1e9 / hbm_gbs})
    return rec


def measure_fused(fg, b, args, world, flush, peak, label_clocks=None):
    """The fused step on one bound workload: autotuned configuration, graphed timed steps,
    the per-stage form, the host-buffer end-to-end step and the kernel-only time for
    the roofline."""
    import torch
    w, S_in, K = b.w, args.inner_steps, b.w.steps

    def fused_step():
        b.q.copy_(b.q0)
        fg.optimize_step(b.hand, b.scene, b.q, w.params, 0, K, S_in, obj_of_cand=b.oc, loss=b.loss)

    best_cfg, cfg_ms = fg.autotune(b.hand, b.scene, b.q0, w.params, 0, K, S_in, obj_of_cand=b.oc, reps=3)
    cfgs = fg.fused_configs()
    if args.config is not None:
        best_cfg = args.config
        fg.fused_config_select(best_cfg)
    g = graphed(fused_step)
    prewarm(g)
    sampler = ClockSampler(label_clocks) if label_clocks is not None else None
    if sampler:
        sampler.start()
    t_wall = time.perf_counter()
    ms = timed(g, args.steps, args.warmup, flush, world, label="fused")
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop() if sampler else None
    out = {"ms": ms, "wall": wall, "clocks": clocks, "best_cfg": best_cfg, "cfg_ms": cfg_ms, "cfgs": cfgs}

    if not args.no_plain:
        ws = torch.empty(fg.plain_workspace_size(b.hand, w.B) + 256, dtype=torch.uint8, device=b.q.device)

        def plain_step():
            b.q.copy_(b.q0)
            fg.optimize_step_plain(b.hand, b.scene, b.q, w.params, 0, K, S_in, obj_of_cand=b.oc, loss=b.loss,
                                   workspace=ws)

        pms = timed(graphed(plain_step), max(3, args.steps // 2), 3, flush, world, label="plain")
        pstep = float(np.mean(pms))
        out["plain"] = {"value": w.B * S_in / (pstep / 1000.0), "ms_per_step": pstep,
                        "speedup_fused_over_plain": pstep / float(np.mean(ms)), "gpu_launches_per_step": 8 * S_in}
        del ws
    else:
        out["plain"] = None

    # end to end: pinned host q in, the step, q and loss back to pinned host memory,
    # every copy made by the library's host-buffer entry point
    hq0 = torch.tensor(w.q0).pin_memory()
    hq = torch.empty_like(hq0).pin_memory()
    hloss = torch.empty(w.B).pin_memory()

    def e2e_step():
        fg.optimize_step_host(b.hand, b.scene, hq0, b.q, w.params, 0, K, S_in, obj_of_cand=b.oc, loss=b.loss,
                              host_q_out=hq, host_loss=hloss)

    ems = timed(e2e_step, max(3, args.steps // 2), 3, flush, world, label="e2e")
    out["e2e_ms"] = float(np.mean(ems))
    out["e2e_bytes"] = (int(hq0.numel() * 4), int(hq.numel() * 4 + hloss.numel() * 4))

    def kernel_only():
        fg.optimize_step(b.hand, b.scene, b.q, w.params, 0, K, S_in, obj_of_cand=b.oc, loss=b.loss)

    def reset_q():
        b.q.copy_(b.q0)

    kms = timed(graphed(kernel_only), max(3, args.steps // 2), 3, flush, world, pre=reset_q, label="kernel")
    out["kern_ms"] = float(np.mean(kms))
    out["fused_step"] = fused_step
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fused", choices=["fused", "reference"])
    ap.add_argument("--inner-steps", type=int, default=1, help="optimisation steps per fused launch")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the 8-superquadric sub-record")
    ap.add_argument("--no-sub-legs", action="store_true",
                    help="in the 8-superquadric sub-record, time the fused and per-stage forms only")
    ap.add_argument("--profile-kernel", action="store_true",
                    help="set up the workload, run a few fused launches and exit (for ncu)")
    ap.add_argument("--config", type=int, default=None, help="fused configuration index (default: autotune)")
    ap.add_argument("--serving", type=int, default=500, help="requests in the serving (p50/p99) run; 0 skips it")
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--tstep", default="",
                    help="comma-separated T: also time the T-step metric (SDF re-queried for T steps) on this workload")
    ap.add_argument("--workload", default="sweep256", choices=WORKLOADS,
                    help="sweep256 (256 objects on 192^3, the default), superquadric8 or polyhedra32")
    ap.add_argument("--gs", action="store_true",
                    help="also time the Gauss-Seidel form (constraints projected in point order) on this workload")
    ap.add_argument("--quality", action="store_true",
                    help="also time the grasp-quality metrics (contact area, epsilon over 1,024 directions) "
                         "over the workload's candidates")
    ap.add_argument("--order-quality", action="store_true",
                    help="also optimise the candidates over the whole schedule in the Jacobi and the Gauss-Seidel "
                         "order and compare the quality metrics of the final grasps")
    ap.add_argument("--order-quality-lr", default="1e-3,1e-5,1e-6,1e-7",
                    help="learning rates of the --order-quality runs")
    ap.add_argument("--mesh", action="store_true",
                    help="also time the fused step on mesh objects (the superquadric8 workload's objects as "
                         "watertight meshes, queried through the BVH with the Phong SDF)")
    ap.add_argument("--mesh-res", default="24,48", help="latitude,longitude divisions of the superquadric meshes")
    ap.add_argument("--serving-sweep", default="",
                    help="comma-separated arrival rates (req/s) for a latency-vs-load sweep of the same stream")
    ap.add_argument("--objects", type=int, default=None,
                    help="a smaller copy of the workload with this many objects and the same candidates per object "
                         "(for profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from __graft_entry__ import build
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    import paper_2306_08132_gb300 as fg
    from paper_2306_08132_gb300 import shard

    w, part = build_workload(dev, rank, world, args.workload, **workload_sizes(args))
    b = Bound(fg, w, dev)
    K, S_in = w.steps, args.inner_steps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    if args.profile_kernel:
        if args.config is not None:
            fg.fused_config_select(args.config)
        if args.tstep:                       # the T-step kernel instead, T = the first value
            prm = dict(w.params, sim_steps=int(args.tstep.split(",")[0]))
        elif args.gs:                        # the Gauss-Seidel kernel
            prm = dict(w.params, gauss_seidel=1)
        else:
            prm = w.params
        if args.mesh:                        # the fused kernel on the superquadrics as meshes
            scene = fg.Scene([fg.Sdf.from_synth(m) for m in superquadric_meshes(w, args.mesh_res)])
        else:
            scene = b.scene
        for _ in range(3 if (args.tstep or args.gs or args.mesh or args.quality) else 5):
            if args.quality:                 # the epsilon kernel over 1,024 directions
                import synth as _synth
                dirs = torch.tensor(_synth.unit_directions(1024), device=dev)
                fg.grasp_epsilon(b.hand, scene, b.q0, 0.005, 0.5, 8, 1.0 / 0.08, dirs, obj_of_cand=b.oc)
            else:
                b.q.copy_(b.q0)
                fg.optimize_step(b.hand, scene, b.q, prm, 0, K, S_in, obj_of_cand=b.oc, loss=b.loss)
        torch.cuda.synchronize()
        return

    peak = measure_fp32_peak(fg, dev, local)
    hbm_gbs, hbm_basis = measured_hbm_gbs()
    res = measure_fused(fg, b, args, world, flush, peak, label_clocks=local)
    ms = res["ms"]
    ms_step = max_over_ranks(float(np.mean(ms)), world, dev)
    cand_steps = sum_over_ranks(w.B * S_in, world, dev)
    value = cand_steps / (ms_step / 1000.0)
    e2e_ms = max_over_ranks(res["e2e_ms"], world, dev)
    e2e = {"value": cand_steps / (e2e_ms / 1000.0), "unit": "candidate-steps/s",
           "h2d_bytes_per_step": res["e2e_bytes"][0], "d2h_bytes_per_step": res["e2e_bytes"][1],
           "entry_point": "fg_optimize_step_host (pinned host q in; q and loss out)"}
    roofline = roofline_of(w, S_in, res["kern_ms"], peak, hbm_gbs, hbm_basis, load_profile("fused_step", w.name))
    cfgs, best_cfg = res["cfgs"], res["best_cfg"]

    sub = None
    if not args.no_sub and args.workload != "superquadric8" and world == 1:
        w2, _ = build_workload(dev, 0, 1, "superquadric8")
        b2 = Bound(fg, w2, dev)
        r2 = measure_fused(fg, b2, args, 1, flush, peak)
        m2 = float(np.mean(r2["ms"]))
        sub = {"workload": w2.name, "value": w2.B * S_in / (m2 / 1000.0), "unit": "candidate-steps/s",
               "ms_per_step": m2, "plain": r2["plain"],
               "e2e": {"value": w2.B * S_in / (r2["e2e_ms"] / 1000.0), "unit": "candidate-steps/s"},
               "roofline": roofline_of(w2, S_in, r2["kern_ms"], peak, hbm_gbs, hbm_basis,
                                       load_profile("fused_step", w2.name)),
               "fused_config": "%dw/%d/%dp" % r2["cfgs"][r2["best_cfg"]]}
        if not args.no_sub_legs:
            # the other forms of the step on this batch: Gauss-Seidel, T-step (T = 1), mesh objects, quality
            sub_args = argparse.Namespace(**dict(vars(args), tstep="1", gs=True, quality=True, mesh=True,
                                                 order_quality=False, serving=0))
            sub.update(run_legs(fg, sub_args, b2, dev, 1, flush, w2.B * S_in, peak))
            for k in ("order_quality", "serving", "serving_sweep"):
                sub.pop(k, None)
        del b2
        fg.autotune(b.hand, b.scene, b.q0, w.params, 0, K, S_in, obj_of_cand=b.oc, reps=3)   # back to the main workload

    legs = run_legs(fg, args, b, dev, world, flush, cand_steps, peak)
    grid_bytes = int(sum_over_ranks(part["grid_bytes"], world, dev))

    # multi-GPU: one optimisation step of every rank's candidates, gathered on rank 0
    gathered = None
    if world > 1:
        b.q.copy_(b.q0)
        fg.optimize_step(b.hand, b.scene, b.q, w.params, 0, K, 1, obj_of_cand=b.oc, loss=b.loss)
        torch.cuda.synchronize()
        Q = shard.gather_rows(b.q.cpu().numpy(), part["candidates"], part["total_candidates"])
        L = shard.gather_rows(b.loss.cpu().numpy(), part["candidates"], part["total_candidates"])
        if rank == 0:
            gathered = {"candidates": int(Q.shape[0]), "finite": bool(np.isfinite(Q).all() and np.isfinite(L).all())}

    if rank == 0:
        from oracle import fastgraspd_oracle as O   # the cpu_baseline leg only
        S, qs, ocs = oracle_sample(w)
        r0 = O.dilation_radius(S.prm, 0, K)
        rate, n, dt, cores = oracle_rate(S, qs, ocs, args.cpu_budget, r0)
        cpu = {"value": rate, "unit": "candidate-steps/s", "cores": cores, "kind": "oracle",
               "sample": "%d candidates x 1 step of the workload's first two objects in %.1f s (FP64, torch CPU)"
                         % (n, dt)}
        if args.cpu_budget > 0:
            threads = torch.get_num_threads()
            torch.set_num_threads(1)
            try:
                r1, n1, dt1, _ = oracle_rate(S, qs, ocs, args.cpu_budget / 3.0, r0)
            finally:
                torch.set_num_threads(threads)
            cpu["value_1_thread"] = r1
            cpu["sample_1_thread"] = "%d candidates x 1 step in %.1f s on one thread" % (n1, dt1)
        line = {"metric": METRIC, "value": value, "unit": "candidate-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": w.name, "objects": part["total_objects"],
                           "grid": "%d^3 f32" % w.objects[0]["grid"].shape[0],
                           "hand": "%d-finger, %d links, %d points" % (w.hand["kind"], w.hand["L"], w.hand["P"]),
                           "candidates": int(cand_steps // S_in), "inner_steps_per_launch": S_in,
                           "state": "q reset to the initial candidates each step",
                           "l2": "flushed between timed steps (256 MiB write)", "parallelism": "dp%d" % world,
                           "partition": ("objects in %d contiguous blocks, one per rank; rank 0 holds %d objects "
                                         "(%d grid bytes) and %d candidates" % (world, len(part["objects"]),
                                                                                part["grid_bytes"], w.B)),
                           "grid_bytes": grid_bytes,
                           "fused_config": {"warps_per_candidate": cfgs[best_cfg][0],
                                            "min_ctas_per_sm": cfgs[best_cfg][1],
                                            "points_per_thread": cfgs[best_cfg][2],
                                            "autotune_ms": {"%dw/%d/%dp" % c: round(t, 4)
                                                            for c, t in zip(cfgs, res["cfg_ms"])}}},
                "plain": res["plain"], "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
                "fp32_peak": peak, "superquadric8": sub,
                "latency": None if legs["serving"] is None else {"p50_s": legs["serving"]["p50_s"],
                                                                 "p99_s": legs["serving"]["p99_s"]},
                **legs, "gathered": gathered,
                "gpu_launches": args.steps, "clocks": res["clocks"],
                "wall_s_timed_region": res["wall"],
                "per_step_ms": {"min": float(np.min(ms)), "median": float(np.median(ms)), "max": float(np.max(ms))}}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def workload_sizes(args) -> dict:
    """Size arguments of a smaller copy of the workload (--objects), the same candidates per object."""
    if args.objects is None:
        return {}
    if args.workload == "sweep256":
        return {"n_obj": args.objects, "total_cand": 256 * args.objects}
    return {"n_obj": args.objects}


def superquadric_meshes(w, mesh_res):
    """The workload's superquadrics as watertight latitude/longitude meshes (exponents
    held to [0.5, 1.5]: sharper ones fold the pole triangles)."""
    from synth import meshes as SM
    n_lat, n_lon = [int(x) for x in mesh_res.split(",")]
    out = []
    for o in w.objects:
        if o["kind"] != "superquadric":
            raise ValueError("the mesh leg needs superquadric objects (--workload superquadric8)")
        pr = o["params"]
        e1, e2 = [float(np.clip(pr[k], 0.5, 1.5)) for k in ("eps1", "eps2")]
        out.append(SM.superquadric_mesh(pr["semi_axes"], e1, e2, n_lat, n_lon))
    return out


def run_legs(fg, args, b, dev, world, flush, cand_steps, peak=None):
    """The optional legs on the bound workload (each None unless asked for)."""
    import torch
    w, K, S_in = b.w, b.w.steps, args.inner_steps
    out = {"tstep": None, "gauss_seidel": None, "mesh": None, "quality": None, "order_quality": None,
           "serving": None, "serving_sweep": None}
    units = w.B * w.hand["P"] * S_in

    def step_with(prm, scene=None):
        def f():
            b.q.copy_(b.q0)
            fg.optimize_step(b.hand, scene or b.scene, b.q, prm, 0, K, S_in, obj_of_cand=b.oc, loss=b.loss)
        return f

    if args.tstep:
        out["tstep"] = []
        for T in [int(x) for x in args.tstep.split(",") if x.strip()]:
            tms = timed(graphed(step_with(dict(w.params, sim_steps=T))), max(3, args.steps // 4), 3, flush, world)
            t_ms = max_over_ranks(float(np.mean(tms)), world, dev)
            rec = {"T": T, "ms_per_step": t_ms, "value": cand_steps / (t_ms / 1000.0),
                   "unit": "candidate-steps/s", "sdf_queries_per_point_step": 2 * 7 * T}
            if T in TSTEP_FLOPS_PER_POINT_STEP:
                rec["flops_per_point_step"] = TSTEP_FLOPS_PER_POINT_STEP[T]
                rec["achieved_tflops"] = TSTEP_FLOPS_PER_POINT_STEP[T] * units / (t_ms / 1e3) / 1e12
            out["tstep"].append(rec)

    if args.gs:
        gms = timed(graphed(step_with(dict(w.params, gauss_seidel=1))), max(3, args.steps // 4), 3, flush, world)
        g_ms = max_over_ranks(float(np.mean(gms)), world, dev)
        out["gauss_seidel"] = {"ms_per_step": g_ms, "value": cand_steps / (g_ms / 1000.0),
                               "unit": "candidate-steps/s", "flops_per_point_step": GS_FLOPS_PER_POINT_STEP,
                               "achieved_tflops": GS_FLOPS_PER_POINT_STEP * units / (g_ms / 1000.0) / 1e12}

    if args.quality:
        import synth as _synth
        areas = torch.tensor(w.hand["point_area"], device=dev)
        dirs = torch.tensor(_synth.unit_directions(1024), device=dev)
        qeps = torch.empty(w.B, device=dev)

        def ca_step():
            fg.contact_measure(b.hand, b.scene, b.q0, areas, 0.005, obj_of_cand=b.oc)

        def eps_step():
            e, _ = fg.grasp_epsilon(b.hand, b.scene, b.q0, 0.005, 0.5, 8, 1.0 / 0.08, dirs, obj_of_cand=b.oc)
            qeps.copy_(e)

        cms = timed(ca_step, max(3, args.steps // 4), 3, flush, world)
        ems_ = timed(eps_step, max(3, args.steps // 4), 3, flush, world)
        _, nc = fg.grasp_epsilon(b.hand, b.scene, b.q0, 0.005, 0.5, 8, 1.0 / 0.08, dirs, obj_of_cand=b.oc)
        ncm = float(nc.float().mean())
        out["quality"] = {"contact_area_ms": float(np.mean(cms)), "epsilon_ms": float(np.mean(ems_)),
                          "candidates": w.B, "threshold_m": 0.005, "directions": 1024, "cone_edges": 8,
                          "mean_contacts": ncm,
                          "epsilon_direction_contact_pairs_per_s": 1024 * ncm * w.B / (float(np.mean(ems_)) / 1e3)}

    if args.mesh:
        mobjs = superquadric_meshes(w, args.mesh_res)
        mscene = fg.Scene([fg.Sdf.from_synth(m) for m in mobjs])
        # the mesh kernels have their own best configuration (latency-bound searches
        # favour more warps per SM): tune on this scene, put the main one back after
        main_cfg = fg.fused_config_current()
        mcfg, mcfg_ms = fg.autotune(b.hand, mscene, b.q0, w.params, 0, K, S_in, obj_of_cand=b.oc, reps=2)
        mms = timed(graphed(step_with(w.params, mscene)), max(3, args.steps // 4), 3, flush, world)
        m_ms = max_over_ranks(float(np.mean(mms)), world, dev)
        cfgs = fg.fused_configs()
        out["mesh"] = {"ms_per_step": m_ms, "value": cand_steps / (m_ms / 1000.0), "unit": "candidate-steps/s",
                       "objects": "%d superquadric meshes, %d faces each, Phong SDF" % (len(mobjs),
                                                                                         len(mobjs[0]["faces"])),
                       "fused_config": "%dw/%d/%dp" % cfgs[mcfg],
                       "autotune_ms": {"%dw/%d/%dp" % c: round(t, 4) for c, t in zip(cfgs, mcfg_ms)},
                       "roofline": None}
        mprof = load_profile("fused_step_mesh", w.name)
        if peak is not None and mprof and "executed_fp32_flops_per_point_step" in mprof:
            # no operation count of the method exists for a BVH / local search (its work depends
            # on the geometry): the FP32 operations the kernel executes, from ncu, per point-step
            x = mprof["executed_fp32_flops_per_point_step"]
            ach = x * units / (m_ms / 1e3) / 1e12
            out["mesh"]["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak["tflops"], "unit": "TFLOP/s",
                                       "frac": ach / peak["tflops"], "flops_per_point_step": x,
                                       "basis": "executed FP32 operations per point-step (FADD, FMUL 1, FFMA 2) "
                                                "from ncu on this launch, the mesh search included; of measured "
                                                "FP32 peak",
                                       "traffic": mprof["traffic"]}
        fg.fused_config_select(main_cfg)
        if args.gs:                          # the paper's combination: Phong SDF of a mesh, Gauss-Seidel
            gms2 = timed(graphed(step_with(dict(w.params, gauss_seidel=1), mscene)), max(3, args.steps // 4), 3,
                         flush, world)
            mg_ms = max_over_ranks(float(np.mean(gms2)), world, dev)
            out["mesh"]["gauss_seidel"] = {"ms_per_step": mg_ms, "value": cand_steps / (mg_ms / 1000.0),
                                           "unit": "candidate-steps/s"}

    if args.order_quality:
        out["order_quality"] = run_order_quality(fg, w, b.hand, b.scene, b.oc, b.q0, dev,
                                                 [float(x) for x in args.order_quality_lr.split(",")])

    if args.serving > 0:
        free, _ = torch.cuda.mem_get_info()
        rates = [args.serving_rate] + [float(x) for x in args.serving_sweep.split(",") if x.strip()]
        runs = run_serving(fg, args.serving, rates, dev, int(0.5 * free))
        out["serving"], out["serving_sweep"] = runs[0], (runs[1:] or None)
    return out


if __name__ == "__main__":
    main()
