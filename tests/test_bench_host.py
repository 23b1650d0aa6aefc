"""Host logic of bench.py's order-quality leg (no GPU): the schedule of launches
that covers the whole optimisation, the parameters each order and learning rate
runs with, the per-object torque scale, and the summary statistics, with a fake
binding standing in for the library."""

import os
import sys
import types

import numpy as np
import torch

import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


class _Event:
    def __init__(self, **_):
        pass

    def record(self):
        pass

    def elapsed_time(self, other):
        return 250.0


def _fake_fg(calls, B):
    fg = types.SimpleNamespace()
    fg.Hand = types.SimpleNamespace(from_synth=lambda h: types.SimpleNamespace(P=h["P"]))

    def optimize_step(hand, scene, q, prm, k, total, n, obj_of_cand=None, loss=None):
        calls.append(("opt", prm["gauss_seidel"], prm["lr"], k, total, n))
        loss.fill_(1.0 + prm["gauss_seidel"])

    def contact_measure(hand, scene, q, weights, tau, obj_of_cand=None):
        calls.append(("measure", tau, hand.P))
        return torch.full((q.shape[0],), 2e-4)          # 2 cm^2 (CA) or 200 cm^3 (IV)

    def grasp_epsilon(hand, scene, q, tau, mu, k, ts, dirs, obj_of_cand=None):
        calls.append(("eps", q.shape[0], ts, int(obj_of_cand[0])))
        n = q.shape[0]
        # the first half of each object's candidates in force closure
        e = torch.where(torch.arange(n) < n // 2, torch.tensor(0.1), torch.tensor(-0.2))
        return e, torch.full((n,), 7, dtype=torch.int32)

    fg.optimize_step = optimize_step
    fg.contact_measure = contact_measure
    fg.grasp_epsilon = grasp_epsilon
    return fg


def test_order_quality_schedule_and_summary(monkeypatch):
    import bench
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    w = synth.batched_superquadric_workload(n_obj=2, per_obj=6, grid_n=12)
    calls = []
    fg = _fake_fg(calls, w.B)
    hand = types.SimpleNamespace(P=w.hand["P"])
    out = bench.run_order_quality(fg, w, hand, None, torch.tensor(w.obj_of_cand), torch.tensor(w.q0), "cpu",
                                  [1e-3, 1e-6], steps_per_launch=30)
    opt = [c for c in calls if c[0] == "opt"]
    # 2 rates x 2 orders, each covering steps 0..w.steps-1 in launches of <= 30 steps
    assert len(opt) == 4 * -(-w.steps // 30)
    for lr in (1e-3, 1e-6):
        for gs in (0, 1):
            run = [c for c in opt if c[1] == gs and c[2] == lr]
            assert [c[3] for c in run] == list(range(0, w.steps, 30))
            assert sum(c[5] for c in run) == w.steps
            assert all(c[4] == w.steps for c in run)
    # one epsilon call per object, torque scaled by 1/rho of that object
    eps = [c for c in calls if c[0] == "eps"]
    assert len(eps) == 4 * len(w.objects)
    for c in eps[:len(w.objects)]:
        assert np.isclose(c[2], 1.0 / w.objects[c[3]]["bound_radius"])
    # contact area on the surface samples at 5 mm, intersection volume on the interior lattice at 0
    meas = [c for c in calls if c[0] == "measure"]
    assert meas[0][1] == 0.005 and meas[1][1] == 0.0 and meas[0][2] == w.hand["P"] and meas[1][2] != w.hand["P"]
    runs = [r for r in out["runs"] if "order" in r]
    assert [(r["lr"], r["order"]) for r in runs] == [(1e-3, "jacobi"), (1e-3, "gauss_seidel"),
                                                     (1e-6, "jacobi"), (1e-6, "gauss_seidel")]
    for r in runs:
        assert r["force_closure_frac"] == 0.5
        assert np.isclose(r["epsilon_median_of_force_closure"], 0.1)
        assert np.isclose(r["contact_area_cm2_mean"], 2.0)
        assert np.isclose(r["intersection_volume_cm3_mean"], 200.0)
        assert r["with_contact_frac"] == 1.0 and r["contacts_mean"] == 7.0
        assert r["optimise_s"] == 0.25
        assert r["loss_median"] == (1.0 if r["order"] == "jacobi" else 2.0)
    cmp_ = [r for r in out["runs"] if "gs_epsilon_above_jacobi_frac" in r]
    assert [r["gs_epsilon_above_jacobi_frac"] for r in cmp_] == [0.0, 0.0]


def test_reference_arm_line():
    """bench.py --impl reference times the FP64 oracle on the host and prints the
    contract's JSON line (same metric and unit as the GPU arm, the oracle as its
    cpu_baseline, no host-device bytes); ranks other than 0 print nothing."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "candidate-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    out1 = subprocess.run(cmd, capture_output=True, text=True, timeout=120, cwd=root,
                          env=dict(env, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1"))
    assert out1.returncode == 0 and out1.stdout.strip() == ""


def test_roofline_takes_the_slower_of_alu_and_hbm_time():
    """bench.roofline_of: the ALU time (the oracle's flop count at the measured FP32
    peak) against the DRAM time (the launch's measured traffic at the HBM bandwidth);
    the slower bounds the launch, and frac is measured against that bound's peak.  The
    three fractions of the ALU peak differ only by their flop basis."""
    import bench
    w = types.SimpleNamespace(B=1000, hand={"P": 100})
    peak = {"tflops": 50.0, "basis": "test", "sms": 10, "clocks": {"sm_mhz": 2000.0}}
    units = 1000 * 100
    flops = bench.FLOPS_PER_POINT_STEP * units
    kern_ms = 1000.0 * flops / 25e12                   # half the ALU peak
    prof = {"traffic": 1e6, "executed_fp32_flops_per_point_step": 500.0}
    r = bench.roofline_of(w, 1, kern_ms, peak, 1000.0, "test", prof)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert np.isclose(r["frac"], 0.5) and np.isclose(r["achieved"], 25.0) and r["peak"] == 50.0
    f = r["fractions"]
    assert np.isclose(f["oracle_count"]["frac"], 0.5)
    assert np.isclose(f["kernel_minimal"]["frac"], 0.5 * bench.KERNEL_MIN_FLOPS_PER_POINT_STEP / bench.FLOPS_PER_POINT_STEP)
    assert np.isclose(f["executed_fp32"]["frac"], 0.5 * 500.0 / bench.FLOPS_PER_POINT_STEP)
    assert np.isclose(r["alu_peak_derived_tflops"], 10 * 128 * 2 * 2000e6 / 1e12)
    # the same launch moving 1e12 bytes at 1,000 GB/s takes 1 s: DRAM-bound
    r = bench.roofline_of(w, 1, 1000.0, peak, 1000.0, "test", {"traffic": 1e12})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and np.isclose(r["frac"], 1.0)
    assert r["fractions"]["executed_fp32"] is None
    # without a traffic record the ALU bounds it
    assert bench.roofline_of(w, 1, kern_ms, peak, 1000.0, "test", None)["bound"] == "alu"


def test_profile_records_are_keyed_by_kernel_workload_and_sources(tmp_path, monkeypatch):
    """bench.load_profile returns a kernel's DRAM traffic only for the workload it was
    captured on and only while the kernel's sources hash to the recorded value."""
    import bench
    from paper_2306_08132_gb300.build import source_hash, FUSED_SOURCES
    cur = source_hash(FUSED_SOURCES)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# kernel workload hash bytes flops\n"
        "fused_step wl_a %s 123 456\nfused_step wl_b deadbeef0000 789 -\nfused_step wl_c %s 5 -\n" % (cur, cur))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_profile("fused_step", "wl_a") == {"traffic": 123.0, "source_hash": cur,
                                                        "executed_fp32_flops_per_point_step": 456.0}
    assert bench.load_profile("fused_step", "wl_b") is None          # stale sources
    assert bench.load_profile("fused_step", "wl_c") == {"traffic": 5.0, "source_hash": cur}
    assert bench.load_profile("fused_step", "wl_d") is None          # another workload
    assert bench.load_profile("gs_step", "wl_a") is None


def test_workload_partition_by_object():
    """bench.build_workload: rank k of N builds only the grids of its block of objects
    and keeps exactly their candidates; the blocks cover the workload."""
    import bench
    sizes = dict(n_obj=5, per_obj=2, grid_n=10, points_per_link=8)
    full, info = bench.build_workload("cpu", 0, 1, "superquadric8", **sizes)
    seen = []
    total = 0
    for r in range(3):
        w, part = bench.build_workload("cpu", r, 3, "superquadric8", **sizes)
        assert len(w.objects) == len(part["objects"]) and part["total_candidates"] == full.B
        np.testing.assert_array_equal(w.q0, full.q0[part["candidates"]])
        np.testing.assert_array_equal(part["objects"][w.obj_of_cand], full.obj_of_cand[part["candidates"]])
        for k, o in zip(part["objects"], w.objects):
            assert torch.equal(o["grid"], full.objects[k]["grid"])
        seen += part["candidates"].tolist()
        total += part["grid_bytes"]
    assert sorted(seen) == list(range(full.B)) and total == info["grid_bytes"]
    lazy, _ = bench.build_workload("cpu", 0, 1, "sweep256", lazy=True)
    assert lazy.B == 65536 and not any("grid" in o for o in lazy.objects)
