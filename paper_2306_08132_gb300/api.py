"""Python binding of libfastgraspd with the C ABI's names.

Argument marshalling only: every function checks tensor device, dtype, shape and
contiguity, passes raw pointers and torch's current CUDA stream to the library,
and returns the output tensors.  All arithmetic runs in the library's kernels.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check, FG_NUM_SIMS

_F32 = torch.float32


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t: torch.Tensor | None, name: str, dtype=_F32, shape=None) -> C.c_void_p | None:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return C.c_void_p(t.data_ptr())


def make_params(d: dict) -> _lib.Params:
    sched = d.get("schedule", "fixed")
    if isinstance(sched, str):
        sched = {"fixed": 0, "linear": 1}[sched]
    return _lib.Params(float(d["alpha_leak"]), float(d["dt"]), float(d["v_test"]), float(d["mu"]),
                       float(d["lr"]), float(d["r0"]), float(d["w_range"]), float(d["w_limit"]),
                       float(d["w_pen"]), int(sched), int(d.get("sim_steps", 0)),
                       int(d.get("gauss_seidel", 0)))


class Hand:
    """fg_hand: link tree, joint limits and link-local surface points."""

    def __init__(self, parent, T_fix, axis, q_low, q_up, pts_local, link_of_point):
        lib = _lib.load()
        self._keep = [np.ascontiguousarray(parent, dtype=np.int32),
                      np.ascontiguousarray(np.asarray(T_fix, dtype=np.float32).reshape(-1, 12)),
                      np.ascontiguousarray(np.asarray(axis, dtype=np.float32).reshape(-1, 3)),
                      np.ascontiguousarray(q_low, dtype=np.float32),
                      np.ascontiguousarray(q_up, dtype=np.float32),
                      np.ascontiguousarray(np.asarray(pts_local, dtype=np.float32).reshape(-1, 3)),
                      np.ascontiguousarray(link_of_point, dtype=np.int32)]
        par, tf, ax, lo, up, pts, lop = self._keep
        ptr = lambda a, t: a.ctypes.data_as(C.POINTER(t))
        desc = _lib.HandDesc(len(par), len(lop), ptr(par, C.c_int), ptr(tf, C.c_float), ptr(ax, C.c_float),
                             ptr(lo, C.c_float), ptr(up, C.c_float), ptr(pts, C.c_float), ptr(lop, C.c_int))
        h = C.c_void_p()
        check(lib.fg_hand_create(C.byref(desc), C.byref(h)), "fg_hand_create")
        self.handle = h
        vals = [C.c_int() for _ in range(4)]
        check(lib.fg_hand_info(h, *[C.byref(v) for v in vals]), "fg_hand_info")
        self.L, self.J, self.D, self.P = [v.value for v in vals]

    @classmethod
    def from_synth(cls, h: dict) -> "Hand":
        return cls(h["parent"], h["T_fix"], h["axis"], h["q_low"], h["q_up"], h["pts_local"], h["link_of_point"])

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib._lib is not None:
            _lib._lib.fg_hand_destroy(self.handle)
            self.handle = None


class Sdf:
    """fg_sdf: a voxel SDF grid [nz, ny, nx] (x fastest) with the object's mass
    properties, or (``Sdf.from_mesh``) a watertight triangle mesh queried directly."""

    PHONG_ALPHA = 0.75

    def __init__(self, grid: torch.Tensor | None, origin=None, pitch: float = 0.0, mass: float = 1.0,
                 inertia: float = 1.0, _handle=None):
        if _handle is not None:
            self.handle = _handle
            self.dims = None
            return
        lib = _lib.load()
        g = grid.detach().to(_F32).contiguous()
        nz, ny, nx = g.shape
        org = (C.c_float * 3)(*[float(v) for v in origin])
        h = C.c_void_p()
        check(lib.fg_sdf_create(C.c_void_p(g.data_ptr()), nx, ny, nz, org, float(pitch), float(mass),
                                float(inertia), C.byref(h)), "fg_sdf_create")
        self.handle = h
        self.dims = (nx, ny, nz)

    @classmethod
    def from_mesh(cls, vertices, faces, mass: float, inertia: float, phong_alpha: float = PHONG_ALPHA) -> "Sdf":
        """fg_sdf_create_mesh: vertices [V,3], faces [F,3] (counter-clockwise about the outward normal)."""
        lib = _lib.load()
        V = np.ascontiguousarray(np.asarray(vertices, dtype=np.float32))
        F = np.ascontiguousarray(np.asarray(faces, dtype=np.int32))
        if V.ndim != 2 or V.shape[1] != 3 or F.ndim != 2 or F.shape[1] != 3:
            raise ValueError("vertices and faces must be [n, 3]")
        h = C.c_void_p()
        check(lib.fg_sdf_create_mesh(V.ctypes.data_as(C.POINTER(C.c_float)), V.shape[0],
                                     F.ctypes.data_as(C.POINTER(C.c_int)), F.shape[0], float(phong_alpha),
                                     float(mass), float(inertia), C.byref(h)), "fg_sdf_create_mesh")
        return cls(None, _handle=h)

    @staticmethod
    def describe_mesh(vertices, faces) -> dict:
        """fg_mesh_describe (host only): how much of a mesh the certified local search covers."""
        lib = _lib.load()
        V = np.ascontiguousarray(np.asarray(vertices, dtype=np.float32))
        F = np.ascontiguousarray(np.asarray(faces, dtype=np.int32))
        if V.ndim != 2 or V.shape[1] != 3 or F.ndim != 2 or F.shape[1] != 3:
            raise ValueError("vertices and faces must be [n, 3]")
        out = (C.c_int * 6)()
        check(lib.fg_mesh_describe(V.ctypes.data_as(C.POINTER(C.c_float)), V.shape[0],
                                   F.ctypes.data_as(C.POINTER(C.c_int)), F.shape[0], out), "fg_mesh_describe")
        keys = ("faces", "hull_faces", "fan_vertices", "bvh_nodes", "bvh_depth", "start_nodes")
        return dict(zip(keys, [int(x) for x in out]))

    @classmethod
    def from_synth(cls, o: dict) -> "Sdf":
        if "faces" in o:
            return cls.from_mesh(o["vertices"], o["faces"], o["mass"], o["inertia"])
        return cls(o["grid"], o["origin"], o["pitch"], o["mass"], o["inertia"])

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib._lib is not None:
            _lib._lib.fg_sdf_destroy(self.handle)
            self.handle = None


class Scene:
    """fg_scene: ordered table of objects, indexed by obj_of_cand."""

    def __init__(self, sdfs):
        lib = _lib.load()
        self.sdfs = list(sdfs)
        arr = (C.c_void_p * len(self.sdfs))(*[s.handle.value for s in self.sdfs])
        h = C.c_void_p()
        check(lib.fg_scene_create(arr, len(self.sdfs), C.byref(h)), "fg_scene_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib._lib is not None:
            _lib._lib.fg_scene_destroy(self.handle)
            self.handle = None


def fk(hand: Hand, q: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    if out is None:
        out = torch.empty(3, B * hand.P, device=q.device, dtype=_F32)
    check(_lib.load().fg_fk(hand.handle, _dptr(q, "q"), B, _dptr(out, "pts", shape=(3, B * hand.P)), _stream()),
          "fg_fk")
    return out


def sdf_query(sdf: Sdf, pts: torch.Tensor, r_dil: float, want_grad: bool = True):
    n = pts.shape[1]
    _dptr(pts, "pts", shape=(3, n))
    phi = torch.empty(n, device=pts.device, dtype=_F32)
    grad = torch.empty(3, n, device=pts.device, dtype=_F32) if want_grad else None
    check(_lib.load().fg_sdf_query(sdf.handle, _dptr(pts, "pts"), n, float(r_dil), _dptr(phi, "phi"),
                                   _dptr(grad, "grad"), _stream()), "fg_sdf_query")
    return phi, grad


def _oc(obj_of_cand, B):
    if obj_of_cand is None:
        return None
    return _dptr(obj_of_cand, "obj_of_cand", dtype=torch.int32, shape=(B,))


def contact_wrench(hand: Hand, scene: Scene, q: torch.Tensor, params: dict, r_dil: float,
                   obj_of_cand: torch.Tensor | None = None, want_bits: bool = False):
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    dev = q.device
    wrench = torch.empty(B, FG_NUM_SIMS, 6, device=dev, dtype=_F32)
    ncontact = torch.empty(B, FG_NUM_SIMS, device=dev, dtype=torch.int32)
    nwords = (hand.P + 31) // 32
    bits = torch.empty(B, FG_NUM_SIMS, nwords, device=dev, dtype=torch.int32) if want_bits else None
    prm = make_params(params)
    check(_lib.load().fg_contact_wrench(hand.handle, scene.handle, _oc(obj_of_cand, B), _dptr(q, "q"), B,
                                        C.byref(prm), float(r_dil), _dptr(wrench, "wrench"),
                                        _dptr(ncontact, "ncontact", dtype=torch.int32),
                                        _dptr(bits, "bits", dtype=torch.int32), _stream()), "fg_contact_wrench")
    return wrench, ncontact, bits


def loss_and_grad(hand: Hand, scene: Scene, q: torch.Tensor, params: dict, r_dil: float,
                  obj_of_cand: torch.Tensor | None = None, want_grad: bool = True):
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    loss = torch.empty(B, device=q.device, dtype=_F32)
    grad = torch.empty(B, hand.D, device=q.device, dtype=_F32) if want_grad else None
    prm = make_params(params)
    check(_lib.load().fg_loss_and_grad(hand.handle, scene.handle, _oc(obj_of_cand, B), _dptr(q, "q"), B,
                                       C.byref(prm), float(r_dil), _dptr(loss, "loss"), _dptr(grad, "grad"),
                                       _stream()), "fg_loss_and_grad")
    return loss, grad


def optimize_step(hand: Hand, scene: Scene, q: torch.Tensor, params: dict, step: int, total_steps: int,
                  nsteps: int = 1, obj_of_cand: torch.Tensor | None = None, loss: torch.Tensor | None = None):
    """In-place gradient descent on q for nsteps (fused persistent kernel); returns the loss tensor."""
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    if loss is None:
        loss = torch.empty(B, device=q.device, dtype=_F32)
    prm = make_params(params)
    check(_lib.load().fg_optimize_step(hand.handle, scene.handle, _oc(obj_of_cand, B), _dptr(q, "q"), B,
                                       C.byref(prm), int(step), int(total_steps), int(nsteps),
                                       _dptr(loss, "loss", shape=(B,)), _stream()), "fg_optimize_step")
    return loss


def contact_measure(hand: Hand, scene: Scene, q: torch.Tensor, weights: torch.Tensor, tau: float,
                    obj_of_cand: torch.Tensor | None = None) -> torch.Tensor:
    """fg_contact_measure: per candidate, the sum of weights[i] over the points with phi < tau
    (contact area with area weights; intersection volume with interior samples and tau = 0)."""
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    _dptr(weights, "weights", shape=(hand.P,))
    out = torch.empty(B, device=q.device, dtype=_F32)
    check(_lib.load().fg_contact_measure(hand.handle, scene.handle, _oc(obj_of_cand, B), _dptr(q, "q"), B,
                                         _dptr(weights, "weights"), float(tau), _dptr(out, "out"), _stream()),
          "fg_contact_measure")
    return out


def grasp_epsilon(hand: Hand, scene: Scene, q: torch.Tensor, tau: float, mu: float, cone_edges: int,
                  torque_scale: float, dirs: torch.Tensor, obj_of_cand: torch.Tensor | None = None):
    """fg_grasp_epsilon: (eps [B], n_contacts [B] int32) over the unit directions dirs [K, 6]."""
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    K = dirs.shape[0]
    _dptr(dirs, "dirs", shape=(K, 6))
    eps = torch.empty(B, device=q.device, dtype=_F32)
    nc = torch.empty(B, device=q.device, dtype=torch.int32)
    check(_lib.load().fg_grasp_epsilon(hand.handle, scene.handle, _oc(obj_of_cand, B), _dptr(q, "q"), B,
                                       float(tau), float(mu), int(cone_edges), float(torque_scale),
                                       _dptr(dirs, "dirs"), K, _dptr(eps, "eps"),
                                       _dptr(nc, "n_contacts", dtype=torch.int32), _stream()), "fg_grasp_epsilon")
    return eps, nc


def plain_workspace_size(hand: Hand, B: int) -> int:
    n = C.c_size_t()
    check(_lib.load().fg_plain_workspace_size(hand.handle, B, C.byref(n)), "fg_plain_workspace_size")
    return n.value


def optimize_step_plain(hand: Hand, scene: Scene, q: torch.Tensor, params: dict, step: int, total_steps: int,
                        nsteps: int = 1, obj_of_cand: torch.Tensor | None = None,
                        loss: torch.Tensor | None = None, workspace: torch.Tensor | None = None):
    """The same step through the plain one-kernel-per-stage form (workspace in device memory)."""
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    need = plain_workspace_size(hand, B)
    if workspace is None:
        workspace = torch.empty(need + 256, device=q.device, dtype=torch.uint8)
    base = workspace.data_ptr()
    aligned = (base + 255) // 256 * 256
    avail = workspace.numel() - (aligned - base)
    if loss is None:
        loss = torch.empty(B, device=q.device, dtype=_F32)
    prm = make_params(params)
    check(_lib.load().fg_optimize_step_plain(hand.handle, scene.handle, _oc(obj_of_cand, B), _dptr(q, "q"), B,
                                             C.byref(prm), int(step), int(total_steps), int(nsteps),
                                             _dptr(loss, "loss", shape=(B,)), C.c_void_p(aligned), avail,
                                             _stream()), "fg_optimize_step_plain")
    return loss


def fused_configs() -> list[tuple[int, int, int]]:
    """Compiled fused-kernel configurations: (warps per candidate, min CTAs per SM,
    points per thread in the adjoint sweep)."""
    lib = _lib.load()
    n = C.c_int()
    check(lib.fg_fused_config_count(C.byref(n)), "fg_fused_config_count")
    out = []
    for i in range(n.value):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        check(lib.fg_fused_config_info(i, C.byref(a), C.byref(b), C.byref(c)), "fg_fused_config_info")
        out.append((a.value, b.value, c.value))
    return out


def fused_config_select(index: int) -> None:
    check(_lib.load().fg_fused_config_select(int(index)), "fg_fused_config_select")


def fused_config_current() -> int:
    i = C.c_int()
    check(_lib.load().fg_fused_config_current(C.byref(i)), "fg_fused_config_current")
    return i.value


def autotune(hand: Hand, scene: Scene, q: torch.Tensor, params: dict, step: int = 0, total_steps: int = 1,
             nsteps: int = 1, obj_of_cand: torch.Tensor | None = None, reps: int = 3):
    """Time every fused configuration on this workload and select the fastest.
    Returns (best index, list of mean milliseconds per configuration)."""
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    n = len(fused_configs())
    times = (C.c_float * n)()
    best = C.c_int()
    prm = make_params(params)
    check(_lib.load().fg_autotune(hand.handle, scene.handle, _oc(obj_of_cand, B), _dptr(q, "q"), B, C.byref(prm),
                                  int(step), int(total_steps), int(nsteps), int(reps), times, C.byref(best),
                                  _stream()), "fg_autotune")
    return best.value, [float(t) for t in times]


def optimize_step_host(hand: Hand, scene: Scene, host_q_in: torch.Tensor, q: torch.Tensor, params: dict, step: int,
                       total_steps: int, nsteps: int = 1, obj_of_cand: torch.Tensor | None = None,
                       loss: torch.Tensor | None = None, host_q_out: torch.Tensor | None = None,
                       host_loss: torch.Tensor | None = None):
    """fg_optimize_step from and to host memory: the library copies host_q_in into the
    device scratch q, steps, and copies q (and the loss) back into host_q_out /
    host_loss (pinned CPU tensors for asynchronous copies; host_q_out defaults to
    host_q_in).  Asynchronous on the current stream."""
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    for t, name in ((host_q_in, "host_q_in"), (host_q_out, "host_q_out"), (host_loss, "host_loss")):
        if t is not None and (t.device.type != "cpu" or t.dtype != _F32 or not t.is_contiguous()):
            raise ValueError("%s must be a contiguous float32 CPU tensor" % name)
    if host_q_out is None:
        host_q_out = host_q_in
    if tuple(host_q_in.shape) != (B, hand.D) or tuple(host_q_out.shape) != (B, hand.D):
        raise ValueError("host q buffers must be [B, D]")
    if host_loss is not None and loss is None:
        loss = torch.empty(B, device=q.device, dtype=_F32)
    prm = make_params(params)
    check(_lib.load().fg_optimize_step_host(hand.handle, scene.handle, _oc(obj_of_cand, B),
                                            C.c_void_p(host_q_in.data_ptr()), _dptr(q, "q"), B, C.byref(prm),
                                            int(step), int(total_steps), int(nsteps),
                                            _dptr(loss, "loss", shape=(B,)) if loss is not None else None,
                                            C.c_void_p(host_q_out.data_ptr()),
                                            C.c_void_p(host_loss.data_ptr()) if host_loss is not None else None,
                                            _stream()), "fg_optimize_step_host")
    return loss


def optimize_step_plain_noalloc(hand: Hand, scene: Scene, q: torch.Tensor, params: dict, step: int,
                                total_steps: int, nsteps: int = 1, obj_of_cand: torch.Tensor | None = None,
                                loss: torch.Tensor | None = None):
    """The per-stage step with its scratch in the library's built-in array instead
    of a workspace (for callers that cannot allocate device memory while running;
    B * P is limited by FG_NOALLOC_SCRATCH_BYTES).  Calls that overlap on the GPU
    share that array and must be ordered."""
    B = q.shape[0]
    _dptr(q, "q", shape=(B, hand.D))
    prm = make_params(params)
    check(_lib.load().fg_optimize_step_plain_noalloc(hand.handle, scene.handle, _oc(obj_of_cand, B), _dptr(q, "q"),
                                                     B, C.byref(prm), int(step), int(total_steps), int(nsteps),
                                                     _dptr(loss, "loss", shape=(B,)) if loss is not None else None,
                                                     _stream()), "fg_optimize_step_plain_noalloc")
    return loss


class Queue:
    """fg_queue: continuous-batching request queue on the current device."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 0, max_requests: int = 0,
                 steps_per_launch: int = 0, timeout_ms: int = 0):
        lib = _lib.load()
        opts = _lib.QueueOpts(max_slots, max_requests, steps_per_launch, timeout_ms)
        h = C.c_void_p()
        check(lib.fg_queue_create(int(hbm_budget_bytes), C.byref(opts), C.byref(h)), "fg_queue_create")
        self.handle = h
        self._shapes = {}

    def submit(self, hand: Hand, sdf: Sdf, q0: np.ndarray, steps: int, params: dict) -> int:
        q0 = np.ascontiguousarray(q0, dtype=np.float32)
        if q0.ndim != 2 or q0.shape[1] != hand.D:
            raise ValueError("q0 must be [B, %d]" % hand.D)
        req = _lib.Request(hand.handle.value, sdf.handle.value, q0.shape[0], int(steps),
                           q0.ctypes.data_as(C.POINTER(C.c_float)), make_params(params))
        rid = C.c_uint64()
        check(_lib.load().fg_queue_submit(self.handle, C.byref(req), C.byref(rid)), "fg_queue_submit")
        self._shapes[rid.value] = q0.shape
        return rid.value

    def poll(self, rid: int) -> bool:
        done = C.c_int()
        check(_lib.load().fg_queue_poll(self.handle, rid, C.byref(done)), "fg_queue_poll")
        return bool(done.value)

    def wait(self, rid: int, timeout_ms: int) -> None:
        check(_lib.load().fg_queue_wait(self.handle, rid, int(timeout_ms)), "fg_queue_wait")

    def result(self, rid: int):
        """(q [B, D], loss [B], latency seconds); forgets the request."""
        B, D = self._shapes[rid]
        q = np.empty((B, D), dtype=np.float32)
        loss = np.empty(B, dtype=np.float32)
        lat = C.c_double()
        check(_lib.load().fg_queue_result(self.handle, rid, q.ctypes.data_as(C.POINTER(C.c_float)),
                                          loss.ctypes.data_as(C.POINTER(C.c_float)), C.byref(lat)),
              "fg_queue_result")
        del self._shapes[rid]
        return q, loss, lat.value

    def stats(self) -> dict:
        st = _lib.QueueStat()
        check(_lib.load().fg_queue_stats(self.handle, C.byref(st)), "fg_queue_stats")
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self, attempts: int = 100) -> None:
        """Destroy the queue.  After a round that exceeded timeout_ms the library may
        report that its stream has not drained yet (FG_ERR_TIMEOUT, each wait bounded
        by timeout_ms); the destroy is retried up to `attempts` times, then raises."""
        if getattr(self, "handle", None) is None or _lib._lib is None:
            return
        for _ in range(max(1, attempts)):
            st = _lib._lib.fg_queue_destroy(self.handle)
            if st != 4:                                  # FG_ERR_TIMEOUT: the stream is still busy
                break
        if st == 4:
            check(st, "fg_queue_destroy")
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_peak_launch(out: torch.Tensor, packed: bool, iters: int) -> float:
    """Enqueue the FP32 fused multiply-add throughput kernel on the current stream:
    out.numel() // 256 CTAs of 256 threads, 8 chains of iters FMAs per thread,
    scalar or packed f32x2.  Returns the launch's floating-point operations; the
    caller times the launch."""
    blocks = out.numel() // 256
    flops = C.c_double()
    check(_lib.load().fg_fp32_peak_launch(int(bool(packed)), int(blocks), int(iters), _dptr(out, "out"),
                                          C.byref(flops), _stream()), "fg_fp32_peak_launch")
    return flops.value


def test_fail_allocation(after: int) -> None:
    """Arm the library's allocation-failure injection (tests): after `after` more
    allocation points pass, the next one fails with FG_ERR_OOM, once; -1 disarms."""
    check(_lib.load().fg_test_fail_allocation(int(after)), "fg_test_fail_allocation")
