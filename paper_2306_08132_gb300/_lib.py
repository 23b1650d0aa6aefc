"""ctypes declarations of the C ABI in include/fastgraspd.h.

Loading fails loudly when libfastgraspd.so is missing: there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfastgraspd.so")

FG_NUM_SIMS = 7
FG_MAX_LINKS = 32

STATUS = {0: "FG_OK", 1: "FG_ERR_INVALID", 2: "FG_ERR_OOM", 3: "FG_ERR_BUDGET", 4: "FG_ERR_TIMEOUT",
          5: "FG_ERR_CUDA", 6: "FG_ERR_BUSY", 7: "FG_ERR_NOT_FOUND"}


class FgError(RuntimeError):
    def __init__(self, status: int, fn: str, detail: str):
        super().__init__("%s failed: %s: %s" % (fn, STATUS.get(status, str(status)), detail))
        self.status = status
        self.name = STATUS.get(status, str(status))


class HandDesc(C.Structure):
    _fields_ = [("n_links", C.c_int), ("n_points", C.c_int), ("parent", C.POINTER(C.c_int)),
                ("T_fix", C.POINTER(C.c_float)), ("axis", C.POINTER(C.c_float)),
                ("q_low", C.POINTER(C.c_float)), ("q_up", C.POINTER(C.c_float)),
                ("pts_local", C.POINTER(C.c_float)), ("link_of_point", C.POINTER(C.c_int))]


class Params(C.Structure):
    _fields_ = [("alpha_leak", C.c_float), ("dt", C.c_float), ("v_test", C.c_float), ("mu", C.c_float),
                ("lr", C.c_float), ("r0", C.c_float), ("w_range", C.c_float), ("w_limit", C.c_float),
                ("w_pen", C.c_float), ("schedule", C.c_int), ("sim_steps", C.c_int),
                ("gauss_seidel", C.c_int)]


class QueueOpts(C.Structure):
    _fields_ = [("max_slots", C.c_int), ("max_requests", C.c_int), ("steps_per_launch", C.c_int),
                ("timeout_ms", C.c_int)]


class Request(C.Structure):
    _fields_ = [("hand", C.c_void_p), ("sdf", C.c_void_p), ("B", C.c_int), ("steps", C.c_int),
                ("host_q0", C.POINTER(C.c_float)), ("params", Params)]


class QueueStat(C.Structure):
    _fields_ = [("pending", C.c_int), ("active", C.c_int), ("finished", C.c_int), ("failed", C.c_int),
                ("bytes_in_use", C.c_size_t), ("budget", C.c_size_t), ("rounds", C.c_uint64),
                ("candidate_steps", C.c_uint64)]


_vp = C.c_void_p
_i = C.c_int
_f = C.c_float
_st = C.c_int

# name -> (argtypes); every function returns fg_status (int) unless listed in _RESTYPE
SIGNATURES = {
    "fg_version": [C.POINTER(_i), C.POINTER(_i)],
    "fg_status_string": [_i],
    "fg_last_error": [C.c_char_p, C.c_size_t],
    "fg_hand_create": [C.POINTER(HandDesc), C.POINTER(_vp)],
    "fg_hand_destroy": [_vp],
    "fg_hand_info": [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)],
    "fg_sdf_create": [_vp, _i, _i, _i, C.POINTER(_f), _f, _f, _f, C.POINTER(_vp)],
    "fg_sdf_destroy": [_vp],
    "fg_sdf_create_mesh": [C.POINTER(_f), _i, C.POINTER(_i), _i, _f, _f, _f, C.POINTER(_vp)],
    "fg_mesh_describe": [C.POINTER(_f), _i, C.POINTER(_i), _i, C.POINTER(_i)],
    "fg_scene_create": [C.POINTER(_vp), _i, C.POINTER(_vp)],
    "fg_scene_destroy": [_vp],
    "fg_fk": [_vp, _vp, _i, _vp, _vp],
    "fg_sdf_query": [_vp, _vp, _i, _f, _vp, _vp, _vp],
    "fg_contact_wrench": [_vp, _vp, _vp, _vp, _i, C.POINTER(Params), _f, _vp, _vp, _vp, _vp],
    "fg_loss_and_grad": [_vp, _vp, _vp, _vp, _i, C.POINTER(Params), _f, _vp, _vp, _vp],
    "fg_optimize_step": [_vp, _vp, _vp, _vp, _i, C.POINTER(Params), _i, _i, _i, _vp, _vp],
    "fg_optimize_step_host": [_vp, _vp, _vp, _vp, _vp, _i, C.POINTER(Params), _i, _i, _i, _vp, _vp, _vp, _vp],
    "fg_contact_measure": [_vp, _vp, _vp, _vp, _i, _vp, _f, _vp, _vp],
    "fg_grasp_epsilon": [_vp, _vp, _vp, _vp, _i, _f, _f, _i, _f, _vp, _i, _vp, _vp, _vp],
    "fg_plain_workspace_size": [_vp, _i, C.POINTER(C.c_size_t)],
    "fg_optimize_step_plain": [_vp, _vp, _vp, _vp, _i, C.POINTER(Params), _i, _i, _i, _vp, _vp, C.c_size_t, _vp],
    "fg_optimize_step_plain_noalloc": [_vp, _vp, _vp, _vp, _i, C.POINTER(Params), _i, _i, _i, _vp, _vp],
    "fg_queue_create": [C.c_size_t, C.POINTER(QueueOpts), C.POINTER(_vp)],
    "fg_queue_submit": [_vp, C.POINTER(Request), C.POINTER(C.c_uint64)],
    "fg_queue_poll": [_vp, C.c_uint64, C.POINTER(_i)],
    "fg_queue_wait": [_vp, C.c_uint64, _i],
    "fg_queue_result": [_vp, C.c_uint64, C.POINTER(_f), C.POINTER(_f), C.POINTER(C.c_double)],
    "fg_queue_stats": [_vp, C.POINTER(QueueStat)],
    "fg_queue_destroy": [_vp],
    "fg_fused_config_count": [C.POINTER(_i)],
    "fg_fused_config_info": [_i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)],
    "fg_fused_config_select": [_i],
    "fg_fused_config_current": [C.POINTER(_i)],
    "fg_autotune": [_vp, _vp, _vp, _vp, _i, C.POINTER(Params), _i, _i, _i, _i, C.POINTER(_f), C.POINTER(_i), _vp],
    "fg_fp32_peak_launch": [_i, _i, _i, _vp, C.POINTER(C.c_double), _vp],
    "fg_test_fail_allocation": [_i],
}
_RESTYPE = {"fg_status_string": C.c_char_p}
OPTIONAL = set()

_lib = None


def load(path: str = LIB_PATH):
    """Load the library and declare its entry points.  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libfastgraspd.so is not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    for name, args in SIGNATURES.items():
        if not hasattr(lib, name):
            if name in OPTIONAL:
                continue
            raise ImportError("libfastgraspd.so does not export %s" % name)
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPE.get(name, _st)
    _lib = lib
    return lib


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    load().fg_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(status: int, fn: str):
    if status != 0:
        raise FgError(status, fn, last_error())
