"""The allocation-free step (fg_optimize_step_plain_noalloc).

This entry point has no counterpart in the paper: it serves callers that cannot
allocate device memory while running (a real-time planning loop, or a host whose
device memory is owned by another runtime), by keeping the per-stage scratch in
an array built into the library.  Here it is called through the C ABI twice in a
row and must agree with the workspace entry point, fg_optimize_step_plain, each
time; a step too large for the built-in array must be refused with a message.
The file is named to run last so that a failure here leaves every other test
already run."""

import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _last_error(lib) -> str:
    buf = C.create_string_buffer(512)
    lib.fg_last_error(buf, 512)
    return buf.value.decode()


def test_noalloc_step_matches_workspace_step_on_two_calls():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as fg
    from paper_2306_08132_gb300 import _lib
    lib = _lib.load()

    w = synth.tiny_sphere_workload(n_cand=32)
    hand = fg.Hand.from_synth(w.hand)
    sdf = fg.Sdf.from_synth(w.objects[0])
    scene = fg.Scene([sdf])
    dev = torch.device("cuda:0")
    B, D = w.q0.shape
    prm = fg.make_params(w.params)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    q_ref = torch.tensor(w.q0, device=dev)
    for call in range(2):
        q_start = q_ref.clone()
        loss_ref = torch.empty(B, device=dev)
        fg.optimize_step_plain(hand, scene, q_ref, w.params, call, w.steps, 1, loss=loss_ref)
        q_new = q_start.clone()
        loss_new = torch.full((B,), float("nan"), device=dev)
        st = lib.fg_optimize_step_plain_noalloc(hand.handle, scene.handle, None, C.c_void_p(q_new.data_ptr()), B,
                                                C.byref(prm), call, w.steps, 1, C.c_void_p(loss_new.data_ptr()),
                                                stream)
        assert st == 0, _last_error(lib)
        torch.cuda.synchronize()
        d_ref = (q_ref - q_start).cpu().numpy().astype(np.float64)
        d_new = (q_new - q_start).cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(d_new - d_ref, axis=1) / np.maximum(np.linalg.norm(d_ref, axis=1), 1e-12)
        assert rel.max() < 1e-4, (call, rel.max())
        lr = loss_ref.cpu().numpy().astype(np.float64)
        ln = loss_new.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(ln - lr) <= 1e-5 * np.maximum(np.abs(lr), 1e-6)), call
        q_ref = q_new.clone()      # the next call starts where this one ended


def test_noalloc_step_refuses_oversized_batches():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as fg
    from paper_2306_08132_gb300 import _lib
    lib = _lib.load()

    w = synth.tiny_sphere_workload(n_cand=4)
    hand = fg.Hand.from_synth(w.hand)
    scene = fg.Scene([fg.Sdf.from_synth(w.objects[0])])
    prm = fg.make_params(w.params)
    need = fg.plain_workspace_size(hand, 4096)
    assert need > (32 << 20)
    q = torch.zeros(1, hand.D, device="cuda:0")          # never read: the call is refused first
    st = lib.fg_optimize_step_plain_noalloc(hand.handle, scene.handle, None, C.c_void_p(q.data_ptr()), 4096,
                                            C.byref(prm), 0, 10, 1, None,
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    assert "too large" in _last_error(lib)


def test_noalloc_step_refuses_what_the_workspace_step_refuses():
    """Both entry points check their arguments with the same routine: parameters the
    workspace form refuses (infinite test velocity, friction or dilation, non-finite
    loss weights, the T-step or Gauss-Seidel forms) are refused here too, before any
    launch, with FG_ERR_INVALID."""
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as fg
    from paper_2306_08132_gb300 import _lib
    lib = _lib.load()

    w = synth.tiny_sphere_workload(n_cand=4)
    hand = fg.Hand.from_synth(w.hand)
    scene = fg.Scene([fg.Sdf.from_synth(w.objects[0])])
    B = 4
    q = torch.tensor(w.q0, device="cuda:0")
    ws = torch.empty(fg.plain_workspace_size(hand, B) + 256, dtype=torch.uint8, device="cuda:0")
    ws_ptr = (ws.data_ptr() + 255) // 256 * 256
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    bad = [{"v_test": float("inf")}, {"mu": float("inf")}, {"r0": float("inf")}, {"w_range": float("nan")},
           {"w_limit": float("inf")}, {"w_pen": float("-inf")}, {"dt": 0.0}, {"alpha_leak": 1.5},
           {"sim_steps": 1}, {"gauss_seidel": 1}]
    for change in bad:
        prm = fg.make_params(dict(w.params, **change))
        st_ws = lib.fg_optimize_step_plain(hand.handle, scene.handle, None, C.c_void_p(q.data_ptr()), B,
                                           C.byref(prm), 0, 10, 1, None, C.c_void_p(ws_ptr), ws.numel() - 256,
                                           stream)
        st_na = lib.fg_optimize_step_plain_noalloc(hand.handle, scene.handle, None, C.c_void_p(q.data_ptr()), B,
                                                   C.byref(prm), 0, 10, 1, None, stream)
        assert st_ws == 1 and st_na == 1, (change, st_ws, st_na)
    torch.cuda.synchronize()
    assert torch.equal(q, torch.tensor(w.q0, device="cuda:0"))    # nothing ran
