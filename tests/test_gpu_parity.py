"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (from the float32 arithmetic and the method's amplification 1/dt):
loss within 1e-4 relative, gradients / wrenches / updates within 1e-3 relative
in norm per candidate, contact flags and contact counts bit-exact.  Candidates are
compared when every decision of the oracle sits outside the guard band (voxel
faces 1e-5 voxel, |phi_m| 1e-6 m, friction cone 1e-6 m, n nearly parallel to v),
where float32 and float64 must branch alike."""

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-4
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def fg():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as m
    return m


def _dev():
    return torch.device("cuda:0")


class Case:
    """A workload bound to both sides: oracle setup and library handles."""

    def __init__(self, fg, w):
        self.w = w
        self.S = O.Setup(w.hand, w.objects, w.params)
        self.hand = fg.Hand.from_synth(w.hand)
        self.sdfs = [fg.Sdf.from_synth(o) for o in w.objects]
        self.scene = fg.Scene(self.sdfs)
        self.oc = torch.tensor(w.obj_of_cand, device=_dev(), dtype=torch.int32)

    def clean(self, q, r):
        mask = np.zeros(len(q), dtype=bool)
        for k in np.unique(self.w.obj_of_cand):
            idx = np.nonzero(self.w.obj_of_cand == k)[0]
            mask[idx] = O.clean_candidates(self.S.hand, self.S.objs[int(k)], q[idx], r, self.S.prm)
        return mask


def rel_rows(a, b, floor=1e-6):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)


@pytest.fixture(scope="module")
def tiny(fg):
    return Case(fg, synth.tiny_sphere_workload(n_cand=64))


def test_fk_matches_oracle(fg):
    for kind, ppl in ((3, 64), (4, 40), (5, 37)):
        h = synth.make_hand(kind, ppl)
        hand = fg.Hand.from_synth(h)
        rng = np.random.default_rng(kind)
        q = np.concatenate([rng.normal(size=(9, 3)) * 0.1, rng.normal(size=(9, 3)) * 1.5,
                            rng.uniform(-1.6, 1.6, size=(9, hand.J))], axis=1).astype(np.float32)
        q[0] = 0.0                                     # rest pose
        q[1, 3:6] = [1e-9, -2e-9, 0.0]                 # tiny rotation (series branch)
        pts = fg.fk(hand, torch.tensor(q, device=_dev())).cpu().numpy().astype(np.float64)
        oh = O.Hand.from_synth(h)
        R, o = O.forward_kinematics(oh, torch.tensor(q.astype(np.float64)))
        ref = O.hand_points(oh, R, o).numpy()               # [B,P,3]
        got = pts.reshape(3, len(q), hand.P).transpose(1, 2, 0)
        assert np.abs(got - ref).max() < 2e-6


def test_sdf_query_matches_oracle(fg):
    o = synth.sphere_grid(0.04, 64, 0.002)
    sdf = fg.Sdf.from_synth(o)
    ob = O.Obj.from_synth(o)
    rng = np.random.default_rng(5)
    for n in (1, 31, 1000, 4097):                     # ragged sizes
        p = rng.uniform(-0.09, 0.09, size=(n, 3))       # includes points outside the grid
        u = (p - ob.origin.numpy()) / ob.pitch
        keep = (np.abs(u - np.round(u)) > 1e-4).all(axis=1)
        p = p[keep].astype(np.float32)
        pts = torch.tensor(p.T.copy(), device=_dev())
        phi, g = fg.sdf_query(sdf, pts, 0.003)
        ref_phi, ref_g = O.sdf_query(ob, torch.tensor(p.astype(np.float64)), 0.003)
        assert np.abs(phi.cpu().numpy() - ref_phi.numpy()).max() < 2e-6
        assert np.abs(g.cpu().numpy().T - ref_g.numpy()).max() < 1e-4
    empty = torch.zeros(3, 0, device=_dev())
    phi, g = fg.sdf_query(sdf, empty, 0.0)
    assert phi.numel() == 0


def _oracle_forward(case, q, r, alpha=None):
    return O.batch_loss_and_grad(case.S, q, case.w.obj_of_cand[:len(q)], r) if alpha is None else None


def test_contact_wrench_matches_oracle(fg, tiny):
    w, r = tiny.w, 0.004
    q = w.q0
    W, N, bits = fg.contact_wrench(tiny.hand, tiny.scene, torch.tensor(q, device=_dev()), w.params, r,
                                   obj_of_cand=tiny.oc, want_bits=True)
    torch.cuda.synchronize()
    ref = O.batch_loss_and_grad(tiny.S, q, w.obj_of_cand, r)
    clean = tiny.clean(q, r)
    assert clean.sum() >= 0.75 * len(q)
    assert (ref["N"].sum(axis=1) > 0).sum() >= 8, "workload must exercise contacts"
    Wg = W.cpu().numpy().astype(np.float64)
    Ng = N.cpu().numpy()
    bw = bits.cpu().numpy().view(np.uint32)
    P = w.hand["P"]
    for b in np.nonzero(clean)[0]:
        assert np.array_equal(Ng[b], ref["N"][b].astype(np.int32)), b
        kap = ref["kappa"][b]                            # [P, 7]
        for m in range(7):
            got = np.unpackbits(bw[b, m].view(np.uint8), bitorder="little")[:P].astype(bool)
            assert np.array_equal(got, kap[:, m]), (b, m)
        err = np.linalg.norm(Wg[b] - ref["W"][b]) / max(np.linalg.norm(ref["W"][b]), 1e-9)
        assert np.linalg.norm(ref["W"][b]) == 0 or err < GRAD_TOL, (b, err)


def _compare_loss_grad(loss, grad, ref, clean):
    L = loss.astype(np.float64)
    G = grad.astype(np.float64)
    idx = np.nonzero(clean)[0]
    lrel = np.abs(L[idx] - ref["L"][idx]) / np.maximum(np.abs(ref["L"][idx]), 1e-6)
    grel = rel_rows(G[idx], ref["grad"][idx])
    assert lrel.max() < LOSS_TOL, (idx[np.argmax(lrel)], lrel.max())
    assert grel.max() < GRAD_TOL, (idx[np.argmax(grel)], grel.max())
    return lrel.max(), grel.max()


@pytest.mark.parametrize("alpha", [0.1, 0.0])
def test_loss_and_grad_matches_oracle(fg, tiny, alpha):
    w, r = tiny.w, 0.004
    params = dict(w.params, alpha_leak=alpha)
    loss, grad = fg.loss_and_grad(tiny.hand, tiny.scene, torch.tensor(w.q0, device=_dev()), params, r,
                                  obj_of_cand=tiny.oc)
    S = O.Setup(w.hand, w.objects, params)
    ref = O.batch_loss_and_grad(S, w.q0, w.obj_of_cand, r)
    _compare_loss_grad(loss.cpu().numpy(), grad.cpu().numpy(), ref, tiny.clean(w.q0, r))


def test_optimize_step_matches_oracle_and_plain(fg, tiny):
    w = tiny.w
    K = w.steps
    q0 = torch.tensor(w.q0, device=_dev())
    q1 = q0.clone()
    loss = fg.optimize_step(tiny.hand, tiny.scene, q1, w.params, 0, K, 1, obj_of_cand=tiny.oc)
    q2 = q0.clone()
    loss2 = fg.optimize_step_plain(tiny.hand, tiny.scene, q2, w.params, 0, K, 1, obj_of_cand=tiny.oc)
    torch.cuda.synchronize()
    r = O.dilation_radius(tiny.S.prm, 0, K)
    ref = O.batch_loss_and_grad(tiny.S, w.q0, w.obj_of_cand, r)
    clean = tiny.clean(w.q0, r)
    lr = w.params["lr"]
    for qq, ll in ((q1, loss), (q2, loss2)):
        step = (qq - q0).cpu().numpy().astype(np.float64)
        _compare_loss_grad(ll.cpu().numpy(), -step / lr, ref, clean)


def test_fused_multi_step_equals_repeated_single_steps(fg, tiny):
    """nsteps = 3 in one persistent launch is bit-identical to three launches."""
    w = tiny.w
    params = dict(w.params, r0=0.01, schedule="linear")
    q0 = torch.tensor(w.q0, device=_dev())
    qa = q0.clone()
    la = fg.optimize_step(tiny.hand, tiny.scene, qa, params, 5, 20, 3, obj_of_cand=tiny.oc)
    qb = q0.clone()
    for s in range(3):
        lb = fg.optimize_step(tiny.hand, tiny.scene, qb, params, 5 + s, 20, 1, obj_of_cand=tiny.oc)
    torch.cuda.synchronize()
    assert torch.equal(qa, qb)
    assert torch.equal(la, lb)


def test_dilation_schedule_on_device(fg, tiny):
    """optimize_step at step k uses r_k = r0 (1 - k/(K-1)): equal to loss_and_grad at r_k."""
    w = tiny.w
    params = dict(w.params, r0=0.01, schedule="linear")
    q0 = torch.tensor(w.q0[:8], device=_dev())
    for k, K in ((0, 11), (4, 11), (10, 11), (15, 11)):
        r = O.dilation_radius(O.Params.from_dict(params), k, K)
        q1 = q0.clone()
        l1 = fg.optimize_step(tiny.hand, tiny.scene, q1, params, k, K, 1, obj_of_cand=tiny.oc[:8])
        l2, g2 = fg.loss_and_grad(tiny.hand, tiny.scene, q0, params, r, obj_of_cand=tiny.oc[:8])
        torch.cuda.synchronize()
        assert torch.equal(l1, l2)
        # the update is q - lr g, rounded once in the kernel (fused multiply-add)
        assert torch.allclose(q1, q0 - params["lr"] * g2, rtol=1e-6, atol=1e-6)


def test_edge_cases(fg, tiny):
    w = tiny.w
    dev = _dev()
    # B = 0 is a no-op
    e = torch.zeros(0, w.hand["D"], device=dev)
    l, g = fg.loss_and_grad(tiny.hand, tiny.scene, e, w.params, 0.0)
    assert l.numel() == 0
    # a hand far from the object: no contact, L_stable = 6V/7
    q = np.zeros((3, w.hand["D"]), dtype=np.float32)
    q[:, 0] = [0.5, -0.4, 0.3]
    q[:, 6:] = 0.5 * (w.hand["q_low"] + w.hand["q_up"])
    loss, grad = fg.loss_and_grad(tiny.hand, tiny.scene, torch.tensor(q, device=dev), w.params, 0.004)
    ref = O.batch_loss_and_grad(tiny.S, q, np.zeros(3, dtype=np.int32), 0.004)
    assert np.allclose(loss.cpu().numpy(), 6.0 / 7.0, rtol=1e-6)
    assert rel_rows(grad.cpu().numpy().astype(np.float64), ref["grad"]).max() < GRAD_TOL
    # an object index outside the scene gives NaN and leaves q alone
    bad = torch.tensor([0, 3, -1], device=dev, dtype=torch.int32)
    qq = torch.tensor(w.q0[:3], device=dev)
    loss, grad = fg.loss_and_grad(tiny.hand, tiny.scene, qq, w.params, 0.004, obj_of_cand=bad)
    ln = loss.cpu().numpy()
    assert np.isfinite(ln[0]) and np.isnan(ln[1]) and np.isnan(ln[2])
    q2 = qq.clone()
    fg.optimize_step(tiny.hand, tiny.scene, q2, w.params, 0, 10, 2, obj_of_cand=bad)
    assert torch.equal(q2[1:], qq[1:])
    # invalid arguments raise with the library's message
    with pytest.raises(Exception, match="nsteps"):
        fg.optimize_step(tiny.hand, tiny.scene, qq.clone(), w.params, 0, 10, 0)


def test_ragged_hand_and_point_counts(fg):
    """Links whose point ranges are not 32-aligned (warps straddle links) and a
    point count that is not a multiple of the CTA size."""
    w = synth.tiny_sphere_workload(n_cand=24)
    h = synth.make_hand(3, 21)                         # P = 210, links at multiples of 21
    qs = synth.sample_candidates(np.random.default_rng(7), h, 24, 0.095)
    w2 = synth.Workload("ragged", h, w.objects, qs, np.zeros(24, dtype=np.int32), w.params, 10)
    case = Case(fg, w2)
    loss, grad = fg.loss_and_grad(case.hand, case.scene, torch.tensor(qs, device=_dev()), w.params, 0.004)
    ref = O.batch_loss_and_grad(case.S, qs, w2.obj_of_cand, 0.004)
    _compare_loss_grad(loss.cpu().numpy(), grad.cpu().numpy(), ref, case.clean(qs, 0.004))
    q1 = torch.tensor(qs, device=_dev())
    q2 = q1.clone()
    fg.optimize_step(case.hand, case.scene, q1, w.params, 0, 10, 1)
    fg.optimize_step_plain(case.hand, case.scene, q2, w.params, 0, 10, 1)
    d1 = (q1 - torch.tensor(qs, device=_dev())).cpu().numpy()
    d2 = (q2 - torch.tensor(qs, device=_dev())).cpu().numpy()
    assert rel_rows(d1.astype(np.float64), d2.astype(np.float64)).max() < 1e-4


def test_mixed_objects_four_finger(fg):
    """Several superquadrics in one batch (object-major candidates), 4-finger hand."""
    w = synth.batched_superquadric_workload(n_obj=3, per_obj=12, grid_n=48, points_per_link=32, steps=50,
                                            device="cuda")
    case = Case(fg, w)
    r = O.dilation_radius(case.S.prm, 7, w.steps)
    loss, grad = fg.loss_and_grad(case.hand, case.scene, torch.tensor(w.q0, device=_dev()), w.params, r,
                                  obj_of_cand=case.oc)
    ref = O.batch_loss_and_grad(case.S, w.q0, w.obj_of_cand, r)
    clean = case.clean(w.q0, r)
    assert clean.sum() >= 0.5 * len(clean)
    _compare_loss_grad(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)


def test_five_finger_polyhedra(fg):
    w = synth.polyhedra_workload(n_obj=2, per_obj=8, grid_n=64, points_per_link=48, steps=20, device="cuda")
    case = Case(fg, w)
    r = 0.006
    loss, grad = fg.loss_and_grad(case.hand, case.scene, torch.tensor(w.q0, device=_dev()), w.params, r,
                                  obj_of_cand=case.oc)
    ref = O.batch_loss_and_grad(case.S, w.q0, w.obj_of_cand, r)
    _compare_loss_grad(loss.cpu().numpy(), grad.cpu().numpy(), ref, case.clean(w.q0, r))


def test_every_fused_configuration_matches_oracle(fg, tiny):
    """Each compiled (warps per candidate, register budget) configuration gives the
    oracle's loss and gradient; the autotuner selects one of them."""
    w, r = tiny.w, 0.004
    ref = O.batch_loss_and_grad(tiny.S, w.q0, w.obj_of_cand, r)
    clean = tiny.clean(w.q0, r)
    q = torch.tensor(w.q0, device=_dev())
    cfgs = fg.fused_configs()
    assert len(cfgs) >= 4
    try:
        for i in range(len(cfgs)):
            fg.fused_config_select(i)
            loss, grad = fg.loss_and_grad(tiny.hand, tiny.scene, q, w.params, r, obj_of_cand=tiny.oc)
            _compare_loss_grad(loss.cpu().numpy(), grad.cpu().numpy(), ref, clean)
            q1 = q.clone()
            fg.optimize_step(tiny.hand, tiny.scene, q1, w.params, 0, w.steps, 1, obj_of_cand=tiny.oc)
            step = (q1 - q).cpu().numpy().astype(np.float64) / -w.params["lr"]
            _compare_loss_grad(loss.cpu().numpy(), step, ref, clean)
        best, times = fg.autotune(tiny.hand, tiny.scene, q, w.params, 0, w.steps, 1, obj_of_cand=tiny.oc, reps=2)
        assert 0 <= best < len(cfgs) and fg.fused_config_current() == best
        assert all(t > 0 for t in times)
        assert torch.equal(q, torch.tensor(w.q0, device=_dev()))     # the autotuner leaves q alone
    finally:
        fg.fused_config_select(-1)


def test_host_buffer_step_equals_device_step(fg, tiny):
    """fg_optimize_step_host (the library copies q in from host memory and q and the
    loss back) gives the device entry point's results bit for bit, from pinned and
    from pageable host buffers, in place (one host buffer) or not; B = 0 is a no-op."""
    w = tiny.w
    q0 = torch.tensor(w.q0, device=_dev())
    q_ref = q0.clone()
    l_ref = fg.optimize_step(tiny.hand, tiny.scene, q_ref, w.params, 2, w.steps, 2, obj_of_cand=tiny.oc)
    torch.cuda.synchronize()
    for pinned in (True, False):
        hq = torch.tensor(w.q0)
        if pinned:
            hq = hq.pin_memory()
        hout = torch.empty_like(hq)
        hloss = torch.empty(w.B, dtype=torch.float32)
        qd = torch.empty_like(q0)
        fg.optimize_step_host(tiny.hand, tiny.scene, hq, qd, w.params, 2, w.steps, 2, obj_of_cand=tiny.oc,
                              host_q_out=hout, host_loss=hloss)
        torch.cuda.synchronize()
        assert torch.equal(hout, q_ref.cpu()) and torch.equal(hloss, l_ref.cpu())
        assert torch.equal(hq, torch.tensor(w.q0))          # the input is left alone
        fg.optimize_step_host(tiny.hand, tiny.scene, hq, qd, w.params, 2, w.steps, 2, obj_of_cand=tiny.oc)
        torch.cuda.synchronize()
        assert torch.equal(hq, q_ref.cpu())                 # in place
    e = torch.zeros(0, w.hand["D"])
    fg.optimize_step_host(tiny.hand, tiny.scene, e, torch.zeros(0, w.hand["D"], device=_dev()), w.params, 0, 10, 1)


def test_fp32_peak_kernel(fg):
    """The FMA throughput kernel behind the ALU roofline's denominator: both forms run,
    report their flops (blocks x 256 threads x iterations x 8 chains x 2 or 4), and
    write one value per thread; invalid sizes are refused."""
    from paper_2306_08132_gb300 import _lib
    out = torch.full((4 * 256,), float("nan"), device=_dev())
    f1 = fg.fp32_peak_launch(out, False, 100)
    torch.cuda.synchronize()
    assert f1 == 4 * 256 * 100 * 8 * 2 and torch.isfinite(out).all()
    out.fill_(float("nan"))
    f2 = fg.fp32_peak_launch(out, True, 100)
    torch.cuda.synchronize()
    assert f2 == 2 * f1 and torch.isfinite(out).all()
    with pytest.raises(_lib.FgError):
        fg.fp32_peak_launch(out, False, 0)
