"""Full-size GPU parity, decision by decision, in the launches the benchmark times.

Workloads at their full sizes: the 8 superquadrics on 128^3 grids with the 4-finger
hand (4,352 points, 8,192 candidates), the 32 convex polyhedra on 128^3 grids with
the 5-finger hand (5,888 points, 131,072 candidates) and the 256-object sweep on
192^3 grids (5,888 points, 65,536 candidates, chunks culled by the min-pyramid).
Both constraint orders: Jacobi-averaged and Gauss-Seidel (Sec. III-C).  Each launch
covers every candidate; the FP64 oracle evaluates a seeded sample of them.

The guard band is located per (point, simulation) by ``O.decision_band``:

* contact flags (Sec. III-C: a point is in contact when its constraint value is
  negative) equal the oracle's bit for bit on every pair outside the band; the pairs
  inside it (within 1 micrometre of the threshold, or changing with an ambiguous
  cell choice, and in the Gauss-Seidel order the rest of a chain after its first
  ambiguous decision) are counted and must stay under 5% of the pairs;
* contact counts N_m equal the oracle's where no flag of (candidate, simulation) is
  masked, and differ by at most the number of masked flags elsewhere;
* loss within 1e-4 relative, gradient, update and wrench within 1e-3 relative (per
  candidate, in norm) of the oracle's result on one of the branches that the
  ambiguous decisions allow (the same branch for all four), for every sampled
  candidate whose branches the oracle enumerates; those must be at least 95% of
  the sample."""

import numpy as np
import pytest
import torch

import synth
from oracle import fastgraspd_oracle as O

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-4
GRAD_TOL = 1e-3
MAX_MASKED_PAIRS = 0.05
MIN_COMPARABLE = 0.95
N_SAMPLE = {"jacobi": 96, "gauss_seidel": 64}

WORKLOADS = {
    "superquadric8": lambda: synth.batched_superquadric_workload(device="cuda"),
    "polyhedra32": lambda: synth.polyhedra_workload(device="cuda"),
    "sweep256": lambda: synth.sweep_workload(device="cuda"),
}


@pytest.fixture(scope="module")
def fg():
    from paper_2306_08132_gb300.build import build_library
    build_library()
    import paper_2306_08132_gb300 as m
    return m


class Full:
    """One workload at full size bound to the library."""

    def __init__(self, fg, w):
        self.w = w
        dev = torch.device("cuda:0")
        self.hand = fg.Hand.from_synth(w.hand)
        self.scene = fg.Scene([fg.Sdf.from_synth(o) for o in w.objects])
        self.oc = torch.tensor(w.obj_of_cand, device=dev, dtype=torch.int32)
        self.q = torch.tensor(w.q0, device=dev)
        self.r = O.dilation_radius(O.Params.from_dict(w.params), 0, w.steps)


@pytest.fixture(scope="module", params=sorted(WORKLOADS))
def full(fg, request):
    case = Full(fg, WORKLOADS[request.param]())
    yield case
    del case
    torch.cuda.empty_cache()


def _unpack_bits(words: np.ndarray, P: int) -> np.ndarray:
    """[n, M, nwords] uint32 -> [n, P, M] bool (bit j of word k is point 32 k + j)."""
    n, M, nw = words.shape
    b = np.unpackbits(words.view(np.uint8).reshape(n, M, nw * 4), axis=-1, bitorder="little")
    return b[..., :P].astype(bool).transpose(0, 2, 1)


def _rel(a, b, floor=1e-6):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)


@pytest.mark.parametrize("form", ["jacobi", "gauss_seidel"])
def test_full_size_decision_parity(fg, full, form):
    w = full.w
    params = dict(w.params, gauss_seidel=int(form == "gauss_seidel"))
    P = w.hand["P"]
    W, N, bits = fg.contact_wrench(full.hand, full.scene, full.q, params, full.r, obj_of_cand=full.oc,
                                   want_bits=True)
    loss, grad = fg.loss_and_grad(full.hand, full.scene, full.q, params, full.r, obj_of_cand=full.oc)
    q1 = full.q.clone()
    fg.optimize_step(full.hand, full.scene, q1, params, 0, w.steps, 1, obj_of_cand=full.oc)
    torch.cuda.synchronize()
    assert torch.isfinite(loss).all() and torch.isfinite(grad).all() and torch.isfinite(q1).all()

    sample = np.sort(np.random.default_rng(31 + len(form)).choice(w.B, size=N_SAMPLE[form], replace=False))
    sel = torch.tensor(sample, device=full.q.device)
    Wg = W[sel].cpu().numpy().astype(np.float64)
    Ng = N[sel].cpu().numpy()
    kap_g = _unpack_bits(bits[sel].cpu().numpy().view(np.uint32), P)
    Lg = loss[sel].cpu().numpy().astype(np.float64)
    Gg = grad[sel].cpu().numpy().astype(np.float64)
    Ug = ((q1 - full.q)[sel].cpu().numpy().astype(np.float64)) / -params["lr"]
    # the launch's counts are its flags' population
    assert np.array_equal(Ng, kap_g.sum(1)), "counts disagree with the launch's own flags"

    objs = sorted({int(w.obj_of_cand[b]) for b in sample})
    S = O.Setup(w.hand, [w.objects[k] for k in objs], params)
    masked_pairs = mismatched = compared = 0
    n_branchy = 0
    worst = 0.0
    for k, ob in enumerate(objs):
        rows = np.nonzero(w.obj_of_cand[sample] == ob)[0]
        band = O.decision_band(S.hand, S.objs[k], w.q0[sample[rows]], full.r, S.prm)
        ref = band["ref"]
        masked = band["masked"]
        masked_pairs += int(masked.sum())
        bad = (kap_g[rows] != ref["kappa"]) & ~masked
        mismatched += int(bad.sum())
        assert not bad.any(), ("flags differ outside the band", sample[rows[np.nonzero(bad.any((1, 2)))[0]]])
        slack = masked.sum(1)                                  # [n, M]
        dN = np.abs(Ng[rows].astype(np.int64) - ref["N"].astype(np.int64))
        assert (dN <= slack).all(), ("counts", sample[rows], dN, slack)
        for j, row in enumerate(rows):
            if not band["comparable"][j]:
                continue
            compared += 1
            br = band["branches"][j]
            n_branchy += len(br["L"]) > 1
            errs = []
            for kk in range(len(br["L"])):
                lrel = abs(Lg[row] - br["L"][kk]) / max(abs(br["L"][kk]), 1e-6)
                errs.append(max(lrel / LOSS_TOL, _rel(Gg[row], br["grad"][kk]) / GRAD_TOL,
                                _rel(Ug[row], br["grad"][kk]) / GRAD_TOL, _rel(Wg[row], br["W"][kk]) / GRAD_TOL))
            e = min(errs)
            worst = max(worst, e)
            assert e <= 1.0, ("candidate", int(sample[row]), errs)
    pairs = len(sample) * P * 7
    frac_masked = masked_pairs / pairs
    frac_compared = compared / len(sample)
    print("%s %s: %d candidates, %d pairs; flags masked %d (%.2e), mismatched outside the band %d; "
          "loss/grad/update/wrench compared on %d (%.1f%%, %d with several branches), worst error %.2f of the "
          "tolerance" % (w.name, form, len(sample), pairs, masked_pairs, frac_masked, mismatched, compared,
                         100 * frac_compared, n_branchy, worst))
    assert frac_masked <= MAX_MASKED_PAIRS
    assert frac_compared >= MIN_COMPARABLE
    assert (np.asarray(N.cpu()) >= 0).all()
