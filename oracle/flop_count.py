"""Floating-point operation count of the oracle's step (a counting instantiation).

TEST INFRASTRUCTURE ONLY, like ``fastgraspd_oracle``: only ``tests/`` and the
benchmark's CPU legs may use it.

The oracle's loss and gradient (forward pass and torch reverse mode, float64)
run under a dispatch mode that counts, per aten operator applied to floating
point tensors:

  * arithmetic: one flop per output element for add, sub, mul, div, neg and
    reciprocal; two for addcmul / addcdiv; a reduction (sum, mean) costs one
    flop per input element it folds in (input elements - output elements);
    a matrix product costs 2 m n k (plus the added term for addmm / baddbmm);
  * special functions: sqrt, rsqrt, exp, log, sin, cos, tan, atan2, pow,
    counted apart (one per output element);
  * everything else (comparisons, selects, clamps, copies, indexing, views) is
    not a flop.

The count is of what the oracle, as written, computes: it evaluates both sides
of every ``where`` select and the contact force of every (point, simulation)
pair, and reverse mode re-derives each of them, so it overstates the work a
kernel has to do.  It is reported next to the kernel's own minimal count.
"""

from __future__ import annotations

from collections import Counter

import numpy as np
import torch
from torch.utils._python_dispatch import TorchDispatchMode

from . import fastgraspd_oracle as O

_UNIT = {"add", "add_", "sub", "sub_", "rsub", "mul", "mul_", "div", "div_", "neg", "neg_", "reciprocal",
         "reciprocal_"}
_TWO = {"addcmul", "addcmul_", "addcdiv", "addcdiv_"}
_SPECIAL = {"sqrt", "rsqrt", "exp", "log", "sin", "cos", "tan", "atan2", "pow", "sqrt_", "exp_", "log_",
            "sin_", "cos_", "pow_"}
_REDUCE = {"sum", "mean"}
_MATMUL = {"mm", "bmm", "addmm", "baddbmm", "matmul", "dot", "mv"}


def _is_float(x) -> bool:
    return isinstance(x, torch.Tensor) and x.is_floating_point()


def _numel_out(out) -> int:
    if isinstance(out, torch.Tensor):
        return out.numel()
    if isinstance(out, (tuple, list)):
        return sum(_numel_out(o) for o in out)
    return 0


class FlopCounter(TorchDispatchMode):
    """Counts flops (and special-function evaluations) of the aten operators run inside it."""

    def __init__(self):
        super().__init__()
        self.flops = 0
        self.special = 0
        self.by_op = Counter()

    def __torch_dispatch__(self, func, types, args=(), kwargs=None):
        kwargs = kwargs or {}
        out = func(*args, **kwargs)
        name = func.overloadpacket.__name__
        tensors = [a for a in list(args) + list(kwargs.values()) if isinstance(a, torch.Tensor)]
        if not any(_is_float(t) for t in tensors) and not (isinstance(out, torch.Tensor) and _is_float(out)):
            return out
        n = 0
        if name in _UNIT:
            n = _numel_out(out)
        elif name in _TWO:
            n = 2 * _numel_out(out)
        elif name in _REDUCE:
            n = max(tensors[0].numel() - _numel_out(out), 0)
        elif name in _MATMUL:
            a, b = tensors[-2], tensors[-1]
            if name in ("dot",):
                n = 2 * a.numel()
            elif name == "mv":
                n = 2 * a.numel()
            else:
                k = a.shape[-1]
                n = 2 * _numel_out(out) * k
                if name in ("addmm", "baddbmm"):
                    n += _numel_out(out)
        elif name in _SPECIAL:
            self.special += _numel_out(out)
            self.by_op[name] += _numel_out(out)
            return out
        if n:
            self.flops += n
            self.by_op[name] += n
        return out


def count_step(setup: O.Setup, q32: np.ndarray, obj_index: int, r: float, want_grad: bool = True) -> dict:
    """Flops of the oracle's loss (and gradient) for candidates q32 [B, D] on one object.
    Returns totals and per point-step figures (divided by B x P)."""
    hand, obj = setup.hand, setup.objs[obj_index]
    q = torch.as_tensor(np.asarray(q32, dtype=np.float64)).clone().requires_grad_(want_grad)
    with FlopCounter() as fc:
        out = O.evaluate_any(hand, obj, q, r, setup.prm)
        if want_grad:
            torch.autograd.grad(out["L"].sum(), q)
    units = q.shape[0] * hand.P
    return {"flops": fc.flops, "special": fc.special, "point_steps": units,
            "flops_per_point_step": fc.flops / units, "special_per_point_step": fc.special / units,
            "by_op": dict(fc.by_op)}


if __name__ == "__main__":
    import synth

    w = synth.batched_superquadric_workload(device="cpu")
    S = O.Setup(w.hand, w.objects, w.params)
    r = O.dilation_radius(S.prm, 0, w.steps)
    for grad in (False, True):
        c = count_step(S, w.q0[:8], 0, r, want_grad=grad)
        print("%s: %.1f flops + %.2f special per point-step"
              % ("forward + gradient" if grad else "forward", c["flops_per_point_step"], c["special_per_point_step"]))
