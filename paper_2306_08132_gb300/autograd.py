"""torch.autograd.Function over the fused loss/adjoint kernel.

Forward runs fg_loss_and_grad for the loss alone (no adjoint sweep) and saves
only q.  Backward runs fg_loss_and_grad again with the gradient: the fused
kernel recomputes the forward quantities of each point inside the adjoint, so
nothing per point is kept between the passes, and a forward-only call pays for
the forward sweep alone.  The gradient is the paper's leaky one (Sec. III-C),
not the exact derivative of the loss.
"""

from __future__ import annotations

import torch

from . import api


class GraspLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, hand, scene, params, r_dil, obj_of_cand):
        qd = q.detach().contiguous()
        loss, _ = api.loss_and_grad(hand, scene, qd, params, r_dil, obj_of_cand=obj_of_cand, want_grad=False)
        ctx.save_for_backward(qd)
        ctx.args = (hand, scene, params, r_dil, obj_of_cand)
        return loss

    @staticmethod
    def backward(ctx, g_loss):
        (qd,) = ctx.saved_tensors
        hand, scene, params, r_dil, obj_of_cand = ctx.args
        _, grad = api.loss_and_grad(hand, scene, qd, params, r_dil, obj_of_cand=obj_of_cand, want_grad=True)
        return g_loss[:, None] * grad, None, None, None, None, None


def grasp_loss(q: torch.Tensor, hand: api.Hand, scene: api.Scene, params: dict, r_dil: float,
               obj_of_cand: torch.Tensor | None = None) -> torch.Tensor:
    """Per-candidate grasp loss [B], differentiable in q (leaky gradient)."""
    return GraspLoss.apply(q, hand, scene, params, float(r_dil), obj_of_cand)
