"""torch.autograd.Function over the fused loss/adjoint kernel.

Forward runs fg_loss_and_grad once: the loss and, when q needs a gradient, dL/dq
from the hand-written adjoint (which recomputes each point's forward quantities
inside the kernel, so nothing per point is kept).  Only the [B, D] gradient is
saved for backward, which scales it by the incoming gradient.  The gradient is
the paper's leaky one (Sec. III-C), not the exact derivative of the loss.
"""

from __future__ import annotations

import torch

from . import api


class GraspLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, hand, scene, params, r_dil, obj_of_cand):
        need = q.requires_grad
        loss, grad = api.loss_and_grad(hand, scene, q.detach().contiguous(), params, r_dil,
                                       obj_of_cand=obj_of_cand, want_grad=need)
        if need:
            ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, g_loss):
        (grad,) = ctx.saved_tensors
        return g_loss[:, None] * grad, None, None, None, None, None


def grasp_loss(q: torch.Tensor, hand: api.Hand, scene: api.Scene, params: dict, r_dil: float,
               obj_of_cand: torch.Tensor | None = None) -> torch.Tensor:
    """Per-candidate grasp loss [B], differentiable in q (leaky gradient)."""
    return GraspLoss.apply(q, hand, scene, params, float(r_dil), obj_of_cand)
