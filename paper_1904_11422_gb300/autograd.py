"""torch.autograd bindings of the gain gradient (epic_grad).

``calib_loss(plan, d_volts, gains, model)`` returns the image-plane loss
L = sum (I - M)^2 over channels, XX/YY and pixels as a differentiable function
of the complex per-antenna gains; its backward pass is the library's adjoint
kernel (no autograd graph through the imaging itself).  Argument marshalling
only: forward and backward both run in libepic.so.
"""
from __future__ import annotations

import torch

from . import epic


class EpicCalibLoss(torch.autograd.Function):
    """gains: float32 CUDA tensor [C][A][P][2] (re, im) -> scalar loss."""

    @staticmethod
    def forward(ctx, gains, plan, d_volts, n_time, model):
        g = gains.detach().contiguous()
        grad = torch.empty_like(g)
        loss = torch.empty((), dtype=torch.float32, device=g.device)
        epic.epic_grad(plan, d_volts, n_time, g, model.contiguous(), grad, loss)
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None, None, None, None


def calib_loss(plan, d_volts, gains, model, n_time: int | None = None):
    """Loss for complex gains [C][A][P] (complex64) or real-view gains [C][A][P][2]."""
    if n_time is None:
        n_time = d_volts.shape[0]
    real = torch.view_as_real(gains) if gains.is_complex() else gains
    return EpicCalibLoss.apply(real, plan, d_volts, n_time, model)
