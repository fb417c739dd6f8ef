"""torch.autograd wrappers of the differentiable RGB -> CIELAB kernels.

``lab(x, h)`` maps linear RGB (N, 3, ...) to CIELAB with the handle's MACT
rational cube root (or the exact cube root for an exact handle); its
backward is the hand-written CUDA vector-Jacobian product (recomputes the
forward from x; nothing but x is saved).  ``delta_e_loss(x, target, h)`` is
the fused mean Delta E*ab loss whose forward already produces the gradient.
"""
import torch

from . import mact


class MactLab(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, h):
        ctx.h = h
        ctx.save_for_backward(x)
        return mact.mact_lab_forward(h, x.contiguous())

    @staticmethod
    def backward(ctx, grad_lab):
        (x,) = ctx.saved_tensors
        return mact.mact_lab_backward(ctx.h, x.contiguous(), grad_lab), None


class MactDeltaELoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, target_lab, h):
        loss, g = mact.mact_lab_delta_e_loss(h, x.contiguous(), target_lab.contiguous(),
                                             grad=ctx.needs_input_grad[0])
        ctx.save_for_backward(g if g is not None else torch.empty(0, device=x.device))
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return g * grad_out, None, None


def lab(x, h):
    return MactLab.apply(x, h)


def delta_e_loss(x, target_lab, h):
    return MactDeltaELoss.apply(x, target_lab, h)
