"""torch.autograd bindings of the forward map u = B g and its adjoint (Sec. 4).

``FemInpaint.apply(g, mesh)`` returns the inpainted image u = B g; its
backward is the hand-written adjoint kernel path (fem_adjoint): dL/dg =
B^T dL/du.  ``TonalLoss.apply(g, f, mesh)`` returns 1/2 ||B g - f||^2 with
gradient B^T (B g - f), the quantity whose zero is the normal equations
(eq. 5), both from fem_tonal_loss.  Every step of the method runs in the
CUDA library; these classes only marshal tensors.
"""
from __future__ import annotations

import torch

from . import Mesh, fem_tonal_loss, params


class FemInpaint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g: torch.Tensor, mesh: Mesh, p=None):
        ctx.mesh = mesh
        ctx.p = p
        return mesh.inpaint(g.detach().contiguous(), p)

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        gbar = ctx.mesh.adjoint(grad_u.detach().to(torch.float32).contiguous(), ctx.p)
        return gbar, None, None


class TonalLoss(torch.autograd.Function):
    """The loss and its gradient both come from one library call
    (fem_tonal_loss): the gradient B^T (B g - f) is computed in the forward
    pass when g requires it, and the backward pass only applies the chain
    rule's scalar factor."""

    @staticmethod
    def forward(ctx, g: torch.Tensor, f: torch.Tensor, mesh: Mesh, p=None):
        loss = torch.empty((), dtype=torch.float64, device=g.device)
        grad = torch.empty(mesh.nmask, dtype=torch.float32, device=g.device) if ctx.needs_input_grad[0] else None
        fem_tonal_loss(mesh.h, g.detach().to(torch.float32).contiguous(), f.detach().contiguous(), loss, grad, p)
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return grad * grad_out.to(grad.dtype), None, None, None


__all__ = ["FemInpaint", "TonalLoss", "params"]
