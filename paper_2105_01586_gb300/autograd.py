"""torch.autograd bindings of the forward map u = B g and its adjoint (Sec. 4).

``FemInpaint.apply(g, mesh)`` returns the inpainted image u = B g; its
backward is the hand-written adjoint kernel path (fem_adjoint): dL/dg =
B^T dL/du.  ``TonalLoss.apply(g, f, mesh)`` returns 1/2 ||B g - f||^2 with
gradient B^T (B g - f), the quantity whose zero is the normal equations
(eq. 5).  Both run entirely in the CUDA library.
"""
from __future__ import annotations

import torch

from . import Mesh, params


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
    @staticmethod
    def forward(ctx, g: torch.Tensor, f: torch.Tensor, mesh: Mesh, p=None):
        u = mesh.inpaint(g.detach().contiguous(), p)
        r = (u - f).contiguous()
        ctx.mesh, ctx.p = mesh, p
        ctx.save_for_backward(r)
        return 0.5 * (r.double() ** 2).sum()

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (r,) = ctx.saved_tensors
        gbar = ctx.mesh.adjoint(r, ctx.p)
        return gbar * grad_out.to(gbar.dtype), None, None, None


__all__ = ["FemInpaint", "TonalLoss", "params"]
