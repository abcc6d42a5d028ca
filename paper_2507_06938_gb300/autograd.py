"""torch.autograd.Function over the adjoint gradient of f_obj.

``FObj.apply(thetas, ctx, model)`` returns f_obj for every row of ``thetas``
(CUDA float64, n_theta x dim(theta)); its backward multiplies the incoming
gradient by d f_obj / d theta computed in the forward pass by
``bta_fobj_grad`` (selected inverses + trace kernels, no finite differences).
Argument marshalling only: all arithmetic runs in libbta.
"""

from __future__ import annotations

import torch

from .bta import BtaContext, BtaModel


class FObj(torch.autograd.Function):
    @staticmethod
    def forward(fctx, thetas: torch.Tensor, ctx: BtaContext, model: BtaModel):
        th = thetas.detach().to(torch.float64).contiguous()
        if th.dim() == 1:
            th = th[None, :]
        f = torch.empty(th.shape[0], dtype=torch.float64, device=th.device)
        g = torch.empty_like(th)
        ctx.fobj_grad(model, th, f, g)
        ctx.sync()
        fctx.save_for_backward(g)
        fctx.squeeze = thetas.dim() == 1
        return f[0] if fctx.squeeze else f

    @staticmethod
    def backward(fctx, grad_f):
        (g,) = fctx.saved_tensors
        if fctx.squeeze:
            return grad_f * g[0], None, None
        return grad_f[:, None] * g, None, None


def fobj(thetas: torch.Tensor, ctx: BtaContext, model: BtaModel) -> torch.Tensor:
    """Differentiable f_obj(theta) (rows of thetas)."""
    return FObj.apply(thetas, ctx, model)
