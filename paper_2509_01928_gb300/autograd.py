"""torch.autograd.Function over the adjoint kernels (ising_backward).

DochRelaxedEnergy(x0, alpha) returns the mean relaxed energy of the final
DOCH iterates, L = (1/R) sum_r (-1/2 x_r^T J x_r - h^T x_r) at x^(N), with
x^(k+1) = cbrt((J x^(k) + alpha_k x^(k) + h) / beta) (Eq. FPE with an
attraction-weight schedule alpha_k). Its backward returns dL/dx0 and
dL/dalpha from the library's hand-written adjoint (checkpoint every
`ckpt_every` steps and recompute). The library computes the loss and both
gradients in one call, so the forward pass runs that call and keeps the
gradients for backward.
"""
from __future__ import annotations

import torch

from . import _native


class DochRelaxedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, alpha, handle, beta, ckpt_every):
        iters = int(alpha.numel())
        x0c = x0.detach().contiguous()
        ga = torch.empty(iters, dtype=torch.float64, device=x0.device)
        gx = torch.empty_like(x0c)
        loss = torch.empty(1, dtype=torch.float64, device=x0.device)
        _native.ising_backward(handle, x0c, alpha.detach().double().cpu().numpy(), float(beta), iters,
                               int(ckpt_every), grad_alpha=ga, grad_x0=gx, loss=loss)
        ctx.save_for_backward(ga, gx)
        ctx.alpha_dtype = alpha.dtype
        ctx.alpha_device = alpha.device
        return loss[0]

    @staticmethod
    def backward(ctx, gout):
        ga, gx = ctx.saved_tensors
        g_x0 = (gout.to(gx.dtype) * gx) if ctx.needs_input_grad[0] else None
        g_alpha = (gout * ga).to(dtype=ctx.alpha_dtype, device=ctx.alpha_device) if ctx.needs_input_grad[1] else None
        return g_x0, g_alpha, None, None, None


def relaxed_energy(x0, alpha, handle, beta, ckpt_every=20):
    """Mean relaxed energy after len(alpha) DOCH steps, differentiable in x0 and alpha."""
    return DochRelaxedEnergy.apply(x0, alpha, handle, beta, ckpt_every)
