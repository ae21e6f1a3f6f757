"""torch.autograd wrapper of the effective stiffness (argument marshalling only).

``effective_stiffness(solver, L, lame, scale)`` returns C_eff (6x6, float64, Mandel) as a torch
tensor that is differentiable with respect to ``lame`` (4: lambda_minus, mu_minus, lambda_plus,
mu_plus) and the per-voxel modulus scale ``scale`` (N float32).  The forward pass is
``xfft_set_microstructure`` + ``xfft_effective_stiffness``; the backward pass is ``xfft_grad``,
the library's adjoint kernels (the operator is symmetric, so the six converged load cases serve
as their own adjoints; dC_kl/dtheta = (1/|Y|) int eps_k : dC/dtheta : eps_l).
"""
from __future__ import annotations

import numpy as np
import torch


class EffectiveStiffness(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lame, scale, solver, L):
        lm = lame.detach().to("cpu", torch.float64).numpy()
        sc = None if scale is None else scale.detach().to("cpu", torch.float32).numpy()
        solver.set_microstructure(L, (float(lm[0]), float(lm[1])), (float(lm[2]), float(lm[3])), sc)
        C, st = solver.effective_stiffness()
        if not st.get("converged", True):
            raise RuntimeError("effective stiffness solve did not converge: %r" % (st,))
        ctx.solver = solver
        ctx.want_scale = scale is not None and scale.requires_grad
        ctx.scale_device = scale.device if scale is not None else None
        return torch.as_tensor(np.asarray(C), dtype=torch.float64, device=lame.device)

    @staticmethod
    def backward(ctx, gC):
        G = gC.detach().to("cpu", torch.float64).numpy()
        dl, ds, _ = ctx.solver.grad(G, scale_grad=ctx.want_scale)
        g_lame = torch.as_tensor(dl, dtype=gC.dtype, device=gC.device)
        g_scale = torch.as_tensor(ds).to(ctx.scale_device) if ctx.want_scale else None
        return g_lame, g_scale, None, None


def effective_stiffness(solver, L, lame, scale=None):
    """Differentiable C_eff(lame, scale) of the microstructure with nodal level set L."""
    return EffectiveStiffness.apply(lame, scale, solver, L)
