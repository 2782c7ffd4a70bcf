"""Differentiable GLRM objective (Section 7.2 "Gradient method": the gradient
of sum_Omega L_j(x_i . y_j, A_ij) with respect to x_i is
sum_j L_j'(x_i . y_j, A_ij) y_j, and likewise for y_j).

GLRMObjective.apply(X, Yt, model) returns the objective of eq. gpca at the
factors X (m x k) and Yt (n x k) as a float64 scalar tensor, computed by the
library's objective kernels; its backward calls the library's gradient
kernels, which recompute the residuals from the saved factors (nothing of
size |Omega| is stored between forward and backward) and multiply by the
incoming derivative on the device.  Regulariser gradients are included
(quadratic: 2 w x, l1: w sign(x)); the nonnegativity indicator has none.
"""
from __future__ import annotations

import torch

from . import glrm as G


class GLRMObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Yt, model):
        X = X.contiguous()
        Yt = Yt.contiguous()
        out = torch.empty(1, dtype=torch.float64, device=X.device)
        G.glrm_objective_at(model.h, X, Yt, out)
        ctx.save_for_backward(X, Yt)
        ctx.model = model
        return out[0]

    @staticmethod
    def backward(ctx, dout):
        X, Yt = ctx.saved_tensors
        gx = torch.empty_like(X) if ctx.needs_input_grad[0] else None
        gy = torch.empty_like(Yt) if ctx.needs_input_grad[1] else None
        if gx is None and gy is None:
            return None, None, None
        scale = dout.detach().to(torch.float64).reshape(1).contiguous()
        # both gradients come from one call; a buffer stands in for the one not needed
        G.glrm_grad_at(ctx.model.h, X, Yt, gx if gx is not None else torch.empty_like(X),
                       gy if gy is not None else torch.empty_like(Yt), True, scale)
        return gx, gy, None


def glrm_objective(X, Yt, model) -> torch.Tensor:
    """Objective of eq. gpca at (X, Yt) for the observed set and losses held by
    `model` (a glrm.GLRM), differentiable in X and Yt."""
    return GLRMObjective.apply(X, Yt, model)
