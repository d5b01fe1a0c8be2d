"""torch.autograd wrapper: u = EXCMG(f, g), with gradients through the discrete solve.

Forward: excmg_solve (Algorithm 1).  Backward: excmg_adjoint, the exact transpose of the
discrete map (f, g) -> u of the compact scheme (eq. compact / FD):
    lambda = A^{-1} (dL/du)_I,   dL/df = -R^T lambda,   dL/dg = LHS_IB^T lambda + (dL/du)_B,
with R the 7-point right-hand-side operator and LHS_IB the boundary columns of the
printed left-hand side.  Both directions run in the CUDA library; torch only supplies
the tensors and the stream.
"""
from __future__ import annotations

import torch

from . import excmg as X


class ExcmgSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, g, L, N0, opts):
        opts = dict(opts or {})
        res = X.solve(f.contiguous(), g.contiguous(), L, N0, **opts)
        ctx.L = tuple(L)
        adj = {k: v for k, v in opts.items() if k in ("precision", "eps", "max_iter", "inner_tol",
                                                       "max_refine", "tile_z", "chunk")}
        adj.setdefault("eps", 1e-12)
        ctx.adj_opts = adj
        return res["u"]

    @staticmethod
    def backward(ctx, dLdu):
        dLdf, dLdg, _ = X.adjoint(dLdu.contiguous(), ctx.L, **ctx.adj_opts)
        return dLdf, dLdg, None, None, None


def excmg_solve(f, g, L, N0, **opts):
    """Differentiable EXCMG solve: u = excmg_solve(f, g, L, N0, eps=..., ...)."""
    return ExcmgSolve.apply(f, g, L, N0, opts)
