"""Autograd wrappers: the backward of hierarchization is its transpose, run by
the library's adjoint kernels (the transpose of Alg. 1, Sec. 3); the backward
of dehierarchization is the transpose of the inverse."""
from __future__ import annotations

import torch

from . import transform, GBH_HIERARCHIZE, GBH_ADJOINT, GBH_DEHIERARCHIZE, GBH_DEHIERARCHIZE_ADJOINT


class HierarchizeFn(torch.autograd.Function):
    """alpha = H u for a grid tensor u (or a batch [B, N] of equal grids).

    forward : out-of-place hierarchization (the input is not modified)
    backward: grad_u = H^T grad_alpha, out of place
    """

    @staticmethod
    def forward(ctx, u, levels, **kw):
        ctx.levels = tuple(int(v) for v in levels)
        batch = u.shape[0] if u.dim() == 2 else None
        ctx.batch = batch
        out = u.detach().clone(memory_format=torch.contiguous_format)
        transform(out, ctx.levels, GBH_HIERARCHIZE, batch=batch)
        return out

    @staticmethod
    def backward(ctx, g):
        gi = g.detach().clone(memory_format=torch.contiguous_format)
        transform(gi, ctx.levels, GBH_ADJOINT, batch=ctx.batch)
        return gi, None


class DehierarchizeFn(torch.autograd.Function):
    """u = D alpha for a grid tensor alpha (or a batch [B, N] of equal grids).

    forward : out-of-place dehierarchization (the input is not modified)
    backward: grad_alpha = D^T grad_u, out of place
    """

    @staticmethod
    def forward(ctx, alpha, levels):
        ctx.levels = tuple(int(v) for v in levels)
        batch = alpha.shape[0] if alpha.dim() == 2 else None
        ctx.batch = batch
        out = alpha.detach().clone(memory_format=torch.contiguous_format)
        transform(out, ctx.levels, GBH_DEHIERARCHIZE, batch=batch)
        return out

    @staticmethod
    def backward(ctx, g):
        gi = g.detach().clone(memory_format=torch.contiguous_format)
        transform(gi, ctx.levels, GBH_DEHIERARCHIZE_ADJOINT, batch=ctx.batch)
        return gi, None


def hierarchize_ad(u, levels):
    """Differentiable hierarchization (functional form of HierarchizeFn)."""
    return HierarchizeFn.apply(u, levels)
