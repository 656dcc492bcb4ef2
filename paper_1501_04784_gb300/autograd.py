"""K(X, c) as a differentiable torch operation.

forward: fem_build_K (values of the lower-CSR K on the mesh's cached pattern);
backward: fem_vjp, which recomputes J and B from X instead of storing them.
The upstream gradient G has K's pattern; L = sum over stored entries G_ij K_ij.
"""
from __future__ import annotations

import torch

from .fem import Mesh, value_dtype


class BuildK(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, c, mesh: Mesh, prec: str):
        vals = mesh.build_K(X.detach().contiguous(), c.detach().contiguous(), prec)
        ctx.save_for_backward(X, c)
        ctx.mesh = mesh
        ctx.prec = prec
        return vals

    @staticmethod
    def backward(ctx, gvals):
        X, c = ctx.saved_tensors
        G = gvals.detach().to(value_dtype(ctx.prec)).contiguous()
        dX, dc = ctx.mesh.vjp(X.detach().contiguous(), c.detach().contiguous(), G, ctx.prec)
        return dX.to(X.dtype), dc.to(c.dtype), None, None


def build_K(mesh: Mesh, X: torch.Tensor, c: torch.Tensor, prec: str = "fp64") -> torch.Tensor:
    """Differentiable build of K's values with respect to X and c."""
    if mesh.nnz is None:
        mesh.pattern()
    return BuildK.apply(X, c, mesh, prec)
