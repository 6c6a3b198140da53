"""TTIE energy as a torch.autograd.Function (argument marshalling around libttie).

``TTIEnergy(tri)(x)`` returns sum T over the intersecting pairs of the mesh at x (Eq. 2).
Its backward is the library's gradient (Eq. 3, assembled per vertex); the backward of that
backward is the library's exact Hessian-vector product (forward-mode dual numbers through
the per-pair gradient), so double backward, gradgradcheck and Newton-Krylov methods work.
Every quantity is computed by the CUDA kernels; this module only routes tensors.
"""
from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable

from . import ttie


class TTIEnergy:
    """Differentiable energy of a mesh with fixed topology (tri, optional group)."""

    def __init__(self, tri: torch.Tensor, group: torch.Tensor | None = None, precision: int = ttie.F32, **params):
        self.ctx = ttie.Context(precision=precision, **params)
        self.tri = tri.contiguous()
        self.group = group.contiguous() if group is not None else None
        self.last = None   # (n_candidates, n_active) of the latest forward

    def _evaluate(self, x: torch.Tensor, grad: torch.Tensor | None):
        self.ctx.build_bvh(x, self.tri, self.group)
        what = ttie.EVAL_E | ttie.EVAL_H | (ttie.EVAL_G if grad is not None else 0)
        return self.ctx.eval_pairs(x, what, grad=grad)

    def __call__(self, x: torch.Tensor) -> torch.Tensor:
        return _Energy.apply(x, self)


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, mod):
        xd = x.detach().contiguous()
        g = torch.empty_like(xd)
        E, n_act = mod._evaluate(xd, g)
        mod.last = n_act
        ctx.mod = mod
        ctx.save_for_backward(x, g)   # x itself, so the gradient stays differentiable in x
        return torch.tensor(E, dtype=x.dtype, device=x.device)

    @staticmethod
    def backward(ctx, gE):
        x, g = ctx.saved_tensors
        return _Gradient.apply(x, g, gE, ctx.mod), None


class _Gradient(torch.autograd.Function):
    """gE * grad E(x); differentiable once more through the exact Hessian-vector product."""

    @staticmethod
    def forward(ctx, x, g, gE, mod):
        ctx.mod = mod
        ctx.save_for_backward(x, g, gE)
        return gE * g

    @staticmethod
    @once_differentiable
    def backward(ctx, w):
        x, g, gE = ctx.saved_tensors
        mod = ctx.mod
        xd = x.detach().contiguous()
        mod._evaluate(xd, None)   # the context's state must be the evaluation at x
        hv = mod.ctx.hvp(xd, w.contiguous().to(x.dtype), exact=True)
        return gE * hv, None, (w * g).sum(), None
