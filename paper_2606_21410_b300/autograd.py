"""Differentiable solve and derivative for PyTorch autograd.

``solve(plan, K, b)`` returns u with A(K) u = b; its backward runs the
discrete adjoint solve A^T lam = dJ/du (``cheb_adjoint_solve``) and returns
dJ/db = lam and dJ/dK = sum_a (D_a^T P_int lam) * (D_a u) (plus the flux-row
term where a face carries flux data).  ``solve_hierarchy(plans, K, b)`` is
the same for the hierarchical solve (Alg. 4) from the finest level's data:
the forward pass recomputes the coarse levels by injection and stores
nothing of them; the converged fine solution does not depend on them, so the
backward pass is the fine-level adjoint solve.  ``deriv(plan, u,
axis)`` is the line derivative D_a u with backward D_a^T (``cheb_deriv_t``),
so objectives such as boundary fluxes K d_x u differentiate end to end.
All arithmetic runs in the library's CUDA kernels.
"""
from __future__ import annotations

import torch


class ChebSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, K, b, opts):
        u, info = plan.solve(K.detach().contiguous(), b.detach().contiguous(), **opts)
        ctx.plan, ctx.opts = plan, opts
        ctx.info = info
        ctx.save_for_backward(K, u)
        return u

    @staticmethod
    def backward(ctx, gu):
        K, u = ctx.saved_tensors
        dK = torch.zeros_like(K) if ctx.needs_input_grad[1] else None
        lam, dK, _ = ctx.plan.adjoint_solve(K.detach().contiguous(), gu.contiguous(), u=u, dJdK=dK,
                                            **ctx.opts)
        return None, dK, (lam if ctx.needs_input_grad[2] else None), None


class ChebHierarchySolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plans, K, b, opts):
        from . import solve_hierarchy_fine
        u, infos, eref = solve_hierarchy_fine(plans, K.detach().contiguous(), b.detach().contiguous(), **opts)
        ctx.plan, ctx.opts = plans[-1], opts
        ctx.infos, ctx.eref = infos, eref
        ctx.save_for_backward(K, u)
        return u

    @staticmethod
    def backward(ctx, gu):
        K, u = ctx.saved_tensors
        dK = torch.zeros_like(K) if ctx.needs_input_grad[1] else None
        lam, dK, _ = ctx.plan.adjoint_solve(K.detach().contiguous(), gu.contiguous(), u=u, dJdK=dK,
                                            **ctx.opts)
        return None, dK, (lam if ctx.needs_input_grad[2] else None), None


class ChebDeriv(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, u, axis):
        ctx.plan, ctx.axis = plan, axis
        return plan.deriv(u.contiguous(), axis)

    @staticmethod
    def backward(ctx, g):
        return None, ctx.plan.deriv(g.contiguous(), ctx.axis, transpose=True), None


def solve(plan, K: torch.Tensor, b: torch.Tensor, **opts) -> torch.Tensor:
    """u = A(K)^{-1} b, differentiable in K and b (FP64 CUDA tensors)."""
    return ChebSolve.apply(plan, K, b, opts)


def solve_hierarchy(plans, K: torch.Tensor, b: torch.Tensor, **opts) -> torch.Tensor:
    """Fine solution of the hierarchical solve from the finest K and b
    (coarse levels recomputed by injection), differentiable in K and b."""
    return ChebHierarchySolve.apply(plans, K, b, opts)


def deriv(plan, u: torch.Tensor, axis: int) -> torch.Tensor:
    """d u / d t_axis, differentiable."""
    return ChebDeriv.apply(plan, u, axis)
