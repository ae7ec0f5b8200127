"""Differentiable solve of the all-at-once optimality system.

``solve(solver, log_a, g, f=None, y0=None)`` returns x = A(a)^{-1} b(g, f, y0)
(Eq. main_system) for the nodal log-coefficient ``log_a`` on the interior
nodes (boundary nodes keep the values the solver holds) and the target ``g``.
Forward: pc_set_log_coefficient (a = exp(log_a) on the device),
pc_build_rhs, pc_gmres_solve.  Backward (hand-written): the forward's
coefficient is set again (another forward on the same solver may have
changed it), then the adjoint solve A^T lam = dL/dx (pc_adjoint_solve,
A^T = S A S), and

    dL/d log a_P = -lam^T (dA/d log a_P) x     (pc_grad_log_a, stencil derivative)
    dL/dg_j      = tau * lam1_j                 (pc_grad_g; b1_j = tau g_j)

``objective(x, g, solver)`` is the discrete tracking objective J_h
(pc_objective) with its gradient (pc_objective_grad).  This module only
marshals tensors: every value is computed by the library's kernels.

Krylov bases are not kept between forward and backward: the adjoint solve
builds its own, so memory is that of one solve.
"""
from __future__ import annotations

import torch

from .solver import Solver


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_a, g, solver, f, y0, rtol):
        la = log_a.detach().contiguous().clone()
        solver.set_log_coefficient(la)
        b = solver.build_rhs(f, g.detach().contiguous(), y0)
        x, iters, rel = solver.solve(b, rtol=rtol)
        ctx.solver = solver
        ctx.rtol = rtol
        ctx.log_a = la
        ctx.shapes = (log_a.shape, g.shape)
        ctx.save_for_backward(x)
        ctx.iters = iters
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        solver: Solver = ctx.solver
        solver.set_log_coefficient(ctx.log_a)
        lam, _, _ = solver.adjoint_solve(gx.contiguous(), rtol=ctx.rtol)
        grad_loga = solver.grad_log_a(x, lam).view(ctx.shapes[0])
        grad_g = solver.grad_g(lam).view(ctx.shapes[1])
        return grad_loga, grad_g, None, None, None, None


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, g, solver):
        xd, gd = x.detach().contiguous(), g.detach().contiguous()
        ctx.solver = solver
        ctx.save_for_backward(xd, gd)
        return solver.objective(xd, gd)

    @staticmethod
    def backward(ctx, gJ):
        xd, gd = ctx.saved_tensors
        gx, gg = ctx.solver.objective_grad(xd, gd, gJ.detach().contiguous())
        return gx.view(xd.shape), gg.view(gd.shape), None


def solve(solver: Solver, log_a: torch.Tensor, g: torch.Tensor, f: torch.Tensor | None = None,
          y0: torch.Tensor | None = None, rtol: float = 1e-10):
    """x(log_a, g) with gradients; log_a and g are float64 CUDA tensors."""
    return _Solve.apply(log_a, g, solver, f, y0, rtol)


def objective(x: torch.Tensor, g: torch.Tensor, solver: Solver) -> torch.Tensor:
    """J_h = h^d tau [1/2 sum ||y - g||^2 + 1/(2 gamma) sum ||p||^2], y = x1/sqrt(gamma), p = x2."""
    return _Objective.apply(x, g, solver)
