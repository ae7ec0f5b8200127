"""Differentiable solve of the all-at-once optimality system.

``solve(solver, log_a, g, f=None, y0=None)`` returns x = A(a)^{-1} b(g, f, y0)
(Eq. main_system) for the nodal log-coefficient ``log_a`` on the interior
nodes (boundary nodes keep the values the solver was set up with) and the
target ``g``.  Forward: pc_set_coefficient, pc_build_rhs, pc_gmres_solve.
Backward (hand-written): the adjoint solve A^T lam = dL/dx (pc_adjoint_solve,
A^T = S A S), then

    dL/d log a_P = -lam^T (dA/d log a_P) x     (pc_grad_log_a, stencil derivative)
    dL/dg_j      = tau * lam1_j                 (b1_j = tau g_j)

Krylov bases are not kept between forward and backward: the adjoint solve
builds its own, so memory is that of one solve.
"""
from __future__ import annotations

import numpy as np
import torch

from .solver import Solver


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_a, g, solver, a_boundary, f, y0, rtol):
        d, m1 = solver.dim, solver.m1
        a_nodes = a_boundary.copy()
        a_nodes[(slice(1, -1),) * d] = np.exp(log_a.detach().cpu().numpy().reshape((m1,) * d))
        solver.set_coefficient(a_nodes)
        b = solver.build_rhs(f, g.detach().contiguous(), y0)
        x, iters, rel = solver.solve(b, rtol=rtol)
        ctx.solver = solver
        ctx.rtol = rtol
        ctx.save_for_backward(x)
        ctx.iters = iters
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        solver: Solver = ctx.solver
        lam, _, _ = solver.adjoint_solve(gx.contiguous(), rtol=ctx.rtol)
        grad_loga = solver.grad_log_a(x, lam)
        grad_g = solver.tau * lam[0]
        return grad_loga, grad_g, None, None, None, None, None


def solve(solver: Solver, log_a: torch.Tensor, g: torch.Tensor, a_nodes: np.ndarray,
          f: torch.Tensor | None = None, y0: torch.Tensor | None = None, rtol: float = 1e-10):
    """x(log_a, g) with gradients.  ``a_nodes`` supplies the boundary values of a."""
    return _Solve.apply(log_a, g, solver, np.array(a_nodes, dtype=np.float64), f, y0, rtol)


def objective(x: torch.Tensor, g: torch.Tensor, solver: Solver) -> torch.Tensor:
    """J_h = h^d tau [1/2 sum ||y - g||^2 + 1/(2 gamma) sum ||p||^2], y = x1/sqrt(gamma), p = x2."""
    h = 1.0 / (solver.m1 + 1)
    y = x[0] / solver.gamma ** 0.5
    p = x[1]
    return h ** solver.dim * solver.tau * (0.5 * ((y - g) ** 2).sum() + 0.5 / solver.gamma * (p ** 2).sum())
