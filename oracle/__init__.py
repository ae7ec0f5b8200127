"""Plain FP64 CPU oracle for the all-at-once parabolic optimal-control solver.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
reference that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
reference-arm legs) may import it.  The product path never routes through it,
and it shares no code with the CUDA library (``paper_2410_22686_gb300``):
neither side imports the other; both take their inputs from ``synthetic``.

Modules (each function cites the passage of the paper it follows):

* ``system``   -- grid, stencil K, T, A, A^T, the unscaled KKT matrix, RHS,
                  end-point solves, error measure e_h         (Section 1, Section 3)
* ``precond``  -- C_{eps,n}, its diagonalisation, dense P / P_eps, the four-step
                  apply of P_eps^{-1}, FST and multigrid spatial solvers
                                                             (Eq. matrix_P_eps, Section 2.1)
* ``krylov``   -- GMRES (left preconditioned) and flexible GMRES (right)
                                                             (Lemma 2.1, Section 3)
* ``gradient`` -- discrete objective, envelope and adjoint gradients
* ``fe``       -- bilinear / trilinear finite elements (mass matrix M, constant a):
                  M, K, the operator, right-hand side, end points and
                  mass-scaled sine-transform solves            (Section 1, the M != I case)
"""
from . import system, precond, krylov, gradient, fe  # noqa: F401
