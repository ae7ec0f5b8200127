"""Differentiation through the solve (autograd Function over the C ABI):
gradients of J_h with respect to the nodal log-coefficient and the target,
against the oracle's FP64 gradient and against central finite differences."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import gradient as ogr, krylov as okr, precond as opc, system as osy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_22686_gb300 import build
    build.build()


def _setup(m1, n, gamma, precision="fp64", max_iter=120):
    from paper_2410_22686_gb300 import Solver
    prob = S.gradient_problem(m1=m1, n=n, gamma=gamma)
    sol = Solver(2, m1, n, prob.T, gamma, prob.eps, prob.a_nodes, spatial="mg", precision=precision,
                 max_iter=max_iter)
    log_a = torch.from_numpy(np.log(prob.a_nodes[1:-1, 1:-1]).copy()).cuda().requires_grad_(True)
    g = torch.from_numpy(prob.g).cuda().requires_grad_(True)
    return prob, sol, log_a, g


def test_autograd_gradient_matches_oracle_fp64_gradient():
    from paper_2410_22686_gb300 import autograd as pag
    m1, n, gamma = 63, 64, 1e-4
    prob, sol, log_a, g = _setup(m1, n, gamma)
    x = pag.solve(sol, log_a, g, prob.a_nodes, rtol=1e-12)
    J = pag.objective(x, g, sol)
    J.backward()
    ga, gg = log_a.grad.cpu().numpy(), g.grad.cpu().numpy()
    # oracle: its own solve, then the envelope (Lagrangian) closed form
    tau, alpha = prob.tau, osy.alpha_weight(prob.T, n, gamma)
    b = osy.build_rhs(prob.f, prob.g, prob.y0, tau, gamma)
    mg = opc.MGSpatialSolver(prob.a_nodes, tau)
    ref = okr.gmres(lambda v: osy.apply_A(v, prob.a_nodes, tau, alpha),
                    lambda v: opc.apply_Peps_inv(v, n, alpha, prob.eps, mg), b, rtol=1e-13, maxit=200)
    ea, eg = ogr.envelope_gradient(ref.x, prob.g, prob.a_nodes, tau, gamma)
    assert np.abs(ga - ea).max() <= 1e-8 * np.abs(ea).max()
    assert np.abs(gg - eg).max() <= 1e-8 * np.abs(eg).max()
    assert abs(J.item() - ogr.objective(ref.x, prob.g, tau, gamma)) <= 1e-10 * abs(J.item())
    sol.close()


def test_gradient_central_differences_at_127_squared_n128():
    # 127^2 nodal parameters and the target, 32 seeded random directions, step 1e-6
    from paper_2410_22686_gb300 import autograd as pag
    m1, n, gamma = 127, 128, 1e-4
    prob, sol, log_a, g = _setup(m1, n, gamma)
    x = pag.solve(sol, log_a, g, prob.a_nodes, rtol=1e-13)
    J = pag.objective(x, g, sol)
    J.backward()
    ga, gg = log_a.grad.detach(), g.grad.detach()

    def J_at(la, gt):
        with torch.no_grad():
            xx = pag.solve(sol, la, gt, prob.a_nodes, rtol=1e-13)
            return pag.objective(xx, gt, sol).item()

    rng = np.random.default_rng(2410)
    h = 1e-6
    worst = 0.0
    for _ in range(32):
        da = torch.from_numpy(rng.standard_normal((m1, m1))).cuda()
        dg = torch.from_numpy(rng.standard_normal(prob.g.shape)).cuda()
        fd = (J_at(log_a.detach() + h * da, g.detach() + h * dg)
              - J_at(log_a.detach() - h * da, g.detach() - h * dg)) / (2 * h)
        an = float((ga * da).sum() + (gg * dg).sum())
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst <= 1e-5, worst
    sol.close()


def test_set_coefficient_equals_fresh_setup():
    from paper_2410_22686_gb300 import Solver
    m1, n = 31, 16
    a1 = np.exp(0.3 * S.random_vector((m1 + 2, m1 + 2), 1))
    a2 = np.exp(0.3 * S.random_vector((m1 + 2, m1 + 2), 2))
    s1 = Solver(2, m1, n, 1.0, 1e-3, 0.3, a1, spatial="mg")
    s2 = Solver(2, m1, n, 1.0, 1e-3, 0.3, a2, spatial="mg")
    s1.set_coefficient(a2)
    v = torch.from_numpy(S.random_vector((2, n, m1, m1), 3)).cuda()
    assert torch.equal(s1.matvec(v), s2.matvec(v))
    assert torch.equal(s1.apply_precond(v), s2.apply_precond(v))
    s1.close()
    s2.close()
