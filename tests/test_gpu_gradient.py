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
    x = pag.solve(sol, log_a, g, rtol=1e-12)
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
    x = pag.solve(sol, log_a, g, rtol=1e-13)
    J = pag.objective(x, g, sol)
    J.backward()
    ga, gg = log_a.grad.detach(), g.grad.detach()

    def J_at(la, gt):
        with torch.no_grad():
            xx = pag.solve(sol, la, gt, rtol=1e-13)
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


def _oracle_gradient(a_nodes, g, prob, n, gamma):
    tau, alpha = prob.tau, osy.alpha_weight(prob.T, n, gamma)
    b = osy.build_rhs(prob.f, g, prob.y0, tau, gamma)
    mg = opc.MGSpatialSolver(a_nodes, tau)
    ref = okr.gmres(lambda v: osy.apply_A(v, a_nodes, tau, alpha),
                    lambda v: opc.apply_Peps_inv(v, n, alpha, prob.eps, mg), b, rtol=1e-13, maxit=200)
    return ogr.envelope_gradient(ref.x, g, a_nodes, tau, gamma)


def test_two_forwards_then_backward_use_each_forwards_coefficient():
    # two samples through one Solver before one backward: each backward must use
    # the coefficient of its own forward; flat parameter tensors keep their shape
    from paper_2410_22686_gb300 import autograd as pag
    m1, n, gamma = 31, 32, 1e-3
    prob = S.gradient_problem(m1=m1, n=n, gamma=gamma)
    from paper_2410_22686_gb300 import Solver
    sol = Solver(2, m1, n, prob.T, gamma, prob.eps, prob.a_nodes, spatial="mg", precision="fp64", max_iter=120)
    la0 = np.log(prob.a_nodes[1:-1, 1:-1])
    la1 = la0 + 0.3 * S.random_vector((m1, m1), 7)
    las = [torch.from_numpy(v.ravel().copy()).cuda().requires_grad_(True) for v in (la0, la1)]
    gs = [torch.from_numpy(prob.g.copy()).cuda().requires_grad_(True) for _ in range(2)]
    xs = [pag.solve(sol, la, gg, rtol=1e-12) for la, gg in zip(las, gs)]
    J = pag.objective(xs[0], gs[0], sol) + pag.objective(xs[1], gs[1], sol)
    J.backward()
    for la, gg, lv in zip(las, gs, (la0, la1)):
        assert la.grad.shape == la.shape and gg.grad.shape == gg.shape
        a_nodes = prob.a_nodes.copy()
        a_nodes[1:-1, 1:-1] = np.exp(lv)
        ea, eg = _oracle_gradient(a_nodes, prob.g, prob, n, gamma)
        ga = la.grad.cpu().numpy().reshape(m1, m1)
        assert np.abs(ga - ea).max() <= 1e-8 * np.abs(ea).max()
        assert np.abs(gg.grad.cpu().numpy() - eg).max() <= 1e-8 * np.abs(eg).max()
    sol.close()


def test_objective_and_its_gradient_match_oracle():
    from paper_2410_22686_gb300 import Solver
    m1, n, gamma = 15, 8, 1e-3
    prob = S.gradient_problem(m1=m1, n=n, gamma=gamma)
    sol = Solver(2, m1, n, prob.T, gamma, prob.eps, prob.a_nodes, spatial="mg", precision="fp64", max_iter=4)
    xh = S.random_vector((2, n, m1, m1), 11)
    x, g = torch.from_numpy(xh).cuda(), torch.from_numpy(prob.g).cuda()
    J = sol.objective(x, g).item()
    ref = ogr.objective(xh, prob.g, prob.tau, gamma)
    assert abs(J - ref) <= 1e-13 * abs(ref)
    gJ = torch.tensor(2.5, dtype=torch.float64, device="cuda")
    gx, gg = sol.objective_grad(x, g, gJ)
    rx = 2.5 * ogr.objective_grad_x(xh, prob.g, prob.tau, gamma)
    assert np.abs(gx.cpu().numpy() - rx).max() <= 1e-13 * np.abs(rx).max()
    h = 1.0 / (m1 + 1)
    rg = -2.5 * h ** 2 * prob.tau * (xh[0] / gamma ** 0.5 - prob.g)
    assert np.abs(gg.cpu().numpy() - rg).max() <= 1e-13 * np.abs(rg).max()
    sol.close()


def test_set_log_coefficient_equals_setup_with_the_same_values():
    # a = exp(log a) on the device rebuilds every level's stencil as pc_setup does;
    # a handle set up with the same nodal values (exp taken on the host) agrees to rounding
    from paper_2410_22686_gb300 import Solver
    for d, m1, n, prec in [(2, 31, 16, "fp64"), (2, 63, 8, "fp32"), (3, 15, 8, "fp64")]:
        a0 = np.exp(0.3 * S.random_vector((m1 + 2,) * d, 1))
        la = 0.4 * S.random_vector((m1,) * d, 2)
        a1 = a0.copy()
        a1[(slice(1, -1),) * d] = np.exp(la)
        s1 = Solver(d, m1, n, 1.0, 1e-3, 0.3, a0, spatial="mg", precision=prec)
        s2 = Solver(d, m1, n, 1.0, 1e-3, 0.3, a1, spatial="mg", precision=prec)
        s1.set_log_coefficient(torch.from_numpy(la).cuda())
        v = torch.from_numpy(S.random_vector((2, n) + (m1,) * d, 3)).cuda()
        for f in (lambda s: s.matvec(v), lambda s: s.apply_precond(v)):
            r1, r2 = f(s1), f(s2)
            err = (r1 - r2).abs().max().item() / r2.abs().max().item()
            assert err <= (1e-12 if prec == "fp64" else 1e-5), (d, m1, prec, err)
        s1.close()
        s2.close()


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
