"""Trilinear elements with a nodal coefficient on the GPU (k_fevar3.cu) against the
oracle (oracle/fe.py, any dimension): the 27-point element product, the eight-colour
element multigrid inside P_eps^{-1}, GMRES solutions and end-point solves, the
objective and the gradients."""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from oracle import fe, krylov as okr, precond as opc, system as osy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_22686_gb300 import build
    build.build()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


def _coef(m1, seed, amp=0.5):
    return np.exp(amp * S.random_vector((m1 + 2,) * 3, seed))


def _solver(m1, n, a, precision="fp64", gamma=1e-3, eps=0.3, max_iter=80):
    from paper_2410_22686_gb300 import Solver
    return Solver(3, m1, n, 1.0, gamma, eps, a, spatial="mg", precision=precision, max_iter=max_iter, space="fe",
                  tiles=None)


@pytest.mark.parametrize("m1,n", [(1, 3), (3, 5), (7, 8), (15, 4)])
def test_element_product_and_transpose_match_oracle_3d(m1, n):
    a = _coef(m1, 1)
    sol = _solver(m1, n, a)
    M, K = fe.fe_matrices_var(a)
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, 1e-3)
    x = S.random_vector((2, n, m1, m1, m1), 2)
    assert _rel(sol.matvec(_dev(x)).cpu().numpy(), fe.apply_A(x, M, K, tau, alpha)) <= 1e-12
    assert _rel(sol.matvec(_dev(x), transpose=True).cpu().numpy(), fe.apply_AT(x, M, K, tau, alpha)) <= 1e-12
    x32 = x.astype(np.float32)
    y32 = sol.matvec_f32(torch.from_numpy(x32).cuda()).cpu().numpy()
    assert _rel(y32, fe.apply_A(x32.astype(np.float64), M, K, tau, alpha)) <= 1e-12
    sol.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("m1,n", [(1, 4), (3, 8), (7, 5), (15, 16)])
def test_element_multigrid_preconditioner_matches_oracle_3d(precision, tol, m1, n):
    a = _coef(m1, 3)
    gamma, eps = 1e-3, 0.3
    sol = _solver(m1, n, a, precision=precision, gamma=gamma, eps=eps, max_iter=4)
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    v = S.random_vector((2, n, m1, m1, m1), 4)
    ref = opc.apply_Peps_inv(v, n, alpha, eps, fe.MGSpatialSolverFE(a, tau))
    assert _rel(sol.apply_precond(_dev(v)).cpu().numpy(), ref) <= tol
    sol.close()


@pytest.mark.parametrize("precision,rtol,tol", [("fp64", 1e-11, 1e-10), ("mixed", 1e-10, 1e-7)])
def test_element_solve_and_end_points_match_oracle_3d(precision, rtol, tol):
    m1, n, gamma = 7, 8, 1e-3
    eps = math.sqrt(osy.time_step(1.0, n))
    a = _coef(m1, 5)
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    M, K = fe.fe_matrices_var(a)
    sh = (m1, m1, m1)
    f = S.random_vector((n,) + sh, 6)
    g = S.random_vector((n,) + sh, 7)
    y0 = S.random_vector(sh, 8)
    b_ref = fe.build_rhs(f, g, y0, tau, gamma, M)
    mg = fe.MGSpatialSolverFE(a, tau)
    ref = okr.gmres(lambda v: fe.apply_A(v, M, K, tau, alpha), lambda v: opc.apply_Peps_inv(v, n, alpha, eps, mg),
                    b_ref, rtol=1e-13, maxit=200, mode="right")
    assert ref.converged
    sol = _solver(m1, n, a, precision=precision, gamma=gamma, eps=eps)
    b = sol.build_rhs(_dev(f), _dev(g), _dev(y0))
    assert _rel(b.cpu().numpy(), b_ref) <= 1e-13
    x, it, rr = sol.solve(b, rtol=rtol)
    assert rr <= rtol
    xg = x.cpu().numpy().reshape(b_ref.shape)
    assert np.linalg.norm(xg - ref.x.reshape(b_ref.shape)) <= tol * np.linalg.norm(ref.x)
    if precision == "fp64":  # iteration counts of the same Krylov process
        ref_it = okr.gmres(lambda v: fe.apply_A(v, M, K, tau, alpha),
                           lambda v: opc.apply_Peps_inv(v, n, alpha, eps, mg),
                           b_ref, rtol=rtol, maxit=200, mode="right").iters
        assert abs(it - ref_it) <= 1, (it, ref_it)
    fT, g0 = S.random_vector(sh, 9), S.random_vector(sh, 10)
    yN, p0, _ = sol.end_point_solves(x, f_T=_dev(fT), g_0=_dev(g0), y0=_dev(y0), rtol=1e-13)
    y, p = osy.unscale(xg, gamma)
    yN_ref, p0_ref = fe.end_point_solves(y, p, M, K, tau, gamma, fT, g0, y0)
    assert _rel(yN.cpu().numpy(), yN_ref) <= 1e-10
    assert _rel(p0.cpu().numpy(), p0_ref) <= 1e-10
    sol.close()


def test_new_coefficient_equals_fresh_setup_3d():
    m1, n = 7, 4
    a1, a2 = _coef(m1, 11), _coef(m1, 12)
    s1, s2 = _solver(m1, n, a1), _solver(m1, n, a2)
    v = _dev(S.random_vector((2, n, m1, m1, m1), 13))
    s1.set_coefficient(a2)
    assert torch.equal(s1.matvec(v), s2.matvec(v))
    assert torch.equal(s1.apply_precond(v), s2.apply_precond(v))
    # log-coefficient on the device: interior nodes exp(log a), boundary kept
    a3 = a1.copy()
    la = 0.4 * S.random_vector((m1, m1, m1), 14)
    a3[1:-1, 1:-1, 1:-1] = np.exp(la)
    s3 = _solver(m1, n, a3)
    s1.set_coefficient(a1)
    s1.set_log_coefficient(_dev(la))
    for fn in (lambda s: s.matvec(v), lambda s: s.apply_precond(v)):
        r1, r3 = fn(s1), fn(s3)
        assert (r1 - r3).abs().max().item() <= 1e-12 * r3.abs().max().item()
    for s in (s1, s2, s3):
        s.close()


def test_element_objective_and_its_gradient_match_oracle_3d():
    m1, n, gamma = 7, 4, 1e-3
    a = _coef(m1, 15)
    sol = _solver(m1, n, a, gamma=gamma)
    M, _ = fe.fe_matrices_var(a)
    tau = osy.time_step(1.0, n)
    sh = (m1, m1, m1)
    xh = S.random_vector((2, n) + sh, 16)
    gh = S.random_vector((n,) + sh, 17)
    x, g = _dev(xh), _dev(gh)
    J = sol.objective(x, g).item()
    ref = fe.objective(xh, gh, M, tau, gamma)
    assert abs(J - ref) <= 1e-13 * abs(ref)
    gJ = torch.tensor(1.5, dtype=torch.float64, device="cuda")
    gx, gg = sol.objective_grad(x, g, gJ)
    assert _rel(gx.cpu().numpy().reshape(xh.shape), 1.5 * fe.objective_grad_x(xh, gh, M, tau, gamma)) <= 1e-13
    y, _ = osy.unscale(xh, gamma)
    assert _rel(gg.cpu().numpy().reshape(gh.shape), -1.5 * tau * fe._apply(M, y - gh)) <= 1e-13
    lam = S.random_vector((2, n) + sh, 18)
    gl = sol.grad_g(_dev(lam)).cpu().numpy().reshape(gh.shape)
    assert _rel(gl, tau * fe._apply(M, lam[0])) <= 1e-13
    # the stiffness derivative of the gradient against the oracle's, on any x and lam
    ga = sol.grad_log_a(x, _dev(lam)).cpu().numpy().reshape(sh)
    ref_ga, _ = fe.adjoint_gradient(xh, lam, gh, a, M, tau, gamma)
    assert _rel(ga, ref_ga) <= 1e-12
    sol.close()


def test_element_gradient_matches_oracle_3d():
    """dJ*/d log a and dJ*/dg through the autograd layer (adjoint solve and stiffness
    derivative on the GPU) against the oracle's envelope gradient at its own optimum."""
    from paper_2410_22686_gb300 import autograd as pag
    m1, n, gamma = 7, 8, 1e-3
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    eps = math.sqrt(tau)
    a = _coef(m1, 19)
    sh = (m1, m1, m1)
    f = S.random_vector((n,) + sh, 20)
    gh = S.random_vector((n,) + sh, 21)
    y0 = S.random_vector(sh, 22)
    sol = _solver(m1, n, a, precision="fp64", gamma=gamma, eps=eps, max_iter=120)
    la = torch.from_numpy(np.log(a[1:-1, 1:-1, 1:-1]).copy()).cuda().requires_grad_(True)
    g = _dev(gh).requires_grad_(True)
    x = pag.solve(sol, la, g, f=_dev(f), y0=_dev(y0), rtol=1e-12)
    M, K = fe.fe_matrices_var(a)
    b_ref = fe.build_rhs(f, gh, y0, tau, gamma, M)
    ref = okr.gmres(lambda v: fe.apply_A(v, M, K, tau, alpha),
                    lambda v: opc.apply_Peps_inv(v, n, alpha, eps, fe.DenseSpatialSolverFE(M, K, tau, sh)),
                    b_ref, rtol=1e-13, maxit=200, mode="right")
    ea, eg = fe.envelope_gradient(ref.x.reshape(b_ref.shape), gh, a, M, tau, gamma)
    J = pag.objective(x, g, sol)
    J.backward()
    assert np.abs(la.grad.cpu().numpy() - ea).max() <= 1e-8 * np.abs(ea).max()
    assert np.abs(g.grad.cpu().numpy() - eg).max() <= 1e-8 * np.abs(eg).max()
    sol.close()


def test_element_graph_and_batched_solves_match_host_solves_3d():
    from paper_2410_22686_gb300 import Batch
    m1, n, gamma = 7, 16, 1e-3
    eps = math.sqrt(osy.time_step(1.0, n))
    a = _coef(m1, 25)
    sols = [_solver(m1, n, a, precision="fp64", gamma=gamma, eps=eps),
            _solver(m1, n, a, precision="mixed", gamma=gamma, eps=eps)]
    sh = (m1, m1, m1)
    f, g, y0 = (_dev(S.random_vector(s, k)) for s, k in (((n,) + sh, 26), ((n,) + sh, 27), (sh, 28)))
    bs = [s.build_rhs(f, g, y0) for s in sols]
    singles = [s.solve(b, rtol=1e-10) for s, b in zip(sols, bs)]
    for s, b, (x_ref, it_ref, _) in zip(sols, bs, singles):
        x, it, rr = s.solve_graph(b, rtol=1e-10)
        assert it == it_ref and rr <= 1e-10
        assert (x - x_ref).norm().item() <= 1e-9 * x_ref.norm().item()
    batch = Batch(sols, bs, rtol=1e-10, maxit=80)
    iters, rel = batch.solve()
    for k, (x_ref, it_ref, _) in enumerate(singles):
        assert iters[k] == it_ref and rel[k] <= 1e-10
        assert (batch.xs[k] - x_ref).norm().item() <= 1e-9 * x_ref.norm().item()
    batch.close()
    for s in sols:
        s.close()


def test_double_float_product_equals_fp64_product_on_the_full_grid():
    """On the 63^3 grid of the 3D workload (n = 32): the product of an FP32 vector in
    double-float arithmetic equals the FP64-arithmetic product of the same (widened)
    vector, which the tests above check against the oracle, to 1e-12."""
    from paper_2410_22686_gb300 import Solver
    p = S.gaussian_field_3d_problem(m1=63, n=32)
    s32 = Solver(3, p.m1, p.n, p.T, p.gamma, p.eps, p.a_nodes, spatial="mg", precision="fp32", max_iter=4,
                 space="fe")
    s64 = Solver(3, p.m1, p.n, p.T, p.gamma, p.eps, p.a_nodes, spatial="mg", precision="fp64", max_iter=4,
                 space="fe")
    x32 = torch.from_numpy(S.random_vector((2 * p.n * p.m1 ** 3,), 3).astype(np.float32)).cuda()
    y32 = s32.matvec_f32(x32)
    y64 = s64.matvec(x32.double())
    assert (y32 - y64).abs().max().item() <= 1e-12 * y64.abs().max().item()
    s32.close()
    s64.close()
