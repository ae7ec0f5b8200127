"""Parity of the finite-element path (mass matrix M != I, Section 1) of the CUDA
library with the FP64 oracle ``oracle.fe``.

Tolerances (relative, max-norm): FP64 operators 1e-12 (same formulas, other
summation order); FP32 preconditioner 1e-5 (as for finite differences: FP32
roundoff times the FFT depth; the sine-transform solves are exact); solutions 1e-10
(FP64 preconditioner) and 1e-7 (mixed) with both sides solved far below that.
"""
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
    assert torch.cuda.is_available()


def _solver(d, m1, n, precision="fp64", gamma=1e-3, eps=0.3, T=1.0, max_iter=60, tiles=None):
    from paper_2410_22686_gb300 import Solver
    s = Solver(d, m1, n, T, gamma, eps, None, spatial="fst", precision=precision, max_iter=max_iter, space="fe")
    if tiles:
        s.set_tiles(**tiles)
    return s


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


# (dim, m1, n, time blocks per thread): one warp with a ragged tail (m1 = 7), several
# 30-column warp segments with a ragged last one (31, 61), a single point (m1 = 1),
# time chunks that split n unevenly (n = 37, chunk 8) or exceed it, and 3D
MATVEC_CASES = [(2, 7, 4, 0), (2, 31, 37, 8), (2, 61, 16, 5), (2, 1, 3, 0), (2, 30, 1, 0), (2, 32, 64, 0),
                (3, 7, 8, 3), (3, 5, 2, 0), (3, 33, 4, 0)]


@pytest.mark.parametrize("d,m1,n,tj", MATVEC_CASES)
def test_fe_matvec_and_transpose_match_oracle(d, m1, n, tj):
    gamma = 2e-3
    sol = _solver(d, m1, n, gamma=gamma, tiles={"mv_tj": tj} if tj else None)
    M, K = fe.fe_matrices(m1, d)
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    x = S.random_vector((2, n) + (m1,) * d, 7)
    assert _rel(sol.matvec(_dev(x)).cpu().numpy(), fe.apply_A(x, M, K, tau, alpha)) <= 1e-12
    assert _rel(sol.matvec(_dev(x), transpose=True).cpu().numpy(), fe.apply_AT(x, M, K, tau, alpha)) <= 1e-12
    # FP32 input (the flexible-GMRES basis; double-float arithmetic, transpose in FP64)
    x32 = x.astype(np.float32)
    y32 = sol.matvec_f32(torch.from_numpy(x32).cuda()).cpu().numpy()
    assert _rel(y32, fe.apply_A(x32.astype(np.float64), M, K, tau, alpha)) <= 1e-12
    sol.close()


def test_fe_build_rhs_matches_oracle():
    P = S.example1_problem(15, 16, 1e-4)
    sol = _solver(2, 15, 16, gamma=P.gamma, eps=P.eps)
    M, _ = fe.fe_matrices(15, 2)
    b = sol.build_rhs(_dev(P.f), _dev(P.g), _dev(P.y0)).cpu().numpy()
    assert _rel(b, fe.build_rhs(P.f, P.g, P.y0, P.tau, P.gamma, M)) <= 1e-13
    # NULL f and y0 mean zero fields
    b2 = sol.build_rhs(None, _dev(P.g), None).cpu().numpy()
    ref2 = fe.build_rhs(np.zeros_like(P.f), P.g, np.zeros_like(P.y0), P.tau, P.gamma, M)
    assert _rel(b2, ref2) <= 1e-13
    sol.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("d,m1,n", [(2, 31, 32), (2, 20, 16), (2, 7, 1), (2, 15, 24), (3, 7, 8), (3, 5, 4)])
def test_fe_precond_apply_matches_oracle(d, m1, n, precision, tol):
    gamma, eps = 1e-4, 0.25
    sol = _solver(d, m1, n, precision=precision, gamma=gamma, eps=eps)
    v = S.random_vector((2, n) + (m1,) * d, 11)
    w = sol.apply_precond(_dev(v)).cpu().numpy()
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    ref = opc.apply_Peps_inv(v, n, alpha, eps, fe.FSTSpatialSolverFE(m1, d, tau))
    assert _rel(w, ref) <= tol
    sol.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("d,m1,n", [(2, 255, 64), (3, 31, 16), (2, 15, 24)])
def test_fe_streaming_sine_transform_precond_matches_oracle(d, m1, n, precision, tol):
    """Persistent streaming sine transforms (several tiles per CTA at 255^2 x 66 planes)
    with the mass-matrix eigenvalues in the spectral divide."""
    gamma, eps = 1e-4, 0.25
    sol = _solver(d, m1, n, precision=precision, gamma=gamma, eps=eps, tiles={"fst_stream": 3})
    v = S.random_vector((2, n) + (m1,) * d, 17)
    w = sol.apply_precond(_dev(v)).cpu().numpy()
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    ref = opc.apply_Peps_inv(v, n, alpha, eps, fe.FSTSpatialSolverFE(m1, d, tau))
    assert _rel(w, ref) <= tol
    sol.close()


def _oracle_fe_solution(P, rtol=1e-13):
    M, K = fe.fe_matrices(P.m1, P.d)
    alpha = osy.alpha_weight(P.T, P.n, P.gamma)
    b = fe.build_rhs(P.f, P.g, P.y0, P.tau, P.gamma, M)
    A = lambda v: fe.apply_A(v, M, K, P.tau, alpha)
    Pi = lambda v: opc.apply_Peps_inv(v, P.n, alpha, P.eps, fe.FSTSpatialSolverFE(P.m1, P.d, P.tau))
    return M, K, b, okr.gmres(A, Pi, b, rtol=rtol, maxit=200, mode="right")


@pytest.mark.parametrize("precision,rtol,tol", [("fp64", 1e-12, 1e-10), ("mixed", 1e-11, 1e-7)])
@pytest.mark.parametrize("how", ["host", "graph"])
def test_fe_gmres_solution_and_end_points_match_oracle(precision, rtol, tol, how):
    P = S.example1_problem(31, 32, 1e-2)
    M, K, b_ref, ref = _oracle_fe_solution(P)
    assert ref.converged
    sol = _solver(2, 31, 32, precision=precision, gamma=P.gamma, eps=P.eps, T=P.T, max_iter=80)
    b = sol.build_rhs(_dev(P.f), _dev(P.g), _dev(P.y0))
    if how == "host":
        x, it, rr = sol.solve(b, rtol=rtol)
    else:
        x, it, rr = sol.solve_graph(b, rtol=rtol)
    assert rr <= rtol
    xr = ref.x.reshape(b_ref.shape)
    xg = x.cpu().numpy().reshape(b_ref.shape)
    assert np.linalg.norm(xg - xr) <= tol * np.linalg.norm(xr)
    # the oracle at the same tolerance takes about as many iterations
    ref_same = okr.gmres(lambda v: fe.apply_A(v, M, K, P.tau, osy.alpha_weight(P.T, P.n, P.gamma)),
                         lambda v: opc.apply_Peps_inv(v, P.n, osy.alpha_weight(P.T, P.n, P.gamma), P.eps,
                                                      fe.FSTSpatialSolverFE(P.m1, 2, P.tau)),
                         b_ref, rtol=rtol, maxit=200, mode="right")
    if precision == "fp64":
        assert abs(it - ref_same.iters) <= 1, (it, ref_same.iters)
    else:
        # the FP32 preconditioner differs from P_eps^{-1} by about u32 / eps (eps = tau/2
        # scales the time axis by up to 1/eps), which costs a few iterations at 1e-11
        assert ref_same.iters <= it <= ref_same.iters + 4, (it, ref_same.iters)
    if how == "host":
        yN, p0, eit = sol.end_point_solves(x, f_T=_dev(P.extra["f_T"]), g_0=_dev(P.extra["g_0"]), y0=_dev(P.y0),
                                           rtol=1e-13)
        assert 1 <= eit <= (2 if precision == "fp64" else 5)  # exact (FP64) sine-transform preconditioner
        # the oracle's end-point solves from the same x (p^(0) of Example 1 is of the size of
        # the discretisation error, so the GMRES tolerance must not enter the comparison)
        y, p = osy.unscale(xg, P.gamma)
        yN_ref, p0_ref = fe.end_point_solves(y, p, M, K, P.tau, P.gamma, P.extra["f_T"], P.extra["g_0"], P.y0)
        assert _rel(yN.cpu().numpy(), yN_ref) <= 1e-11
        assert _rel(p0.cpu().numpy(), p0_ref) <= 1e-11
    sol.close()


def test_fe_adjoint_solve_matches_oracle():
    d, m1, n, gamma = 2, 15, 16, 1e-3
    sol = _solver(d, m1, n, gamma=gamma)
    M, K = fe.fe_matrices(m1, d)
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    c = S.random_vector((2, n) + (m1,) * d, 5)
    lam, _, rr = sol.adjoint_solve(_dev(c), rtol=1e-12)
    assert rr <= 1e-12
    # A^T lam = c checked with the oracle's transpose
    res = fe.apply_AT(lam.cpu().numpy().reshape(c.shape), M, K, tau, alpha) - c
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(c)
    sol.close()


def test_fe_3d_gradient_pieces_match_oracle_and_fixed_coefficient_fails_loudly():
    """A 3D constant-coefficient element handle (sine transforms): the stiffness
    derivative of the gradient and the element objective match the oracle; its
    coefficient cannot be changed on the device."""
    from paper_2410_22686_gb300 import capi
    d, m1, n, gamma = 3, 7, 4, 1e-3
    sol = _solver(d, m1, n, gamma=gamma)
    a = np.ones((m1 + 2,) * d)
    M, _ = fe.fe_matrices(m1, d)
    tau = osy.time_step(1.0, n)
    xh = S.random_vector((2, n) + (m1,) * d, 31)
    lam = S.random_vector((2, n) + (m1,) * d, 32)
    gh = S.random_vector((n,) + (m1,) * d, 33)
    ga = sol.grad_log_a(_dev(xh), _dev(lam)).cpu().numpy().reshape((m1,) * d)
    ref_ga, _ = fe.adjoint_gradient(xh, lam, gh, a, M, tau, gamma)
    assert _rel(ga, ref_ga) <= 1e-12
    J = sol.objective(_dev(xh), _dev(gh)).item()
    ref = fe.objective(xh, gh, M, tau, gamma)
    assert abs(J - ref) <= 1e-13 * abs(ref)
    with pytest.raises(capi.PCError) as ei:
        sol.set_log_coefficient(torch.zeros((m1,) * d, dtype=torch.float64, device="cuda"))
    assert ei.value.status == capi.PC_ERR_UNSUPPORTED
    sol.close()


@pytest.mark.parametrize("fst_stream", [0, 1], ids=["tiles", "stream"])
def test_fe_full_size_operators_match_oracle(fst_stream):
    """255^2 grid, n = 256 (the size the finite-element solve is timed on): the whole
    product (FP64 and FP32 input) and the FP32 preconditioner against the oracle, with
    the sine-transform axis passes as one CTA per tile or as persistent streaming CTAs."""
    d, m1, n, gamma, eps = 2, 255, 256, 1e-2, 0.5
    sol = _solver(d, m1, n, precision="mixed", gamma=gamma, eps=eps, max_iter=4, tiles={"fst_stream": fst_stream})
    M, K = fe.fe_matrices(m1, d)
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    x = S.random_vector((2, n) + (m1,) * d, 21)
    assert _rel(sol.matvec(_dev(x)).cpu().numpy(), fe.apply_A(x, M, K, tau, alpha)) <= 1e-12
    x32 = x.astype(np.float32)
    y32 = sol.matvec_f32(torch.from_numpy(x32).cuda()).cpu().numpy()
    assert _rel(y32, fe.apply_A(x32.astype(np.float64), M, K, tau, alpha)) <= 1e-12
    w = sol.apply_precond(_dev(x)).cpu().numpy()
    ref = opc.apply_Peps_inv(x, n, alpha, eps, fe.FSTSpatialSolverFE(m1, d, tau))
    assert _rel(w, ref) <= 1e-5
    sol.close()


@pytest.mark.parametrize("precision,rtol,tol", [("fp64", 1e-12, 1e-10), ("mixed", 1e-11, 1e-7)])
def test_fe_3d_solve_and_end_points_match_oracle(precision, rtol, tol):
    d, m1, n, gamma, eps = 3, 7, 8, 1e-3, 0.25
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    M, K = fe.fe_matrices(m1, d)
    f = S.random_vector((n,) + (m1,) * d, 31)
    g = S.random_vector((n,) + (m1,) * d, 32)
    y0 = S.random_vector((m1,) * d, 33)
    b_ref = fe.build_rhs(f, g, y0, tau, gamma, M)
    ref = okr.gmres(lambda v: fe.apply_A(v, M, K, tau, alpha),
                    lambda v: opc.apply_Peps_inv(v, n, alpha, eps, fe.FSTSpatialSolverFE(m1, d, tau)),
                    b_ref, rtol=1e-13, maxit=200, mode="right")
    assert ref.converged
    sol = _solver(d, m1, n, precision=precision, gamma=gamma, eps=eps)
    b = sol.build_rhs(_dev(f), _dev(g), _dev(y0))
    assert _rel(b.cpu().numpy(), b_ref) <= 1e-13
    x, it, rr = sol.solve(b, rtol=rtol)
    assert rr <= rtol
    xg = x.cpu().numpy().reshape(b_ref.shape)
    xr = ref.x.reshape(b_ref.shape)
    assert np.linalg.norm(xg - xr) <= tol * np.linalg.norm(xr)
    fT, g0 = S.random_vector((m1,) * d, 34), S.random_vector((m1,) * d, 35)
    yN, p0, _ = sol.end_point_solves(x, f_T=_dev(fT), g_0=_dev(g0), y0=_dev(y0), rtol=1e-13)
    y, p = osy.unscale(xg, gamma)
    yN_ref, p0_ref = fe.end_point_solves(y, p, M, K, tau, gamma, fT, g0, y0)
    assert _rel(yN.cpu().numpy(), yN_ref) <= 1e-11
    assert _rel(p0.cpu().numpy(), p0_ref) <= 1e-11
    sol.close()


def test_fe_and_fd_handles_in_one_batch_match_individual_solves():
    from paper_2410_22686_gb300 import Batch, Solver
    P = S.example1_problem(31, 32, 1e-2)
    sols = [Solver(2, 31, 32, P.T, P.gamma, P.eps, None, spatial="fst", precision=prec, max_iter=60, space=sp)
            for sp, prec in (("fe", "fp64"), ("fd", "fp64"), ("fe", "fp32"))]
    bs = [s.build_rhs(_dev(P.f), _dev(P.g), _dev(P.y0)) for s in sols]
    singles = [s.solve(b, rtol=1e-10) for s, b in zip(sols, bs)]
    batch = Batch(sols, bs, rtol=1e-10, maxit=60)
    iters, rel = batch.solve()
    for k, (x_ref, it_ref, _) in enumerate(singles):
        assert iters[k] == it_ref
        assert rel[k] <= 1e-10
        assert (batch.xs[k] - x_ref).norm().item() <= 1e-12 * x_ref.norm().item()
    batch.close()
    for s in sols:
        s.close()


def test_fe_set_coefficient_and_autotune():
    """A constant coefficient c scales K (the sine-transform eigenvalues follow); the
    tuner's shapes leave the results unchanged."""
    d, m1, n, gamma, eps = 2, 31, 16, 1e-3, 0.3
    sol = _solver(d, m1, n, gamma=gamma, eps=eps, precision="fp32")
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    sol.set_coefficient(np.full((m1 + 2,) * d, 2.5))
    M, K = fe.fe_matrices(m1, d, coeff=2.5)
    x = S.random_vector((2, n) + (m1,) * d, 41)
    assert _rel(sol.matvec(_dev(x)).cpu().numpy(), fe.apply_A(x, M, K, tau, alpha)) <= 1e-12
    ref = opc.apply_Peps_inv(x, n, alpha, eps, fe.FSTSpatialSolverFE(m1, d, tau, coeff=2.5))
    w0 = sol.apply_precond(_dev(x)).cpu().numpy()
    assert _rel(w0, ref) <= 1e-5
    chosen = sol.autotune(2)
    assert chosen["mv_tj"] > 0
    assert _rel(sol.matvec(_dev(x)).cpu().numpy(), fe.apply_A(x, M, K, tau, alpha)) <= 1e-12
    assert _rel(sol.apply_precond(_dev(x)).cpu().numpy(), ref) <= 1e-5
    with pytest.raises(Exception):
        a = np.full((m1 + 2,) * d, 1.0)
        a[5, 5] = 2.0
        sol.set_coefficient(a)  # element handles keep a constant coefficient
    sol.close()


def test_fe_left_preconditioned_gmres_matches_oracle():
    """The paper's own GMRES mode (left preconditioning, stop on the preconditioned
    residual) with elements and a length n = 2^k - 1 (direct DFT in time)."""
    P = S.example1_problem(15, 15, 1e-2)
    M, K = fe.fe_matrices(15, 2)
    alpha = osy.alpha_weight(P.T, P.n, P.gamma)
    b_ref = fe.build_rhs(P.f, P.g, P.y0, P.tau, P.gamma, M)
    A = lambda v: fe.apply_A(v, M, K, P.tau, alpha)
    Pi = lambda v: opc.apply_Peps_inv(v, P.n, alpha, P.eps, fe.FSTSpatialSolverFE(15, 2, P.tau))
    ref = okr.gmres(A, Pi, b_ref, rtol=1e-10, maxit=100, mode="left")
    assert ref.converged
    sol = _solver(2, 15, 15, gamma=P.gamma, eps=P.eps, T=P.T, max_iter=60)
    b = sol.build_rhs(_dev(P.f), _dev(P.g), _dev(P.y0))
    x, it, rr = sol.solve(b, rtol=1e-10, mode="left")
    assert it == ref.iters
    xr = ref.x.reshape(b_ref.shape)
    assert np.linalg.norm(x.cpu().numpy().reshape(b_ref.shape) - xr) <= 1e-9 * np.linalg.norm(xr)
    sol.close()
