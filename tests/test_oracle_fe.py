"""Pins of the finite-element oracle (oracle/fe.py): Q1 mass and stiffness matrices,
the all-at-once operator with M != I, the four-step P_eps^{-1} with (sigma M + tau K)
spatial solves, and the discrete solution's convergence to a manufactured solution."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import fe, krylov as okr, precond as opc, system as osy


@pytest.mark.parametrize("d,m1", [(2, 3), (2, 5), (3, 3)])
def test_kronecker_matrices_equal_element_assembly(d, m1):
    M, K = fe.fe_matrices(m1, d, coeff=1.7)
    Me, Ke = fe.fe_matrices_by_elements(m1, d, coeff=1.7)
    assert abs(M - Me).max() < 1e-15
    assert abs(K - Ke).max() < 1e-13


def test_1d_matrices_closed_form():
    M1, K1 = fe.fe_1d(4)
    h = 0.2
    ref_M = h / 6 * np.array([[4, 1, 0, 0], [1, 4, 1, 0], [0, 1, 4, 1], [0, 0, 1, 4]])
    ref_K = 1 / h * np.array([[2, -1, 0, 0], [-1, 2, -1, 0], [0, -1, 2, -1], [0, 0, -1, 2]])
    assert np.allclose(M1.toarray(), ref_M, rtol=0, atol=1e-15)
    assert np.allclose(K1.toarray(), ref_K, rtol=0, atol=1e-12)


def test_mass_matrix_integrates_constants_and_matrices_are_spd():
    M, K = fe.fe_matrices(7, 2)
    Md = M.toarray()
    # sum of all entries = integral of (sum of interior basis functions)^2 > 0, and M, K SPD
    assert np.all(np.linalg.eigvalsh(Md) > 0) and np.all(np.linalg.eigvalsh(K.toarray()) > 0)
    # a full row of the 9-point mass stencil sums to h^2 (interior node)
    h = 1 / 8
    row = Md[3 * 7 + 3]
    assert math.isclose(row.sum(), h * h, rel_tol=1e-14)


@pytest.mark.parametrize("d,m1", [(2, 5), (3, 3)])
def test_sine_transform_eigenvalues(d, m1):
    M, K = fe.fe_matrices(m1, d, coeff=0.6)
    lamM, lamK = fe.fe_eigenvalues(m1, d, coeff=0.6)
    assert np.allclose(np.sort(lamM.ravel()), np.linalg.eigvalsh(M.toarray()), rtol=1e-12, atol=0)
    assert np.allclose(np.sort(lamK.ravel()), np.linalg.eigvalsh(K.toarray()), rtol=1e-12, atol=0)
    # and the transform diagonalises both: S M S = diag(lamM) entry by entry
    sol = fe.FSTSpatialSolverFE(m1, d, tau=0.1, coeff=0.6)
    dense = fe.DenseSpatialSolverFE(M, K, 0.1, (m1,) * d)
    R = S.random_vector((3,) + (m1,) * d, 1) + 1j * S.random_vector((3,) + (m1,) * d, 2)
    sig = np.array([1.0 + 0.3j, 0.2 - 0.1j, 2.0])
    assert np.abs(sol(sig, R) - dense(sig, R)).max() < 1e-12 * np.abs(dense(sig, R)).max()


def test_operator_matches_dense_kronecker_form():
    m1, n, tau, alpha = 4, 3, 0.2, 0.7
    M, K = fe.fe_matrices(m1, 2, coeff=1.3)
    x = S.random_vector((2, n, m1, m1), 3)
    A = fe.A_dense(M, K, n, tau, alpha)
    assert np.allclose(fe.apply_A(x, M, K, tau, alpha).ravel(), A @ x.ravel(), rtol=1e-13, atol=1e-13)
    assert np.allclose(fe.apply_AT(x, M, K, tau, alpha).ravel(), A.T @ x.ravel(), rtol=1e-13, atol=1e-13)
    # A^T = S A S with S = blockdiag(I, -I)
    Sg = np.diag(np.r_[np.ones(n * m1 * m1), -np.ones(n * m1 * m1)])
    assert np.allclose(A.T, Sg @ A @ Sg)


def test_four_step_apply_matches_dense_P_eps():
    m1, n, tau, alpha, eps = 5, 4, 0.2, 0.8, 0.3
    M, K = fe.fe_matrices(m1, 2, coeff=1.0)
    P = fe.P_eps_dense(M, K, n, tau, alpha, eps)
    v = S.random_vector((2, n, m1, m1), 4)
    w = opc.apply_Peps_inv(v, n, alpha, eps, fe.FSTSpatialSolverFE(m1, 2, tau))
    ref = np.linalg.solve(P, v.ravel())
    assert np.abs(w.ravel() - ref).max() < 1e-11 * np.abs(ref).max()


def _fe_solution(m1, gamma, n=None):
    n = m1 if n is None else n
    P = S.example1_problem(m1, n, gamma)
    M, K = fe.fe_matrices(m1, 2)
    tau, alpha = P.tau, osy.alpha_weight(P.T, n, gamma)
    b = fe.build_rhs(P.f, P.g, P.y0, tau, gamma, M)
    spat = fe.FSTSpatialSolverFE(m1, 2, tau)
    A = lambda v: fe.apply_A(v, M, K, tau, alpha)
    Pi = lambda v: opc.apply_Peps_inv(v, n, alpha, P.eps, spat)
    res = okr.gmres(A, Pi, b, rtol=1e-12, maxit=200, mode="right")
    assert res.converged
    x, it = res.x.reshape(b.shape), res.iters
    y, p = osy.unscale(x, gamma)
    yN, p0 = fe.end_point_solves(y, p, M, K, tau, gamma, P.extra["f_T"], P.extra["g_0"], P.y0)
    x1, x2 = S.interior_grid(m1, 2)
    tl = tau * np.arange(n + 2)
    yex = [S.example1_exact(x1, x2, tl[j])[0] for j in range(1, n + 2)]
    pex = [S.example1_exact(x1, x2, tl[j])[1] for j in range(0, n + 1)]
    eh = osy.error_measure(list(y) + [yN], [p0] + list(p), yex, pex, P.h, 2)
    return eh, it


def test_discrete_eigenvalue_is_second_order():
    # sin(pi x1) sin(pi x2) is an eigenvector of both M and K; its Rayleigh quotient
    # converges to the continuous eigenvalue 2 pi^2 at O(h^2)
    err = []
    for m1 in (7, 15, 31, 63):
        lamM, lamK = fe.fe_eigenvalues(m1, 2)
        err.append(lamK[0, 0] / lamM[0, 0] - 2 * math.pi ** 2)
    for a, b in zip(err, err[1:]):
        assert 3.9 < a / b < 4.1, err


def test_discrete_solution_converges_to_the_manufactured_solution():
    # tau = h^2: backward Euler (first order in tau) and the elements (second order in
    # h) both contribute O(h^2), so e_h falls by ~4 per halving of h.  (With tau = h the
    # two errors of Example 1 have opposite signs and cancel near m1 = 31.)
    errs = [_fe_solution(m1, 1e-2, n=(m1 + 1) ** 2 - 1)[0] for m1 in (3, 7, 15)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.4 and 3.6 < r2 < 4.4, errs


def test_gmres_iterations_stay_bounded_across_n_and_gamma():
    its = [_fe_solution(m1, g)[1] for m1 in (7, 15) for g in (1e-2, 1e-6)]
    assert max(its) <= 30 and max(its) - min(its) <= 12, its
