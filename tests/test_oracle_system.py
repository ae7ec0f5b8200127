"""Pins of the oracle's discrete system (Section 1) against facts the paper and
the mathematics fix, not against the oracle itself."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import system as sy

from conftest import read_golden


def _lap1d(m):
    h = 1.0 / (m + 1)
    return (2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)) / (h * h)


@pytest.mark.parametrize("d,m1,c", [(2, 5, 1.0), (2, 7, 2.5), (3, 3, 1.0), (3, 4, 0.7)])
def test_K_constant_coefficient_is_kronecker_sum_of_1d_laplacians(d, m1, c):
    # textbook: -Laplacian with Dirichlet BCs = sum of 1D second differences
    L1 = _lap1d(m1)
    I = np.eye(m1)
    if d == 2:
        Kref = np.kron(I, L1) + np.kron(L1, I)
    else:
        Kref = np.kron(np.kron(I, I), L1) + np.kron(np.kron(I, L1), I) + np.kron(np.kron(L1, I), I)
    Kref *= c
    a = np.full((m1 + 2,) * d, c)
    u = S.random_vector((m1,) * d, 1)
    assert np.allclose(sy.apply_K(u, a).ravel(), Kref @ u.ravel(), rtol=1e-13, atol=1e-10)
    assert np.allclose(sy.K_sparse(a).toarray(), Kref, rtol=1e-13, atol=1e-10)


@pytest.mark.parametrize("d", [2, 3])
def test_K_variable_coefficient_second_order_consistency(d):
    # closed form: u = prod sin(pi x_k), a = 1 + 0.5 sin(2 pi x1) cos(2 pi x2);
    # -div(a grad u) = -a Lap u - grad a . grad u, computed analytically.
    errs = []
    for m1 in ([15, 31, 63] if d == 2 else [7, 15, 31]):
        xs = S.interior_grid(m1, d)
        Xs = S.node_grid(m1, d)
        a_nodes = 1 + 0.5 * np.sin(2 * math.pi * Xs[0]) * np.cos(2 * math.pi * Xs[1])
        x1, x2 = xs[0], xs[1]
        u = np.ones_like(x1)
        for k in range(d):
            u = u * np.sin(math.pi * xs[k])
        a = 1 + 0.5 * np.sin(2 * math.pi * x1) * np.cos(2 * math.pi * x2)
        ax1 = math.pi * np.cos(2 * math.pi * x1) * np.cos(2 * math.pi * x2)
        ax2 = -math.pi * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2)
        lap = -d * math.pi ** 2 * u
        ux1 = math.pi * np.cos(math.pi * x1) * u / np.sin(math.pi * x1)
        ux2 = math.pi * np.cos(math.pi * x2) * u / np.sin(math.pi * x2)
        exact = -(a * lap + ax1 * ux1 + ax2 * ux2)
        errs.append(np.abs(sy.apply_K(u, a_nodes) - exact).max())
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(r > 3.5 for r in rates), (errs, rates)


def test_K_symmetric_positive_definite():
    a = np.exp(0.5 * S.random_vector((9, 9), 3))
    K = sy.K_sparse(a).toarray()
    assert np.allclose(K, K.T, atol=1e-12)
    assert np.linalg.eigvalsh(K).min() > 0


@pytest.mark.parametrize("d,m1,n", [(2, 3, 5), (2, 4, 1), (3, 2, 3), (2, 3, 2)])
def test_matrix_free_A_matches_kronecker_block_form(d, m1, n):
    a = np.exp(0.3 * S.random_vector((m1 + 2,) * d, 5))
    K = sy.K_sparse(a).toarray()
    tau, alpha = sy.time_step(1.0, n), sy.alpha_weight(1.0, n, 1e-3)
    A = sy.A_dense(K, n, tau, alpha)
    x = S.random_vector((2, n) + (m1,) * d, 6)
    assert np.allclose(sy.apply_A(x, a, tau, alpha).ravel(), A @ x.ravel(), atol=1e-11)
    assert np.allclose(sy.apply_AT(x, a, tau, alpha).ravel(), A.T @ x.ravel(), atol=1e-11)
    # A^T = S A S with S = diag(I, -I): follows from the block form with K symmetric
    Sg = np.diag(np.concatenate([np.ones(n * m1 ** d), -np.ones(n * m1 ** d)]))
    assert np.allclose(A.T, Sg @ A @ Sg, atol=1e-12)


def test_B_matrix_backward_euler_difference():
    B = sy.B_matrix(4)
    v = np.array([1.0, 3.0, 6.0, 10.0])
    assert np.allclose(B @ v, [1.0, 2.0, 3.0, 4.0])


def test_scaled_system_equals_unscaled_kkt_system():
    # Eq. main_system_before vs Eq. main_system: x = [sqrt(gamma) y; p], b = [g; -sqrt(gamma) f]
    m1, n, gamma = 3, 4, 3e-3
    a = np.exp(0.3 * S.random_vector((m1 + 2,) * 2, 7))
    K = sy.K_sparse(a).toarray()
    tau, alpha = sy.time_step(1.0, n), sy.alpha_weight(1.0, n, gamma)
    f = S.random_vector((n, m1, m1), 8)
    g = S.random_vector((n, m1, m1), 9)
    y0 = S.random_vector((m1, m1), 10)
    At = sy.A_tilde_dense(K, n, tau, gamma)
    gv = tau * g
    fv = tau * f
    fv[0] += y0
    yp = np.linalg.solve(At, np.concatenate([gv.ravel(), fv.ravel()]))
    x = np.linalg.solve(sy.A_dense(K, n, tau, alpha), sy.build_rhs(f, g, y0, tau, gamma).ravel())
    half = n * m1 * m1
    assert np.allclose(x[:half], math.sqrt(gamma) * yp[:half], rtol=1e-10, atol=1e-13)
    assert np.allclose(x[half:], yp[half:], rtol=1e-10, atol=1e-13)


def test_backward_euler_rows_of_the_kkt_system():
    # the forward equation y_j - y_{j-1} + tau K y_j - (tau/gamma) p_j = tau f_j (Section 1)
    # must hold for the solution of the all-at-once system, time step by time step
    m1, n, gamma = 3, 5, 1e-2
    a = np.exp(0.2 * S.random_vector((m1 + 2,) * 2, 11))
    tau, alpha = sy.time_step(1.0, n), sy.alpha_weight(1.0, n, gamma)
    K = sy.K_sparse(a).toarray()
    f = S.random_vector((n, m1, m1), 12)
    g = S.random_vector((n, m1, m1), 13)
    y0 = S.random_vector((m1, m1), 14)
    x = np.linalg.solve(sy.A_dense(K, n, tau, alpha), sy.build_rhs(f, g, y0, tau, gamma).ravel())
    y, p = sy.unscale(x.reshape((2, n, m1, m1)), gamma)
    yprev = y0.ravel()
    for j in range(n):
        lhs = y[j].ravel() - yprev + tau * K @ y[j].ravel() - tau / gamma * p[j].ravel()
        assert np.allclose(lhs, tau * f[j].ravel(), atol=1e-10)
        yprev = y[j].ravel()
    # backward equation -(p_{j+1} - p_j) + tau K p_j = tau (g_j - y_j), p_{n+1} = 0
    for j in range(n):
        pn = p[j + 1].ravel() if j + 1 < n else np.zeros(m1 * m1)
        lhs = -(pn - p[j].ravel()) + tau * K @ p[j].ravel()
        assert np.allclose(lhs, tau * (g[j].ravel() - y[j].ravel()), atol=1e-10)


def _solve_example(ex, m1, n, gamma, smoother="red-black", ideal=False):
    """Paper-mode GMRES (left, tol 1e-8) iteration count and e_h of the discrete
    solution (a tight right-preconditioned solve); ideal: the preconditioner P of
    Eq. matrix_P instead of P_eps, e_h of the paper-mode iterate."""
    from oracle import precond as pc, krylov as kr
    P = (S.example1_problem if ex == 1 else S.example2_problem)(m1, n, gamma)
    a = P.a_nodes if P.a_nodes is not None else sy.unit_coefficient(m1, 2)
    tau, al = P.tau, sy.alpha_weight(P.T, n, gamma)
    b = sy.build_rhs(P.f, P.g, P.y0, tau, gamma)
    sol = pc.make_spatial_solver("fst" if ex == 1 else "mg", P.a_nodes, m1, 2, tau, smoother)
    Aop = lambda v: sy.apply_A(v, a, tau, al)
    if ideal:
        Pinv = lambda v: pc.apply_P_inv(v, n, al, sol)
    else:
        Pinv = lambda v: pc.apply_Peps_inv(v, n, al, P.eps, sol)
    paper_run = kr.gmres(Aop, Pinv, b, rtol=1e-8, maxit=100, mode="left")
    if ideal:  # e_h of the paper-mode iterate itself (tol 1e-8), as the table reports it
        y, p = sy.unscale(paper_run.x, gamma)
    else:
        tight = kr.gmres(Aop, Pinv, b, rtol=1e-13, maxit=300, mode="right")
        y, p = sy.unscale(tight.x, gamma)
    yN, p0 = sy.end_point_solves(y, p, a, tau, gamma, P.extra["f_T"], P.extra["g_0"], P.y0)
    N = n + 1
    x1, x2 = S.interior_grid(m1, 2)
    tl = tau * np.arange(N + 1)
    if ex == 1:
        exact = S.example1_exact
    else:
        exact = lambda u, v, t: S.example2_exact(u, v, t, gamma)
    yex = [exact(x1, x2, tl[j])[0] for j in range(1, N + 1)]
    pex = [exact(x1, x2, tl[j])[1] for j in range(0, N)]
    eh = sy.error_measure(list(y) + [yN], [p0] + list(p), yex, pex, P.h, 2)
    return paper_run.iters, eh


def _matches_printed(value, printed):
    # the tables print e_h with three significant digits: allow 0.6 of a unit
    # in the last printed digit
    unit = 10.0 ** (math.floor(math.log10(abs(printed))) - 2)
    return abs(value - printed) <= 0.6 * unit


@pytest.mark.parametrize("row", read_golden("table3_example1.txt"))
def test_example1_error_and_iterations_match_table3(row):
    gamma, lh, lt, dof, it, eh = float(row[0]), int(row[1]), int(row[2]), int(row[3]), int(row[4]), float(row[5])
    m1, n = 2 ** lh - 1, 2 ** lt - 1
    assert 2 * m1 * m1 * (n + 1) == dof          # the paper's DoF counts the two end blocks
    iters, got = _solve_example(1, m1, n, gamma)
    assert _matches_printed(got, eh), (got, eh)
    assert abs(iters - it) <= 1, (iters, it)


@pytest.mark.parametrize("row", read_golden("table7_example2.txt"))
def test_example2_error_and_iterations_match_table7(row):
    gamma, lh, lt, dof, it, eh = float(row[0]), int(row[1]), int(row[2]), int(row[3]), int(row[4]), float(row[5])
    m1, n = 2 ** lh - 1, 2 ** lt - 1
    assert 2 * m1 * m1 * (n + 1) == dof
    iters, got = _solve_example(2, m1, n, gamma)
    assert _matches_printed(got, eh), (got, eh)
    # red-black ordering (the parallel default): within 3 of the printed count
    assert abs(iters - it) <= 3, (iters, it)


@pytest.mark.parametrize("row", read_golden("table7_example2.txt"))
def test_example2_lexicographic_gauss_seidel_gives_table7_counts(row):
    # the paper does not state the Gauss-Seidel ordering; a sweep in the natural order
    # reproduces every iteration count of Table 7
    gamma, lh, lt, it = float(row[0]), int(row[1]), int(row[2]), int(row[4])
    iters, _ = _solve_example(2, 2 ** lh - 1, 2 ** lt - 1, gamma, "lexicographic")
    assert iters == it, (iters, it)


@pytest.mark.parametrize("row", read_golden("table4_example1_P.txt"))
def test_example1_with_ideal_P_matches_table4(row):
    # GMRES-P (Eq. matrix_P, sine-transform solves): every count of Table 4 and e_h
    gamma, lh, lt, dof, it, eh = float(row[0]), int(row[1]), int(row[2]), int(row[3]), int(row[4]), float(row[5])
    m1, n = 2 ** lh - 1, 2 ** lt - 1
    assert 2 * m1 * m1 * (n + 1) == dof
    iters, got = _solve_example(1, m1, n, gamma, ideal=True)
    assert iters == it, (iters, it)
    assert _matches_printed(got, eh), (got, eh)


@pytest.mark.parametrize("row", read_golden("table8_example2_P.txt"))
def test_example2_with_ideal_P_matches_table8(row):
    gamma, lh, lt, dof, it, eh = float(row[0]), int(row[1]), int(row[2]), int(row[3]), int(row[4]), float(row[5])
    m1, n = 2 ** lh - 1, 2 ** lt - 1
    assert 2 * m1 * m1 * (n + 1) == dof
    iters, got = _solve_example(2, m1, n, gamma, ideal=True)
    assert abs(iters - it) <= 2, (iters, it)         # red-black V-cycle
    if gamma >= 1e-4:                                 # rows where Tables 7 and 8 agree on e_h
        assert _matches_printed(got, eh), (got, eh)
    if lt == 5:  # natural-order Gauss-Seidel gives the printed count exactly (the oracle's
        # natural-order sweep is slow, so the tau = 2^-6 rows are left to the GPU test)
        iters_lex, _ = _solve_example(2, m1, n, gamma, "lexicographic", ideal=True)
        assert iters_lex == it, (iters_lex, it)
