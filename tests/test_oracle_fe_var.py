"""Pins of the variable-coefficient element oracle (oracle/fe.py): K(a) = sum_e a_e K_e
with a_e the nodal interpolant at the element centre, the multicolour V(1,0) cycle for
(sigma M + tau K(a)), the element objective and its gradient."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synthetic as S
from oracle import fe, gradient as ogr, krylov as okr, precond as opc, system as osy


@pytest.mark.parametrize("d,m1", [(2, 5), (3, 3)])
def test_constant_coefficient_reduces_to_the_kronecker_form(d, m1):
    M, K = fe.fe_matrices(m1, d, coeff=2.3)
    Mv, Kv = fe.fe_matrices_var(np.full((m1 + 2,) * d, 2.3))
    assert abs(M - Mv).max() < 1e-15
    assert abs(K - Kv).max() < 1e-13


def test_element_coefficient_of_a_bilinear_field_is_its_centre_value():
    # a(x) = 1 + x1 + 2 x2 + x1 x2 is its own bilinear interpolant: a_e = a(centre of e)
    m1 = 6
    h = 1 / (m1 + 1)
    x = np.arange(m1 + 2) * h
    X2, X1 = np.meshgrid(x, x, indexing="ij")
    a = 1 + X1 + 2 * X2 + X1 * X2
    c = (np.arange(m1 + 1) + 0.5) * h
    C2, C1 = np.meshgrid(c, c, indexing="ij")
    assert np.allclose(fe.element_coefficients(a), 1 + C1 + 2 * C2 + C1 * C2, rtol=0, atol=1e-14)


def test_stiffness_is_symmetric_positive_definite_and_kills_constants_inside():
    m1 = 7
    a = np.exp(0.5 * S.random_vector((m1 + 2, m1 + 2), 3))
    _, K = fe.fe_matrices_var(a)
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() < 1e-14
    assert np.linalg.eigvalsh(Kd).min() > 0
    # rows of nodes away from the boundary: K applied to a constant vanishes
    row = Kd[(m1 // 2) * m1 + m1 // 2]
    assert abs(row.sum()) < 1e-13 * np.abs(row).max()


def test_variable_coefficient_solution_is_second_order():
    # -div(a grad u) = f with u = sin(pi x1) sin(pi x2), a = 1 + x1 x2 + x2^2 / 2
    def err(m1):
        h = 1 / (m1 + 1)
        xn = np.arange(m1 + 2) * h
        X2, X1 = np.meshgrid(xn, xn, indexing="ij")
        a = 1 + X1 * X2 + 0.5 * X2 ** 2
        xi = xn[1:-1]
        Y2, Y1 = np.meshgrid(xi, xi, indexing="ij")
        s1, c1 = np.sin(np.pi * Y1), np.cos(np.pi * Y1)
        s2, c2 = np.sin(np.pi * Y2), np.cos(np.pi * Y2)
        aa = 1 + Y1 * Y2 + 0.5 * Y2 ** 2
        a1, a2 = Y2, Y1 + Y2                     # da/dx1, da/dx2
        u = s1 * s2
        f = 2 * np.pi ** 2 * aa * u - np.pi * (a1 * c1 * s2 + a2 * s1 * c2)
        M, K = fe.fe_matrices_var(a)
        uh = spla.spsolve(K.tocsc(), M @ f.ravel())
        return np.abs(uh - u.ravel()).max()

    e1, e2 = err(15), err(31)
    assert 3.5 < e1 / e2 < 4.6, (e1, e2)


def test_stiffness_derivative_equals_central_differences():
    m1, d = 5, 2
    a = np.exp(0.3 * S.random_vector((m1 + 2,) * d, 5))
    u = S.random_vector((3, m1, m1), 6)
    v = S.random_vector((3, m1, m1), 7)
    Sd = fe.stiffness_derivative(u, v, a)

    def form(ax):
        _, K = fe.fe_matrices_var(ax)
        return sum(float(u[t].ravel() @ (K @ v[t].ravel())) for t in range(3))

    h = 1e-6
    for P in [(1, 1), (2, 4), (5, 5), (4, 2)]:
        ap, am = a.copy(), a.copy()
        ap[P] *= math.exp(h)
        am[P] *= math.exp(-h)
        fd = (form(ap) - form(am)) / (2 * h)
        assert abs(fd - Sd[P[0] - 1, P[1] - 1]) <= 1e-7 * abs(fd)


def _prolongation_matrix(mc, d):
    cols = []
    for k in range(mc ** d):
        e = np.zeros(mc ** d)
        e[k] = 1.0
        cols.append(opc.prolong_linear(e.reshape((1,) + (mc,) * d), d).ravel())
    return np.array(cols).T


def test_restriction_is_the_transpose_of_the_interpolation():
    for d, mc in [(2, 3), (3, 1)]:
        P = _prolongation_matrix(mc, d)
        r = S.random_vector((2,) + (2 * mc + 1,) * d, 9)
        got = fe.restrict_transpose(r, d).reshape(2, -1)
        assert np.abs(got - (P.T @ r.reshape(2, -1).T).T).max() < 1e-14


def _vcycle_by_loops(a_nodes, tau, sigma, r):
    """The V(1,0) cycle written out point by point with dense matrices: Gauss-Seidel
    over colour 0, 1, 2, 3 (each colour in index order), residual, P^T, recursion,
    correction by P."""
    m = a_nodes.shape[0] - 2
    M, K = fe.fe_matrices_var(a_nodes)
    A = sigma * M.toarray() + tau * K.toarray()
    if m == 1:
        return r / A[0, 0]
    col = fe.colour_of(m, 2).ravel()
    u = np.zeros(m * m, dtype=complex)
    for c in range(4):
        for pnt in range(m * m):
            if col[pnt] != c:
                continue
            u[pnt] = (r[pnt] - sum(A[pnt, q] * u[q] for q in range(m * m) if q != pnt)) / A[pnt, pnt]
    res = r - A @ u
    mc = (m - 1) // 2
    P = _prolongation_matrix(mc, 2)
    ec = _vcycle_by_loops(a_nodes[::2, ::2], tau, sigma, P.T @ res)
    return u + P @ ec


@pytest.mark.parametrize("m1", [3, 7])
def test_vcycle_equals_the_point_by_point_cycle(m1):
    a = np.exp(0.4 * S.random_vector((m1 + 2, m1 + 2), 11))
    tau = 0.05
    mg = fe.MGSpatialSolverFE(a, tau)
    sig = np.array([0.7 + 0.4j, 1.3 - 0.2j])
    r = S.random_vector((2, m1, m1), 12) + 1j * S.random_vector((2, m1, m1), 13)
    got = mg(sig, r)
    for k in range(2):
        ref = _vcycle_by_loops(a, tau, sig[k], r[k].ravel())
        assert np.abs(got[k].ravel() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_vcycle_is_a_contraction():
    m1 = 31
    a = np.exp(0.5 * S.random_vector((m1 + 2, m1 + 2), 14))
    tau = 1 / 65
    mg = fe.MGSpatialSolverFE(a, tau)
    M, K = fe.fe_matrices_var(a)
    for sig in (1.0, 0.3 + 0.8j, 1e-3 + 0.05j):
        A = (sig * M + tau * K).tocsr()
        b = A @ S.random_vector((m1 * m1,), 15)
        u = np.zeros(m1 * m1, dtype=complex)
        for _ in range(6):
            r = b - A @ u
            u = u + mg(np.array([sig]), r.reshape(1, m1, m1))[0].ravel()
        rate = np.linalg.norm(b - A @ u) / np.linalg.norm(r)
        assert rate < 0.5, (sig, rate)


def test_preconditioned_gmres_converges_in_few_iterations():
    m1, n, gamma = 15, 16, 1e-3
    a = np.exp(0.4 * S.random_vector((m1 + 2, m1 + 2), 16))
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    eps = math.sqrt(tau)
    M, K = fe.fe_matrices_var(a)
    mg = fe.MGSpatialSolverFE(a, tau)
    b = fe.build_rhs(S.random_vector((n, m1, m1), 17), S.random_vector((n, m1, m1), 18),
                     S.random_vector((m1, m1), 19), tau, gamma, M)
    res = okr.gmres(lambda v: fe.apply_A(v, M, K, tau, alpha),
                    lambda v: opc.apply_Peps_inv(v, n, alpha, eps, mg), b, rtol=1e-10, maxit=80, mode="right")
    assert res.converged and res.iters <= 40


def test_objective_with_scaled_identity_mass_is_the_difference_objective():
    m1, n, gamma = 7, 4, 1e-2
    h = 1 / (m1 + 1)
    x = S.random_vector((2, n, m1, m1), 21)
    g = S.random_vector((n, m1, m1), 22)
    tau = osy.time_step(1.0, n)
    Mh = sp.identity(m1 * m1, format="csr") * h * h
    assert math.isclose(fe.objective(x, g, Mh, tau, gamma), ogr.objective(x, g, tau, gamma), rel_tol=1e-14)


def test_objective_gradient_equals_central_differences():
    m1, n, gamma = 5, 3, 1e-2
    a = np.exp(0.3 * S.random_vector((m1 + 2, m1 + 2), 23))
    M, _ = fe.fe_matrices_var(a)
    x = S.random_vector((2, n, m1, m1), 24)
    g = S.random_vector((n, m1, m1), 25)
    tau = osy.time_step(1.0, n)
    gx = fe.objective_grad_x(x, g, M, tau, gamma)
    d = S.random_vector(x.shape, 26)
    h = 1e-6
    fd = (fe.objective(x + h * d, g, M, tau, gamma) - fe.objective(x - h * d, g, M, tau, gamma)) / (2 * h)
    assert abs(fd - float(np.sum(gx * d))) <= 1e-7 * abs(fd)


def test_gradient_routes_agree_with_finite_differences_of_the_optimum():
    """dJ*/d log a and dJ*/dg at the exact optimum: envelope form, adjoint form and
    central differences of J(x*(theta)) with x* from a dense solve."""
    m1, n, gamma = 3, 4, 1e-2
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    a0 = np.exp(0.3 * S.random_vector((m1 + 2, m1 + 2), 27))
    f = S.random_vector((n, m1, m1), 28)
    g0 = S.random_vector((n, m1, m1), 29)
    y0 = S.random_vector((m1, m1), 30)

    def optimum(a, g):
        M, K = fe.fe_matrices_var(a)
        A = fe.A_dense(M, K, n, tau, alpha)
        b = fe.build_rhs(f, g, y0, tau, gamma, M)
        return np.linalg.solve(A, b.ravel()).reshape(b.shape), M, K, A

    x, M, K, A = optimum(a0, g0)
    ea, eg = fe.envelope_gradient(x, g0, a0, M, tau, gamma)
    lam = np.linalg.solve(A.T, fe.objective_grad_x(x, g0, M, tau, gamma).ravel()).reshape(x.shape)
    aa, ag = fe.adjoint_gradient(x, lam, g0, a0, M, tau, gamma)
    assert np.abs(ea - aa).max() <= 1e-10 * np.abs(ea).max()
    assert np.abs(eg - ag).max() <= 1e-10 * np.abs(eg).max()
    h = 1e-6
    J = lambda a, g: fe.objective(optimum(a, g)[0], g, optimum(a, g)[1], tau, gamma)
    for P in [(1, 1), (2, 3), (3, 2)]:
        ap, am = a0.copy(), a0.copy()
        ap[P] *= math.exp(h)
        am[P] *= math.exp(-h)
        fd = (J(ap, g0) - J(am, g0)) / (2 * h)
        assert abs(fd - ea[P[0] - 1, P[1] - 1]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(ea).max())
    dg = S.random_vector(g0.shape, 31)
    fd = (J(a0, g0 + h * dg) - J(a0, g0 - h * dg)) / (2 * h)
    assert abs(fd - float(np.sum(eg * dg))) <= 1e-6 * abs(fd)


# ---------------------------------------------------------------------------
# trilinear elements with a nodal coefficient (3D)
# ---------------------------------------------------------------------------

def test_trilinear_element_matrices_have_the_closed_form_entries():
    # K_e = h/12 [4, 0, -1, -1] and M_e = h^3/216 [8, 4, 2, 1] for corners differing in
    # 0, 1, 2, 3 coordinates (the tensor products of the 1D element matrices)
    m1 = 3
    h = 1 / (m1 + 1)
    corners, Me, Ke = fe.reference_element(m1, 3)
    kv, mv = [4.0, 0.0, -1.0, -1.0], [8.0, 4.0, 2.0, 1.0]
    for p, cp in enumerate(corners):
        for q, cq in enumerate(corners):
            t = sum(a != b for a, b in zip(cp, cq))
            assert abs(Ke[p, q] - h / 12 * kv[t]) < 1e-15
            assert abs(Me[p, q] - h ** 3 / 216 * mv[t]) < 1e-17


def test_variable_coefficient_solution_is_second_order_in_3d():
    # -div(a grad u) = f, u = sin(pi x1) sin(pi x2) sin(pi x3), a = 1 + x1 x3 + x2^2 / 2
    def err(m1):
        h = 1 / (m1 + 1)
        xn = np.arange(m1 + 2) * h
        X3, X2, X1 = np.meshgrid(xn, xn, xn, indexing="ij")
        a = 1 + X1 * X3 + 0.5 * X2 ** 2
        xi = xn[1:-1]
        Y3, Y2, Y1 = np.meshgrid(xi, xi, xi, indexing="ij")
        s = [np.sin(np.pi * Y) for Y in (Y1, Y2, Y3)]
        c = [np.cos(np.pi * Y) for Y in (Y1, Y2, Y3)]
        aa = 1 + Y1 * Y3 + 0.5 * Y2 ** 2
        da = (Y3, Y2, Y1)                        # da/dx1, da/dx2, da/dx3
        u = s[0] * s[1] * s[2]
        grad = (np.pi * c[0] * s[1] * s[2], np.pi * s[0] * c[1] * s[2], np.pi * s[0] * s[1] * c[2])
        f = 3 * np.pi ** 2 * aa * u - sum(dk * gk for dk, gk in zip(da, grad))
        M, K = fe.fe_matrices_var(a)
        uh = spla.spsolve(K.tocsc(), M @ f.ravel())
        return np.abs(uh - u.ravel()).max()

    e1, e2 = err(7), err(15)
    assert 3.3 < e1 / e2 < 4.8, (e1, e2)


def test_stiffness_derivative_equals_central_differences_in_3d():
    m1, d = 3, 3
    a = np.exp(0.3 * S.random_vector((m1 + 2,) * d, 32))
    u = S.random_vector((2, m1, m1, m1), 33)
    v = S.random_vector((2, m1, m1, m1), 34)
    Sd = fe.stiffness_derivative(u, v, a)

    def form(ax):
        _, K = fe.fe_matrices_var(ax)
        return sum(float(u[t].ravel() @ (K @ v[t].ravel())) for t in range(2))

    h = 1e-6
    for P in [(1, 1, 1), (2, 3, 1), (3, 3, 3), (1, 2, 3)]:
        ap, am = a.copy(), a.copy()
        ap[P] *= math.exp(h)
        am[P] *= math.exp(-h)
        fd = (form(ap) - form(am)) / (2 * h)
        assert abs(fd - Sd[P[0] - 1, P[1] - 1, P[2] - 1]) <= 1e-7 * abs(fd)


def _vcycle_by_loops_d(a_nodes, tau, sigma, r):
    """_vcycle_by_loops for any dimension: Gauss-Seidel over the 2^d colours in order."""
    d = a_nodes.ndim
    m = a_nodes.shape[0] - 2
    M, K = fe.fe_matrices_var(a_nodes)
    A = sigma * M.toarray() + tau * K.toarray()
    N = m ** d
    if m == 1:
        return r / A[0, 0]
    col = fe.colour_of(m, d).ravel()
    u = np.zeros(N, dtype=complex)
    for c in range(2 ** d):
        for pnt in range(N):
            if col[pnt] != c:
                continue
            u[pnt] = (r[pnt] - sum(A[pnt, q] * u[q] for q in range(N) if q != pnt)) / A[pnt, pnt]
    res = r - A @ u
    P = _prolongation_matrix((m - 1) // 2, d)
    ec = _vcycle_by_loops_d(a_nodes[(slice(None, None, 2),) * d], tau, sigma, P.T @ res)
    return u + P @ ec


def test_vcycle_equals_the_point_by_point_cycle_in_3d():
    m1 = 3
    a = np.exp(0.4 * S.random_vector((m1 + 2,) * 3, 35))
    tau = 0.05
    mg = fe.MGSpatialSolverFE(a, tau)
    sig = np.array([0.7 + 0.4j, 1e-2 + 0.3j])
    r = S.random_vector((2, m1, m1, m1), 36) + 1j * S.random_vector((2, m1, m1, m1), 37)
    got = mg(sig, r)
    for k in range(2):
        ref = _vcycle_by_loops_d(a, tau, sig[k], r[k].ravel())
        assert np.abs(got[k].ravel() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_preconditioned_gmres_converges_in_few_iterations_in_3d():
    m1, n, gamma = 7, 8, 1e-3
    a = np.exp(0.4 * S.random_vector((m1 + 2,) * 3, 38))
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    M, K = fe.fe_matrices_var(a)
    mg = fe.MGSpatialSolverFE(a, tau)
    b = fe.build_rhs(S.random_vector((n, m1, m1, m1), 39), S.random_vector((n, m1, m1, m1), 40),
                     S.random_vector((m1, m1, m1), 41), tau, gamma, M)
    res = okr.gmres(lambda v: fe.apply_A(v, M, K, tau, alpha),
                    lambda v: opc.apply_Peps_inv(v, n, alpha, math.sqrt(tau), mg), b, rtol=1e-10, maxit=80,
                    mode="right")
    assert res.converged and res.iters <= 40
