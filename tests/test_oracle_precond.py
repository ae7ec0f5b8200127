"""Pins of the oracle's preconditioner (Eqs. matrix_P_eps, decomposition_eps,
Section 2.1) and Krylov solver (Lemma 2.1, Theorems 2.3, 2.6, 2.13) against
dense definitions, textbook identities and the paper's theorems."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import system as sy, precond as pc, krylov as kr


def _setup(d, m1, n, gamma=1e-3, T=1.0, seed=0, const=False):
    a = np.full((m1 + 2,) * d, 1.0) if const else np.exp(0.4 * S.random_vector((m1 + 2,) * d, seed))
    K = sy.K_sparse(a).toarray()
    tau, alpha = sy.time_step(T, n), sy.alpha_weight(T, n, gamma)
    return a, K, tau, alpha


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 16])
@pytest.mark.parametrize("eps", [1.0, 0.5, 0.05])
def test_eps_circulant_diagonalisation(n, eps):
    # Eq. decomposition_eps against the definition Eq. matrix_C_eps_n
    C = pc.C_eps_matrix(n, eps)
    D = np.diag(pc.D_eps_diag(n, eps))
    F = pc.fourier_matrix(n)
    L = np.diag(pc.eigenvalues_lambda(n, eps))
    assert np.allclose(F @ F.conj().T, np.eye(n), atol=1e-13)
    assert np.abs(np.linalg.inv(D) @ F @ L @ F.conj().T @ D - C).max() < 1e-13
    # the eigenvalues are those of C itself
    ev = np.linalg.eigvals(C)
    lam = np.diag(L)
    assert max(np.abs(lam - e).min() for e in ev) < 1e-7
    assert max(np.abs(ev - l).min() for l in lam) < 1e-7


def test_eps_circulant_corner_entry():
    C = pc.C_eps_matrix(5, 0.3)
    assert C[0, 4] == -0.3 and C[1, 0] == -1 and C[0, 0] == 1 and np.count_nonzero(C) == 10


@pytest.mark.parametrize("d,m1,n,eps", [(2, 3, 5, 0.3), (2, 3, 4, 0.5), (2, 2, 1, 1.0),
                                        (2, 3, 2, 0.1), (3, 2, 3, 0.2), (2, 4, 6, 0.02)])
def test_four_step_apply_matches_dense_P_eps(d, m1, n, eps):
    a, K, tau, alpha = _setup(d, m1, n, seed=d + m1 + n)
    P = pc.P_eps_dense(K, n, tau, alpha, eps)
    v = S.random_vector((2, n) + (m1,) * d, 20)
    ref = np.linalg.solve(P, v.ravel())
    got = pc.apply_Peps_inv(v, n, alpha, eps, pc.DenseSpatialSolver(a, tau))
    assert np.linalg.norm(got.ravel() - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,m1", [(2, 5), (2, 8), (3, 3)])
def test_fst_solver_matches_dense_solve(d, m1):
    a, K, tau, _ = _setup(d, m1, 4, const=True)
    sig = np.array([0.3 + 0.7j, 2.0 - 0.1j, 1e-3 + 0j])
    R = S.random_vector((3,) + (m1,) * d, 3) + 1j * S.random_vector((3,) + (m1,) * d, 4)
    got = pc.FSTSpatialSolver(m1, d, tau)(sig, R)
    ref = pc.DenseSpatialSolver(a, tau)(sig, R)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_dst1_matrix_orthonormal_and_diagonalises_second_difference():
    m = 9
    Smat = pc.dst1_matrix(m)
    assert np.allclose(Smat @ Smat, np.eye(m), atol=1e-13)
    L = (2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1))
    D = Smat @ L @ Smat
    mu = 4 * np.sin(math.pi * np.arange(1, m + 1) / (2 * (m + 1))) ** 2
    assert np.allclose(D, np.diag(mu), atol=1e-12)


def test_P_eps_tends_to_ideal_P_linearly_in_eps():
    a, K, tau, alpha = _setup(2, 3, 6)
    v = S.random_vector(2 * 6 * 9, 5)
    ref = np.linalg.solve(pc.P_dense(K, 6, tau, alpha), v)
    errs = [np.linalg.norm(np.linalg.solve(pc.P_eps_dense(K, 6, tau, alpha, e), v) - ref)
            for e in (1e-2, 1e-3, 1e-4)]
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 8


@pytest.mark.parametrize("d,m1,n", [(2, 3, 5), (2, 4, 1), (2, 2, 3), (3, 2, 3), (2, 3, 8)])
def test_ideal_P_block_substitution_matches_dense_P(d, m1, n):
    # Eq. matrix_P assembled densely and solved by LU, against the sequential
    # forward / backward substitution in time with exact spatial solves
    a, K, tau, alpha = _setup(d, m1, n, seed=3 * d + m1 + n)
    v = S.random_vector((2, n) + (m1,) * d, 31)
    ref = np.linalg.solve(pc.P_dense(K, n, tau, alpha), v.ravel())
    got = pc.apply_P_inv(v, n, alpha, pc.DenseSpatialSolver(a, tau))
    assert np.linalg.norm(got.ravel() - ref) <= 1e-12 * np.linalg.norm(ref)


def test_ideal_P_with_sine_transforms_equals_dense_solves():
    a, K, tau, alpha = _setup(2, 7, 6, const=True)
    v = S.random_vector((2, 6, 7, 7), 32)
    got = pc.apply_P_inv(v, 6, alpha, pc.FSTSpatialSolver(7, 2, tau))
    ref = pc.apply_P_inv(v, 6, alpha, pc.DenseSpatialSolver(a, tau))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_ideal_P_is_the_eps_to_zero_limit_of_the_four_step_apply():
    # P_eps -> P as eps -> 0 (the eps-circulant corner entry vanishes): the two
    # independent routes (FFT diagonalisation vs block substitution) meet linearly
    a, K, tau, alpha = _setup(2, 3, 8)
    v = S.random_vector((2, 8, 3, 3), 33)
    sp = pc.DenseSpatialSolver(a, tau)
    ref = pc.apply_P_inv(v, 8, alpha, sp)
    errs = [np.linalg.norm(pc.apply_Peps_inv(v, 8, alpha, e, sp) - ref) / np.linalg.norm(ref)
            for e in (1e-3, 1e-4, 1e-5)]
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 8 and errs[2] < 1e-4


@pytest.mark.parametrize("gamma", [1e-8, 1e-4, 1.0])
def test_theorem_ideal_spectrum_on_the_line_re_1(gamma):
    # Theorem 2.3 (M = I): sigma(P^{-1} A) lies in {1 + i x, |x| <= 1}
    a, K, tau, alpha = _setup(2, 3, 5, gamma=gamma)
    A = sy.A_dense(K, 5, tau, alpha)
    ev = np.linalg.eigvals(np.linalg.solve(pc.P_dense(K, 5, tau, alpha), A))
    assert np.abs(ev.real - 1).max() < 1e-8
    assert np.abs(ev.imag).max() <= 1 + 1e-10


def _H_blocks(K, n, tau, alpha, eps=None):
    ms = K.shape[0]
    Bt = pc.C_eps_matrix(n, eps) if eps is not None else sy.B_matrix(n)
    Cb = np.kron(Bt, np.eye(ms)) + tau * np.kron(np.eye(n), K) + alpha * np.eye(n * ms)
    Z = np.zeros_like(Cb)
    return np.block([[Cb.T, Z], [Z, Cb]])


@pytest.mark.parametrize("eps", [0.5, 0.1, 0.01])
def test_theorem_low_rank_and_eigenvalue_bound(eps):
    # Theorem 2.6: rank(H_eps^{-1} H - I) = 2m and |lambda - 1| <= eps/(1-eta), eps <= eta
    n, m1 = 5, 3
    a, K, tau, alpha = _setup(2, m1, n)
    H = _H_blocks(K, n, tau, alpha)
    He = _H_blocks(K, n, tau, alpha, eps)
    E = np.linalg.solve(He, H) - np.eye(H.shape[0])
    sv = np.linalg.svd(E, compute_uv=False)
    assert int(np.sum(sv > 1e-10 * sv[0])) == 2 * m1 * m1
    ev = np.linalg.eigvals(np.linalg.solve(He, H))
    assert np.abs(ev - 1).max() <= eps / (1 - eps) + 1e-12


@pytest.mark.parametrize("eps", [0.5, 0.1])
def test_lemmas_norm_bounds(eps):
    # Lemma 2.7: ||(C+aI)^{-1}(T+aI) - I|| <= eps sqrt(n)/(1-eta);
    # Lemma 2.9: ||H_eps^{-1} B|| <= sqrt(2)(1 + eps sqrt(n)/(1-eta))
    n, m1 = 6, 3
    a, K, tau, alpha = _setup(2, m1, n)
    ms = K.shape[0]
    Tm = sy.T_dense(K, n, tau) + alpha * np.eye(n * ms)
    Cm = np.kron(pc.C_eps_matrix(n, eps), np.eye(ms)) + tau * np.kron(np.eye(n), K) + alpha * np.eye(n * ms)
    lhs = np.linalg.norm(np.linalg.solve(Cm, Tm) - np.eye(n * ms), 2)
    assert lhs <= eps * math.sqrt(n) / (1 - eps) + 1e-12
    T = sy.T_dense(K, n, tau)
    I = np.eye(n * ms)
    B = np.block([[T.T + alpha * I, T.T - alpha * I], [-T + alpha * I, T + alpha * I]])
    He = _H_blocks(K, n, tau, alpha, eps)
    assert np.linalg.norm(np.linalg.solve(He, B), 2) <= math.sqrt(2) * (1 + eps * math.sqrt(n) / (1 - eps)) + 1e-12
    # A = B G and P_eps = H_eps G (Section 2)
    G = 0.5 * np.block([[I, I], [-I, I]])
    assert np.allclose(B @ G, sy.A_dense(K, n, tau, alpha), atol=1e-12)
    assert np.allclose(He @ G, pc.P_eps_dense(K, n, tau, alpha, eps), atol=1e-12)


# ---------------------------------------------------------------------------- multigrid


def _dense_of(op, shape):
    size = int(np.prod(shape))
    cols = []
    for i in range(size):
        e = np.zeros(size)
        e[i] = 1
        cols.append(op(e.reshape((1,) + shape)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("d,mf", [(2, 7), (3, 7), (2, 3)])
def test_full_weighting_is_scaled_transpose_of_linear_interpolation(d, mf):
    mc = (mf - 1) // 2
    R = _dense_of(lambda r: pc.restrict_full_weighting(r, d), (mf,) * d)
    P = _dense_of(lambda e: pc.prolong_linear(e, d), (mc,) * d)
    assert np.allclose(R, P.T / 2 ** d, atol=1e-15)
    # interpolation is exact for a field that is linear in each coordinate on the
    # interior cells and reproduces coarse values at coincident fine points
    xc = np.arange(1, mc + 1) / (mc + 1)
    xf = np.arange(1, mf + 1) / (mf + 1)
    ec = np.ones((mc,) * d)
    fc = np.ones((mf,) * d)
    for k in range(d):
        shp = [1] * d
        shp[k] = -1
        ec = ec * (2.0 + xc.reshape(shp))
        fc = fc * (2.0 + xf.reshape(shp))
    ef = pc.prolong_linear(ec[None], d)[0]
    inner = (slice(1, -1),) * d
    assert np.allclose(ef[inner], fc[inner], atol=1e-14)


def test_multigrid_coarsest_level_is_exact():
    a = np.exp(0.3 * S.random_vector((3, 3), 2))       # m1 = 1
    tau = 0.1
    sol = pc.MGSpatialSolver(a, tau)
    sig = np.array([0.5 + 0.2j])
    r = np.array([[[1.7 - 0.3j]]])
    ref = pc.DenseSpatialSolver(a, tau)(sig, r)
    assert np.allclose(sol(sig, r), ref)


@pytest.mark.parametrize("smoother", ["red-black", "lexicographic"])
@pytest.mark.parametrize("d,m1", [(2, 15), (3, 7)])
def test_multigrid_vcycle_is_a_convergent_linear_approximate_inverse(d, m1, smoother):
    a = np.exp(0.5 * S.random_vector((m1 + 2,) * d, 7))
    tau = 1.0 / 17
    sol = pc.MGSpatialSolver(a, tau, smoother)
    dense = pc.DenseSpatialSolver(a, tau)
    sig = np.array([1 + 0.05 + 0j, 0.3 + 0.8j, 0.01 - 0.9j])   # lambda_k + alpha-like shifts
    r = S.random_vector((3,) + (m1,) * d, 8) + 1j * S.random_vector((3,) + (m1,) * d, 9)
    r2 = S.random_vector((3,) + (m1,) * d, 10) + 0j
    # linearity
    assert np.allclose(sol(sig, r + 2 * r2), sol(sig, r) + 2 * sol(sig, r2), atol=1e-12)
    # iterated defect correction with the V-cycle converges to the exact solution
    exact = dense(sig, r)
    u = np.zeros_like(r)
    norms = []
    for _ in range(25):
        res = r - (sig.reshape((-1,) + (1,) * d) * u + tau * sy.apply_K(u, a))
        u = u + sol(sig, res)
        norms.append(np.abs(u - exact).max() / np.abs(exact).max())
    assert norms[-1] < 1e-8, norms
    assert max(norms[i + 1] / norms[i] for i in range(4)) < 0.6


@pytest.mark.parametrize("d,m1", [(2, 7), (3, 3)])
def test_lexicographic_sweep_is_pointwise_gauss_seidel_in_the_natural_order(d, m1):
    # brute force: visit the points one by one in the natural order (x1 fastest) and
    # solve each row of the dense shifted matrix with the values computed so far
    a = np.exp(0.5 * S.random_vector((m1 + 2,) * d, 21))
    tau = 0.07
    sol = pc.MGSpatialSolver(a, tau, "lexicographic")
    lev = sol.levels[0]
    sig = np.array([0.6 + 0.4j, 1.1 - 0.2j])
    r = S.random_vector((2,) + (m1,) * d, 22) + 1j * S.random_vector((2,) + (m1,) * d, 23)
    dg = sig.reshape((-1,) + (1,) * d) + tau * lev.diagK[None]
    got = sol._lex_sweep(lev, dg, r)
    K = sy.K_sparse(a).toarray()
    ms = K.shape[0]
    for k in range(2):
        Ak = sig[k] * np.eye(ms) + tau * K
        rk = r[k].reshape(ms)
        u = np.zeros(ms, dtype=complex)
        for i in range(ms):  # flattened order = natural order, x1 fastest
            u[i] = (rk[i] - Ak[i, :i] @ u[:i]) / Ak[i, i]
        assert np.allclose(got[k].reshape(ms), u, rtol=0, atol=1e-13 * np.abs(u).max())


def test_red_black_sweep_leaves_zero_residual_on_black_points():
    m1, d = 7, 2
    a = np.exp(0.5 * S.random_vector((m1 + 2,) * d, 11))
    tau = 0.05
    sol = pc.MGSpatialSolver(a, tau)
    lev = sol.levels[0]
    sig = np.array([0.7 + 0.3j])
    r = S.random_vector((1, m1, m1), 12) + 0j
    # reproduce just the smoothing by forcing a zero coarse correction: coarse
    # residual is irrelevant for the black equations, which GS solves exactly
    dg = sig[:, None, None] + tau * lev.diagK[None]
    u = np.zeros_like(r)
    u[:, lev.red] = r[:, lev.red] / dg[:, lev.red]
    off = sol._op(lev, sig, u) - dg * u
    u[:, lev.black] = (r[:, lev.black] - off[:, lev.black]) / dg[:, lev.black]
    res = r - sol._op(lev, sig, u)
    assert np.abs(res[:, lev.black]).max() < 1e-13
    assert np.abs(res[:, lev.red]).max() > 1e-3


# ---------------------------------------------------------------------------- GMRES


@pytest.mark.parametrize("mode", ["left", "right"])
def test_gmres_iterate_is_the_krylov_minimiser(mode):
    # Lemma 2.1, by brute force on a tiny system
    d, m1, n, eps = 2, 2, 3, 0.3
    a, K, tau, alpha = _setup(d, m1, n)
    b = S.random_vector((2, n, m1, m1), 30)
    Aop = lambda v: sy.apply_A(v, a, tau, alpha)
    Pi = lambda v: pc.apply_Peps_inv(v, n, alpha, eps, pc.DenseSpatialSolver(a, tau))
    for j in (1, 2, 3):
        res = kr.gmres(Aop, Pi, b, rtol=0.0, maxit=j, mode=mode)
        if mode == "left":
            op = lambda v: Pi(Aop(v.reshape(b.shape))).ravel()
            rhs = Pi(b).ravel()
            xb = kr.krylov_minimiser(op, rhs, np.zeros(b.size), j)
        else:
            op = lambda u: Aop(Pi(u.reshape(b.shape))).ravel()
            ub = kr.krylov_minimiser(op, b.ravel(), np.zeros(b.size), j)
            xb = Pi(ub.reshape(b.shape)).ravel()
        assert np.allclose(res.x.ravel(), xb, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("mode", ["left", "right"])
def test_gmres_history_is_the_residual_of_each_iterate(mode):
    # the least-squares estimate after k steps equals the (preconditioned, for left)
    # relative residual of the k-th iterate, computed from the iterate itself
    d, m1, n, eps = 2, 3, 4, 0.3
    a, K, tau, alpha = _setup(d, m1, n)
    b = S.random_vector((2, n, m1, m1), 33)
    Aop = lambda v: sy.apply_A(v, a, tau, alpha)
    Pi = lambda v: pc.apply_Peps_inv(v, n, alpha, eps, pc.DenseSpatialSolver(a, tau))
    hist = kr.gmres(Aop, Pi, b, rtol=0.0, maxit=6, mode=mode).resid_history
    assert len(hist) == 7 and hist[0] == pytest.approx(1.0)
    for k in range(1, 7):
        xk = kr.gmres(Aop, Pi, b, rtol=0.0, maxit=k, mode=mode).x
        r = b - Aop(xk)
        if mode == "left":
            true = np.linalg.norm(Pi(r)) / np.linalg.norm(Pi(b))
        else:
            true = np.linalg.norm(r) / np.linalg.norm(b)
        assert hist[k] == pytest.approx(true, rel=1e-8, abs=1e-14)
        assert hist[k] <= hist[k - 1] * (1 + 1e-12)


def test_gmres_reaches_dense_solution():
    d, m1, n = 2, 3, 4
    a, K, tau, alpha = _setup(d, m1, n)
    b = S.random_vector((2, n, m1, m1), 31)
    Aop = lambda v: sy.apply_A(v, a, tau, alpha)
    Pi = lambda v: pc.apply_Peps_inv(v, n, alpha, 0.2, pc.DenseSpatialSolver(a, tau))
    res = kr.gmres(Aop, Pi, b, rtol=1e-13, maxit=100, mode="right")
    ref = np.linalg.solve(sy.A_dense(K, n, tau, alpha), b.ravel())
    assert np.linalg.norm(res.x.ravel() - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("gamma", [1e-8, 1e-4, 1e-1])
@pytest.mark.parametrize("n", [7, 15])
def test_theorem_gmres_rate_bound(gamma, n):
    # Theorem 2.13 with M = I (c0 = 1): for eps <= c_tau(delta) the preconditioned
    # residuals satisfy ||r_k|| <= rho(delta)^k ||r_0||
    delta = 0.5
    m1 = 7
    a, K, tau, alpha = _setup(2, m1, n, gamma=gamma)
    eps = sy.theorem_eps(1.0, n, delta)
    rho = sy.theorem_rate(delta)
    b = S.random_vector((2, n, m1, m1), 32)
    Aop = lambda v: sy.apply_A(v, a, tau, alpha)
    Pi = lambda v: pc.apply_Peps_inv(v, n, alpha, eps, pc.DenseSpatialSolver(a, tau))
    res = kr.gmres(Aop, Pi, b, rtol=1e-10, maxit=80, mode="left")
    assert res.converged
    for k, rk in enumerate(res.resid_history):
        assert rk <= rho ** k * (1 + 1e-9)


@pytest.mark.parametrize("n,eps", [(1, 0.5), (4, 0.3), (8, 1e-3), (31, 0.01), (32, 1.0)])
def test_transposed_block_is_the_time_reversal_of_the_block(n, eps):
    # C_eps is Toeplitz, so C^T = J C J with J the reversal of the time index, and the
    # transposed block of P_eps can be solved through the block itself:
    # (C^T + alpha I)^{-1} v = J (C + alpha I)^{-1} J v
    C = pc.C_eps_matrix(n, eps)
    J = np.eye(n)[::-1]
    assert np.array_equal(C.T, J @ C @ J)
    alpha = 0.37
    v = S.random_vector((n,), 40)
    lhs = np.linalg.solve(C.T + alpha * np.eye(n), v)
    rhs = J @ np.linalg.solve(C + alpha * np.eye(n), J @ v)
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(lhs).max()
    # and through the diagonalisation of C: J D^{-1} F (Lambda + alpha)^{-1} F^* D J v
    D = pc.D_eps_diag(n, eps)
    lam = pc.eigenvalues_lambda(n, eps)
    via = J @ ((np.fft.ifft(np.fft.fft(D * (J @ v)) / (lam + alpha)) / D).real)
    assert np.abs(via - lhs).max() <= 1e-12 / min(eps, 1.0) * np.abs(lhs).max()
