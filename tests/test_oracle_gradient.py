"""Pins of the oracle's gradient: three independent routes must agree --
the envelope (Lagrangian) closed form, the adjoint solve, and central finite
differences of the re-solved objective."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import system as sy, gradient as gr


def _solve(a, g, f, y0, n, gamma, T=1.0):
    m1 = a.shape[0] - 2
    d = a.ndim
    K = sy.K_sparse(a).toarray()
    tau, alpha = sy.time_step(T, n), sy.alpha_weight(T, n, gamma)
    A = sy.A_dense(K, n, tau, alpha)
    b = sy.build_rhs(f, g, y0, tau, gamma)
    return np.linalg.solve(A, b.ravel()).reshape((2, n) + (m1,) * d), A, tau


@pytest.mark.parametrize("d,m1,n,gamma", [(2, 3, 4, 1e-2), (2, 4, 3, 1e-4), (3, 2, 3, 1e-1)])
def test_envelope_equals_adjoint_equals_finite_differences(d, m1, n, gamma):
    loga = 0.3 * S.random_vector((m1 + 2,) * d, 40)
    g = S.random_vector((n,) + (m1,) * d, 41)
    f = 0.5 * S.random_vector((n,) + (m1,) * d, 42)
    y0 = S.random_vector((m1,) * d, 43)
    a = np.exp(loga)
    x, A, tau = _solve(a, g, f, y0, n, gamma)
    env_a, env_g = gr.envelope_gradient(x, g, a, tau, gamma)
    rhs = gr.objective_grad_x(x, g, tau, gamma)
    lam = np.linalg.solve(A.T, rhs.ravel()).reshape(x.shape)
    adj_a, adj_g = gr.adjoint_gradient(x, lam, g, a, tau, gamma)
    scale_a = np.abs(env_a).max()
    assert np.abs(env_a - adj_a).max() <= 1e-10 * scale_a
    assert np.abs(env_g - adj_g).max() <= 1e-10 * np.abs(env_g).max()

    def J(la, gg):
        xx, _, tt = _solve(np.exp(la), gg, f, y0, n, gamma)
        return gr.objective(xx, gg, tt, gamma)

    h = 1e-6
    rng = np.random.default_rng(44)
    inner = (slice(1, -1),) * d
    for _ in range(4):
        da = np.zeros_like(loga)
        da[inner] = rng.standard_normal((m1,) * d)
        dg = rng.standard_normal(g.shape)
        fd = (J(loga + h * da, g + h * dg) - J(loga - h * da, g - h * dg)) / (2 * h)
        an = np.sum(env_a * da[inner]) + np.sum(env_g * dg)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12) + 1e-10, (fd, an)


def test_gradient_of_boundary_free_constant_rescaling():
    # scaling a -> c a everywhere scales K by c; d/dc J at c=1 equals the sum of
    # dJ/dlog a over interior nodes plus the boundary-node terms.  With a = const
    # and all boundary faces involving boundary nodes, check against FD directly.
    d, m1, n, gamma = 2, 3, 3, 1e-2
    a = np.ones((m1 + 2,) * d)
    g = S.random_vector((n, m1, m1), 45)
    f = np.zeros_like(g)
    y0 = np.zeros((m1, m1))
    x, A, tau = _solve(a, g, f, y0, n, gamma)
    env_a, _ = gr.envelope_gradient(x, g, a, tau, gamma)

    def J(c_int):
        aa = a.copy()
        aa[1:-1, 1:-1] *= c_int
        xx, _, tt = _solve(aa, g, f, y0, n, gamma)
        return gr.objective(xx, g, tt, gamma)

    h = 1e-6
    fd = (J(1 + h) - J(1 - h)) / (2 * h)
    assert abs(fd - env_a.sum()) <= 1e-6 * abs(fd)
