"""Oracle: the all-at-once system with a finite-element discretisation in space
(Section 1: mass matrix M != I and stiffness matrix K).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain FP64 numpy / scipy.

Discretisation: conforming bilinear (2D) / trilinear (3D) elements on the uniform
grid of the unit box with mesh width h = 1/(m1+1), homogeneous Dirichlet boundary,
constant coefficient a = c.  Both matrices are Kronecker products of the 1D linear
element matrices
    M_1 = h/6 tridiag(1, 4, 1),     K_1 = 1/h tridiag(-1, 2, -1):
    M = M_1 (x) ... (x) M_1,        K = c sum_axis (M_1 (x) .. K_1 .. (x) M_1).
Field conventions are those of ``oracle.system`` (last axis = x1, flattened row-major,
so the Kronecker factor of x1 is the last one).

With the backward-Euler steps of Section 1 and x = [sqrt(gamma) y; p]:
    A = [[alpha I (x) M, T^T], [-T, alpha I (x) M]],   T = B_n (x) M + tau I_n (x) K,
    b = [tau (I (x) M) g (+ M p^(N) at j = n);  -sqrt(gamma) (tau (I (x) M) f + M y^(0) e_1)],
and P_eps keeps its form with C_eps = C_{eps,n} (x) M + tau I_n (x) K, so the four-step
apply (``oracle.precond.apply_Peps_inv``) needs spatial solvers for (sigma M + tau K).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import precond, system


# ----------------------------------------------------------------------------
# element matrices                                                  (Section 1)
# ----------------------------------------------------------------------------


def fe_1d(m1: int):
    """1D linear-element mass and stiffness matrices on m1 interior nodes."""
    h = system.mesh_width(m1)
    M1 = sp.diags([np.full(m1 - 1, h / 6), np.full(m1, 4 * h / 6), np.full(m1 - 1, h / 6)], [-1, 0, 1])
    K1 = sp.diags([np.full(m1 - 1, -1 / h), np.full(m1, 2 / h), np.full(m1 - 1, -1 / h)], [-1, 0, 1])
    return M1.tocsr(), K1.tocsr()


def fe_matrices(m1: int, d: int, coeff: float = 1.0):
    """(M, K) of the Q1 discretisation (Kronecker form, sparse)."""
    M1, K1 = fe_1d(m1)
    M = M1
    for _ in range(d - 1):
        M = sp.kron(M1, M).tocsr()
    K = None
    for ax in range(d):  # ax 0 = x1 = the last Kronecker factor
        facs = [K1 if a == ax else M1 for a in range(d)]
        term = facs[d - 1]
        for a in range(d - 2, -1, -1):
            term = sp.kron(term, facs[a]).tocsr()
        K = term if K is None else K + term
    return M, (coeff * K).tocsr()


def fe_matrices_by_elements(m1: int, d: int, coeff: float = 1.0):
    """The same matrices assembled element by element from the reference-element
    integrals (tensor-product Gauss rule, exact for these polynomials), for pinning."""
    h = system.mesh_width(m1)
    g = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
    corners = list(np.ndindex(*(2,) * d))
    nloc = len(corners)

    def shape(xi):  # values and gradients of the 2^d local bilinear functions
        vals = np.ones(nloc)
        grads = np.ones((nloc, d))
        for q, c in enumerate(corners):
            for a in range(d):
                phi = xi[a] if c[a] else 1.0 - xi[a]
                dphi = 1.0 if c[a] else -1.0
                vals[q] *= phi
                for b in range(d):
                    grads[q, b] *= dphi if a == b else phi
        return vals, grads / h

    Me = np.zeros((nloc, nloc))
    Ke = np.zeros((nloc, nloc))
    for pt in np.ndindex(*(2,) * d):
        xi = g[list(pt)]
        v, gr = shape(xi)
        wq = (0.5 ** d) * h ** d
        Me += wq * np.outer(v, v)
        Ke += wq * coeff * gr @ gr.T
    N = m1 + 2
    ms = m1 ** d
    rows, cols, mv, kv = [], [], [], []
    for el in np.ndindex(*(N - 1,) * d):  # element lower corner in node coordinates (axis order x1, x2, ..)
        glob = []
        for c in corners:
            node = [el[a] + c[a] for a in range(d)]
            if any(t == 0 or t == N - 1 for t in node):
                glob.append(-1)
            else:
                idx = 0
                for a in range(d - 1, -1, -1):  # x_d slowest ... x1 fastest
                    idx = idx * m1 + (node[a] - 1)
                glob.append(idx)
        for p_, gp in enumerate(glob):
            if gp < 0:
                continue
            for q_, gq in enumerate(glob):
                if gq < 0:
                    continue
                rows.append(gp)
                cols.append(gq)
                mv.append(Me[p_, q_])
                kv.append(Ke[p_, q_])
    M = sp.csr_matrix((mv, (rows, cols)), shape=(ms, ms))
    K = sp.csr_matrix((kv, (rows, cols)), shape=(ms, ms))
    return M, K


# ----------------------------------------------------------------------------
# the all-at-once operator and right-hand side
# ----------------------------------------------------------------------------


def _apply(Mat, v: np.ndarray) -> np.ndarray:
    """Mat applied to every time block of v (shape (n,) + spatial)."""
    n = v.shape[0]
    flat = v.reshape(n, -1)
    return (Mat @ flat.T).T.reshape(v.shape)


def apply_T(v, M, K, tau):
    """(T v)_j = M v_j - M v_{j-1} + tau K v_j, v_0 = 0."""
    Mv = _apply(M, v)
    out = Mv + tau * _apply(K, v)
    out[1:] -= Mv[:-1]
    return out


def apply_TT(v, M, K, tau):
    """(T^T v)_j = M v_j - M v_{j+1} + tau K v_j, v_{n+1} = 0."""
    Mv = _apply(M, v)
    out = Mv + tau * _apply(K, v)
    out[:-1] -= Mv[1:]
    return out


def apply_A(x, M, K, tau, alpha):
    """A x with A = [[alpha I (x) M, T^T], [-T, alpha I (x) M]]."""
    x1, x2 = x[0], x[1]
    y = np.empty(x.shape)
    y[0] = alpha * _apply(M, x1) + apply_TT(x2, M, K, tau)
    y[1] = -apply_T(x1, M, K, tau) + alpha * _apply(M, x2)
    return y


def apply_AT(x, M, K, tau, alpha):
    """A^T x = [[alpha I (x) M, -T^T], [T, alpha I (x) M]] x (M, K symmetric)."""
    x1, x2 = x[0], x[1]
    y = np.empty(x.shape)
    y[0] = alpha * _apply(M, x1) - apply_TT(x2, M, K, tau)
    y[1] = apply_T(x1, M, K, tau) + alpha * _apply(M, x2)
    return y


def A_dense(M, K, n, tau, alpha):
    """Dense A from the Kronecker form (tiny sizes only)."""
    Md, Kd = M.toarray(), K.toarray()
    T = np.kron(system.B_matrix(n), Md) + tau * np.kron(np.eye(n), Kd)
    IM = np.kron(np.eye(n), Md)
    return np.block([[alpha * IM, T.T], [-T, alpha * IM]])


def P_eps_dense(M, K, n, tau, alpha, eps):
    """P_eps = 1/2 blockdiag(C_eps^T + alpha I (x) M, C_eps + alpha I (x) M) [[I, I], [-I, I]],
    C_eps = C_{eps,n} (x) M + tau I_n (x) K."""
    Md, Kd = M.toarray(), K.toarray()
    nm = n * Md.shape[0]
    Ce = np.kron(precond.C_eps_matrix(n, eps), Md) + tau * np.kron(np.eye(n), Kd)
    IM = np.kron(np.eye(n), Md)
    Z = np.zeros((nm, nm))
    H = np.block([[Ce.T + alpha * IM, Z], [Z, Ce + alpha * IM]])
    R = np.block([[np.eye(nm), np.eye(nm)], [-np.eye(nm), np.eye(nm)]])
    return 0.5 * H @ R


def build_rhs(f, g, y0, tau, gamma, M, p_final=None):
    """b = [tau M g_j (+ M p^(N) at j = n);  -sqrt(gamma) (tau M f_j + [j = 1] M y^(0))]."""
    gv = tau * _apply(M, g)
    if p_final is not None:
        gv[-1] += (M @ p_final.ravel()).reshape(p_final.shape)
    fv = tau * _apply(M, f)
    fv[0] += (M @ y0.ravel()).reshape(y0.shape)
    return np.stack([gv, -math.sqrt(gamma) * fv])


def end_point_solves(y, p, M, K, tau, gamma, f_T, g_0, y0, p_final=None):
    """(M + tau K) y^(N) = M y^(N-1) + tau M f^(N) + (tau/gamma) M p^(N);
    (M + tau K) p^(0) = M p^(1) + tau M g^(0) - tau M y^(0)."""
    shape = y.shape[1:]
    E = (M + tau * K).tocsc()
    pN = np.zeros(shape) if p_final is None else p_final
    rhs_y = M @ (y[-1] + tau * f_T + (tau / gamma) * pN).ravel()
    rhs_p = M @ (p[0] + tau * g_0 - tau * y0).ravel()
    return spla.spsolve(E, rhs_y).reshape(shape), spla.spsolve(E, rhs_p).reshape(shape)


# ----------------------------------------------------------------------------
# spatial solvers for (sigma_k M + tau K) z_k = r_k
# ----------------------------------------------------------------------------


class DenseSpatialSolverFE:
    """Exact solves with the dense matrix sigma M + tau K (tiny sizes)."""

    def __init__(self, M, K, tau: float, shape):
        self.M, self.K, self.tau, self.shape = M.toarray(), K.toarray(), tau, shape

    def __call__(self, sigma, R):
        out = np.empty(R.shape, dtype=complex)
        ms = self.M.shape[0]
        for k in range(R.shape[0]):
            out[k] = np.linalg.solve(sigma[k] * self.M + self.tau * self.K, R[k].reshape(ms)).reshape(self.shape)
        return out


def fe_eigenvalues(m1: int, d: int, coeff: float = 1.0):
    """Eigenvalues of M and K on the DST-I basis: 1D mu_M(i) = h/6 (4 + 2 cos(pi i/(m1+1))),
    mu_K(i) = (2 - 2 cos(pi i/(m1+1)))/h; products and sums over the axes."""
    h = system.mesh_width(m1)
    th = math.pi * np.arange(1, m1 + 1) / (m1 + 1)
    mM = h / 6.0 * (4.0 + 2.0 * np.cos(th))
    mK = (2.0 - 2.0 * np.cos(th)) / h
    lamM = np.ones((m1,) * d)
    lamK = np.zeros((m1,) * d)
    for ax in range(d):
        shp = [1] * d
        shp[d - 1 - ax] = m1
        lamM = lamM * mM.reshape(shp)
    for ax in range(d):
        term = np.ones((m1,) * d)
        for b in range(d):
            shp = [1] * d
            shp[d - 1 - b] = m1
            term = term * (mK if b == ax else mM).reshape(shp)
        lamK = lamK + term
    return lamM, coeff * lamK


class FSTSpatialSolverFE:
    """Exact solves of (sigma M + tau K) z = r by the sine transform: M and K are
    Kronecker products of tridiagonal Toeplitz matrices, all diagonal on DST-I."""

    def __init__(self, m1: int, d: int, tau: float, coeff: float = 1.0):
        self.d, self.tau = d, tau
        self.S = precond.dst1_matrix(m1)
        self.lamM, self.lamK = fe_eigenvalues(m1, d, coeff)

    def _transform(self, R):
        out = R
        for ax in range(self.d):
            out = np.moveaxis(np.tensordot(self.S, out, axes=([1], [1 + ax])), 0, 1 + ax)
        return out

    def __call__(self, sigma, R):
        Rh = self._transform(R)
        den = sigma.reshape((-1,) + (1,) * self.d) * self.lamM[None] + self.tau * self.lamK[None]
        return self._transform(Rh / den)
