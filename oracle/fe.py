"""Oracle: the all-at-once system with a finite-element discretisation in space
(Section 1: mass matrix M != I and stiffness matrix K).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain FP64 numpy / scipy.

Discretisation: conforming bilinear (2D) / trilinear (3D) elements on the uniform
grid of the unit box with mesh width h = 1/(m1+1), homogeneous Dirichlet boundary.
With a constant coefficient a = c both matrices are Kronecker products of the 1D
linear element matrices
    M_1 = h/6 tridiag(1, 4, 1),     K_1 = 1/h tridiag(-1, 2, -1):
    M = M_1 (x) ... (x) M_1,        K = c sum_axis (M_1 (x) .. K_1 .. (x) M_1).
With a variable coefficient given at the nodes (reading: the coefficient of element
e is the value of the nodal interpolant at its centre, a_e = mean of its 2^d corner
values, and the element integral of grad phi_p . grad phi_q is exact),
    K(a) = sum_e a_e K_e,   K_e the element matrix of a = 1;  M as above.
Its shifted systems (sigma M + tau K(a)) are solved by one multigrid V(1,0) cycle
(``MGSpatialSolverFE``).
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


def element_coefficients(a_nodes: np.ndarray) -> np.ndarray:
    """a_e = mean of the 2^d corner values of element e (the nodal interpolant at the
    element centre); a_nodes has shape (m1+2,)*d with x1 last, the result (m1+1,)*d."""
    d = a_nodes.ndim
    ne = a_nodes.shape[0] - 1
    out = np.zeros((ne,) * d)
    for c in np.ndindex(*(2,) * d):
        out += a_nodes[tuple(slice(ci, ci + ne) for ci in c)]
    return out / 2 ** d


def fe_matrices_var(a_nodes: np.ndarray):
    """(M, K(a)) for a nodal coefficient, element by element (K(a) = sum_e a_e K_e)."""
    d = a_nodes.ndim
    return fe_matrices_by_elements(a_nodes.shape[0] - 2, d, element_coefficients(a_nodes))


def reference_element(m1: int, d: int):
    """Corner list (offsets along x1, x2, ..) and the element mass and stiffness matrices
    of one element of width h = 1/(m1+1) for a = 1, from a tensor-product Gauss rule
    (exact for these polynomials)."""
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
        Ke += wq * gr @ gr.T
    return corners, Me, Ke


def fe_matrices_by_elements(m1: int, d: int, coeff=1.0):
    """The same matrices assembled element by element from the reference-element
    integrals, for pinning.  coeff: a constant, or one value per element (shape
    (m1+1,)*d, x1 last)."""
    corners, Me, Ke = reference_element(m1, d)
    cel = np.broadcast_to(np.asarray(coeff, dtype=float), (m1 + 1,) * d)
    N = m1 + 2
    ms = m1 ** d
    rows, cols, mv, kv = [], [], [], []
    for el in np.ndindex(*(N - 1,) * d):  # element lower corner in node coordinates (axis order x1, x2, ..)
        ce = cel[tuple(el[::-1])]         # coefficient arrays index x_d first, x1 last
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
                kv.append(ce * Ke[p_, q_])
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


# ----------------------------------------------------------------------------
# variable coefficient: multigrid for (sigma M + tau K(a))
# ----------------------------------------------------------------------------


def colour_of(m: int, d: int) -> np.ndarray:
    """Colour of each interior point (shape (m,)*d, x1 last): c = sum_k (i_k & 1) 2^k with
    i_k the 0-based index along x_{k+1}.  The 3^d-point element stencils never couple two
    points of one colour."""
    idx = np.indices((m,) * d)          # idx[0] is the x_d index ... idx[d-1] the x1 index
    c = np.zeros((m,) * d, dtype=int)
    for k in range(d):
        c += (idx[d - 1 - k] & 1) << k
    return c


def restrict_transpose(r: np.ndarray, d: int) -> np.ndarray:
    """P^T, the transpose of the (bi/tri)linear interpolation: 2^d times full weighting
    (weights 1 at the coincident fine point, 1/2 and 1/4 at its neighbours)."""
    return (2 ** d) * precond.restrict_full_weighting(r, d)


class MGLevelFE:
    def __init__(self, a_nodes: np.ndarray):
        self.d = a_nodes.ndim
        self.m = a_nodes.shape[0] - 2
        self.M, self.K = fe_matrices_var(a_nodes)
        self.colour = colour_of(self.m, self.d).ravel()


class MGSpatialSolverFE:
    """One V(1,0) cycle per shifted system (sigma_k M + tau K(a)) z_k = r_k, the analogue
    of the finite-difference cycle for element matrices:
      * levels m -> (m-1)/2 -> ... -> 1, the nodal coefficient injected (a_c(I) = a(2I)),
        each level's M and K(a) assembled on its own grid;
      * pre-smoothing: one Gauss-Seidel sweep from zero in colour order (colours 0, 1, ..,
        2^d - 1 of ``colour_of``; points of one colour are independent);
      * residual, restriction by P^T, recursion, correction by bilinear interpolation P,
        no post-smoothing; the one-point level is solved exactly."""

    def __init__(self, a_nodes: np.ndarray, tau: float):
        m = a_nodes.shape[0] - 2
        if m < 1 or (m + 1) & m:
            raise ValueError("multigrid needs m1 = 2^k - 1")
        self.tau = tau
        self.d = a_nodes.ndim
        self.levels = []
        a = a_nodes
        while True:
            self.levels.append(MGLevelFE(a))
            if a.shape[0] - 2 == 1:
                break
            a = a[(slice(None, None, 2),) * self.d]

    def _op(self, lev: MGLevelFE, sigma: np.ndarray, U: np.ndarray) -> np.ndarray:
        """(sigma_k M + tau K) u_k for every plane k; U has shape (planes, m^d)."""
        return (lev.M @ U.T).T * sigma[:, None] + self.tau * (lev.K @ U.T).T

    def vcycle(self, l: int, sigma: np.ndarray, r: np.ndarray) -> np.ndarray:
        lev = self.levels[l]
        P = r.shape[0]
        R = r.reshape(P, -1)
        dg = sigma[:, None] * lev.M.diagonal()[None] + self.tau * lev.K.diagonal()[None]
        if lev.m == 1:
            return (R / dg).reshape(r.shape)
        U = np.zeros_like(R)
        for c in range(2 ** self.d):
            sel = lev.colour == c
            # the colour's own values are still zero, so (A u) holds only its neighbours
            U[:, sel] = (R[:, sel] - self._op(lev, sigma, U)[:, sel]) / dg[:, sel]
        res = (R - self._op(lev, sigma, U)).reshape(r.shape)
        ec = self.vcycle(l + 1, sigma, restrict_transpose(res, self.d))
        return U.reshape(r.shape) + precond.prolong_linear(ec, self.d)

    def __call__(self, sigma: np.ndarray, R: np.ndarray) -> np.ndarray:
        return self.vcycle(0, np.asarray(sigma, dtype=complex), R.astype(complex))


# ----------------------------------------------------------------------------
# objective and gradient with element matrices
# ----------------------------------------------------------------------------


def objective(x: np.ndarray, g: np.ndarray, M, tau: float, gamma: float) -> float:
    """J_h = tau [1/2 sum_j (y_j - g_j)^T M (y_j - g_j) + 1/(2 gamma) sum_j p_j^T M p_j]
    (the finite-difference J_h with h^d I replaced by M)."""
    y, p = system.unscale(x, gamma)
    e = y - g
    return tau * (0.5 * float(np.sum(e * _apply(M, e))) + 0.5 / gamma * float(np.sum(p * _apply(M, p))))


def objective_grad_x(x: np.ndarray, g: np.ndarray, M, tau: float, gamma: float) -> np.ndarray:
    y, p = system.unscale(x, gamma)
    return np.stack([tau * _apply(M, y - g) / math.sqrt(gamma), tau * _apply(M, p) / gamma])


def stiffness_derivative(u: np.ndarray, v: np.ndarray, a_nodes: np.ndarray) -> np.ndarray:
    """S_P = sum over the leading (time) axis of u^T (dK/d log a_P) v.  a_P enters the
    coefficients of the 2^d elements around P with weight 1/2^d, so
    S_P = a_P / 2^d sum_{e around P} B_e,  B_e = sum_time u_e^T K_e v_e,
    K_e the element stiffness of a = 1 and u_e, v_e the values at e's corners (zero on
    boundary nodes)."""
    d = a_nodes.ndim
    m1 = a_nodes.shape[0] - 2
    corners, _, Ke = reference_element(m1, d)
    pad = [(0, 0)] + [(1, 1)] * d
    up, vp = np.pad(u, pad), np.pad(v, pad)

    def at_corner(w, c):  # values at corner c of every element, shape (time,) + (m1+1,)*d
        return w[(slice(None),) + tuple(slice(c[a], c[a] + m1 + 1) for a in range(d - 1, -1, -1))]

    B = np.zeros((m1 + 1,) * d)
    for p_, cp in enumerate(corners):
        for q_, cq in enumerate(corners):
            B += Ke[p_, q_] * np.sum(at_corner(up, cp) * at_corner(vp, cq), axis=0)
    S = np.zeros((m1,) * d)
    for c in np.ndindex(*(2,) * d):  # the element with lower corner P - c (in node coordinates) contains P
        S += B[tuple(slice(1 - ci, 1 - ci + m1) for ci in c)]
    return a_nodes[(slice(1, -1),) * d] * S / 2 ** d


def envelope_gradient(x: np.ndarray, g: np.ndarray, a_nodes: np.ndarray, M, tau: float, gamma: float):
    """dJ*/d log a_P = tau sum_j p_j^T (dK/d log a_P) y_j,  dJ*/dg_j = -tau M (y_j - g_j)."""
    y, p = system.unscale(x, gamma)
    return tau * stiffness_derivative(p, y, a_nodes), -tau * _apply(M, y - g)


def adjoint_gradient(x: np.ndarray, lam: np.ndarray, g: np.ndarray, a_nodes: np.ndarray, M, tau: float,
                     gamma: float):
    """dJ/dtheta|_x + lam^T (db/dtheta - dA/dtheta x), A^T lam = dJ/dx, with
    dA/d log a_P = tau [[0, I (x) K'_P], [-I (x) K'_P, 0]] and db_1/dg_j = tau M."""
    y, _ = system.unscale(x, gamma)
    g_loga = -tau * (stiffness_derivative(lam[0], x[1], a_nodes) - stiffness_derivative(lam[1], x[0], a_nodes))
    g_g = -tau * _apply(M, y - g) + tau * _apply(M, lam[0])
    return g_loga, g_g
