"""Oracle: the discrete all-at-once optimality system (Section 1).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain FP64 numpy, no
blocking or fusion beyond what the definitions state.

Array conventions (shared with ``synthetic``): interior spatial fields have
shape ``(m1,)*d`` with the last axis = x1; nodal coefficient fields have shape
``(m1+2,)*d``; space-time fields ``(n,)+(m1,)*d`` hold time levels j = 1..n;
an all-at-once vector has shape ``(2, n) + (m1,)*d`` = [half][time][space],
half 0 = sqrt(gamma) y, half 1 = p (Eq. main_system).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ----------------------------------------------------------------------------
# parameters (Section 1 and Section 3)
# ----------------------------------------------------------------------------


def mesh_width(m1: int) -> float:
    """h = 1/(m+1) (Section 3)."""
    return 1.0 / (m1 + 1)


def time_step(T: float, n: int) -> float:
    """tau = T/N with n = N - 1 time blocks, i.e. tau = T/(n+1) (Section 1, Lemma 2.12)."""
    return T / (n + 1)


def alpha_weight(T: float, n: int, gamma: float) -> float:
    """alpha = tau / sqrt(gamma) (Eq. matrix_A)."""
    return time_step(T, n) / math.sqrt(gamma)


def theorem_eps(T: float, n: int, delta: float) -> float:
    """c_tau = delta sqrt(tau) / (delta sqrt(tau) + 2 sqrt(T)) (Lemma 2.12)."""
    tau = time_step(T, n)
    return delta * math.sqrt(tau) / (delta * math.sqrt(tau) + 2.0 * math.sqrt(T))


def theorem_rate(delta: float) -> float:
    """rho(delta) = sqrt(-delta^2 + 8 delta + 2) / (2 + delta) (Lemma 2.12)."""
    return math.sqrt(-delta * delta + 8.0 * delta + 2.0) / (2.0 + delta)


# ----------------------------------------------------------------------------
# spatial operator K = -L_h (finite differences, M = I)           (Section 1)
# ----------------------------------------------------------------------------


def unit_coefficient(m1: int, d: int) -> np.ndarray:
    return np.ones((m1 + 2,) * d)


def face_coefficients(a_nodes: np.ndarray):
    """Coefficient on the face between neighbouring nodes P, Q: the arithmetic
    mean (a_P + a_Q)/2 (the paper does not state the face rule; this is the
    reading used throughout).  Returns, per array axis, an array with m1+1
    entries along that axis (faces between node i and i+1, i = 0..m1) and the
    m1 interior entries along the other axes."""
    d = a_nodes.ndim
    faces = []
    for ax in range(d):
        lo = [slice(1, -1)] * d
        hi = [slice(1, -1)] * d
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        faces.append(0.5 * (a_nodes[tuple(lo)] + a_nodes[tuple(hi)]))
    return faces


def apply_K(u: np.ndarray, a_nodes: np.ndarray) -> np.ndarray:
    """(K u)_P = h^-2 sum_{faces f=(P,Q)} a_f (u_P - u_Q), u = 0 on the boundary:
    the conservative finite-difference form of -div(a grad u) with homogeneous
    Dirichlet conditions (Eq. heat, Section 1: K = -L_h, M = I).
    ``u`` may carry leading batch axes; the last d axes are space."""
    d = a_nodes.ndim
    m1 = a_nodes.shape[0] - 2
    h = mesh_width(m1)
    nb = u.ndim - d
    out = np.zeros(u.shape, dtype=np.result_type(u.dtype, np.float64))
    for ax, af in enumerate(face_coefficients(a_nodes)):
        axis = nb + ax
        pad = [(0, 0)] * u.ndim
        pad[axis] = (1, 1)
        up = np.pad(u, pad)                       # zero Dirichlet values
        flux = af * np.diff(up, axis=axis)        # a_{i+1/2} (u_{i+1} - u_i)
        out -= np.diff(flux, axis=axis)           # -(F_{i+1/2} - F_{i-1/2})
    return out / (h * h)


def K_diagonal(a_nodes: np.ndarray) -> np.ndarray:
    """Diagonal of K: h^-2 times the sum of the face coefficients around P."""
    d = a_nodes.ndim
    m1 = a_nodes.shape[0] - 2
    h = mesh_width(m1)
    diag = np.zeros((m1,) * d)
    for ax, af in enumerate(face_coefficients(a_nodes)):
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        diag += af[tuple(lo)] + af[tuple(hi)]
    return diag / (h * h)


def K_sparse(a_nodes: np.ndarray) -> sp.csr_matrix:
    """K assembled entry by entry from the stencil definition: diagonal
    h^-2 sum_f a_f, off-diagonal -h^-2 a_f for each interior neighbour Q."""
    d = a_nodes.ndim
    m1 = a_nodes.shape[0] - 2
    h = mesh_width(m1)
    ms = m1 ** d
    idx = np.arange(ms).reshape((m1,) * d)
    rows, cols, vals = [], [], []
    diag = np.zeros((m1,) * d)
    for ax in range(d):
        for shift in (-1, +1):
            # interior node P at index p (0-based) is node p+1; neighbour node p+1+shift
            nodesP = [slice(1, -1)] * d
            nodesQ = [slice(1, -1)] * d
            nodesQ[ax] = slice(1 + shift, m1 + 1 + shift)
            af = 0.5 * (a_nodes[tuple(nodesP)] + a_nodes[tuple(nodesQ)])
            diag += af
            # neighbour inside the domain?
            src = [slice(None)] * d
            dst = [slice(None)] * d
            if shift == -1:
                src[ax] = slice(1, None)
                dst[ax] = slice(0, -1)
            else:
                src[ax] = slice(0, -1)
                dst[ax] = slice(1, None)
            rows.append(idx[tuple(src)].ravel())
            cols.append(idx[tuple(dst)].ravel())
            vals.append(-af[tuple(src)].ravel())
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ms, ms))
    return K / (h * h)


# ----------------------------------------------------------------------------
# time coupling and the all-at-once matrices        (Eqs. Toeplitz_Mat_B, matrix_T, matrix_A)
# ----------------------------------------------------------------------------


def B_matrix(n: int) -> np.ndarray:
    """B_n: 1 on the diagonal, -1 on the sub-diagonal (Eq. Toeplitz_Mat_B)."""
    return np.eye(n) - np.eye(n, k=-1)


def apply_T(v: np.ndarray, a_nodes: np.ndarray, tau: float) -> np.ndarray:
    """T v = (B_n (x) M + tau I_n (x) K) v:  (T v)_j = v_j - v_{j-1} + tau K v_j,
    v_0 = 0 (Eq. matrix_T)."""
    out = v + tau * apply_K(v, a_nodes)
    out[1:] -= v[:-1]
    return out


def apply_TT(v: np.ndarray, a_nodes: np.ndarray, tau: float) -> np.ndarray:
    """T^T v:  (T^T v)_j = v_j - v_{j+1} + tau K v_j, v_{n+1} = 0."""
    out = v + tau * apply_K(v, a_nodes)
    out[:-1] -= v[1:]
    return out


def apply_A(x: np.ndarray, a_nodes: np.ndarray, tau: float, alpha: float) -> np.ndarray:
    """A x with A = [[alpha I, T^T], [-T, alpha I]] (Eq. matrix_A)."""
    x1, x2 = x[0], x[1]
    y = np.empty(x.shape, dtype=np.result_type(x.dtype, np.float64))
    y[0] = alpha * x1 + apply_TT(x2, a_nodes, tau)
    y[1] = -apply_T(x1, a_nodes, tau) + alpha * x2
    return y


def apply_AT(x: np.ndarray, a_nodes: np.ndarray, tau: float, alpha: float) -> np.ndarray:
    """A^T x, the block transpose of Eq. matrix_A: [[alpha I, -T^T], [T, alpha I]]."""
    x1, x2 = x[0], x[1]
    y = np.empty(x.shape, dtype=np.result_type(x.dtype, np.float64))
    y[0] = alpha * x1 - apply_TT(x2, a_nodes, tau)
    y[1] = apply_T(x1, a_nodes, tau) + alpha * x2
    return y


def T_dense(K: np.ndarray, n: int, tau: float) -> np.ndarray:
    ms = K.shape[0]
    return np.kron(B_matrix(n), np.eye(ms)) + tau * np.kron(np.eye(n), K)


def A_dense(K: np.ndarray, n: int, tau: float, alpha: float) -> np.ndarray:
    """Dense A from the Kronecker form of Eq. matrix_A (tiny sizes only)."""
    ms = K.shape[0]
    T = T_dense(K, n, tau)
    I = np.eye(n * ms)
    return np.block([[alpha * I, T.T], [-T, alpha * I]])


def A_tilde_dense(K: np.ndarray, n: int, tau: float, gamma: float) -> np.ndarray:
    """The unscaled saddle-point matrix of Eq. matrix_A_before (tiny sizes only)."""
    ms = K.shape[0]
    T = T_dense(K, n, tau)
    I = np.eye(n * ms)
    return np.block([[tau * I, T.T], [T, -(tau / gamma) * I]])


# ----------------------------------------------------------------------------
# right-hand side and unscaling                      (Eqs. main_system_before, main_system)
# ----------------------------------------------------------------------------


def build_rhs(f: np.ndarray, g: np.ndarray, y0: np.ndarray, tau: float, gamma: float,
              p_final: np.ndarray | None = None) -> np.ndarray:
    """b = [g_vec; -sqrt(gamma) f_vec] with g_vec_j = tau g^(j) (+ p^(N) at j = n) and
    f_vec_1 = tau f^(1) + y^(0), f_vec_j = tau f^(j) (M = I)."""
    gv = tau * g
    if p_final is not None:
        gv = gv.copy()
        gv[-1] += p_final
    fv = tau * f
    fv = fv.copy()
    fv[0] += y0
    return np.stack([gv, -math.sqrt(gamma) * fv])


def unscale(x: np.ndarray, gamma: float):
    """x = [sqrt(gamma) y; p]  ->  (y, p) (Eq. main_system)."""
    return x[0] / math.sqrt(gamma), x[1]


# ----------------------------------------------------------------------------
# end-point solves and the error measure (Section 1, Section 3)
# ----------------------------------------------------------------------------


def end_point_solves(y: np.ndarray, p: np.ndarray, a_nodes: np.ndarray, tau: float,
                     gamma: float, f_T: np.ndarray, g_0: np.ndarray, y0: np.ndarray,
                     p_final: np.ndarray | None = None):
    """(M + tau K) y^(N) = M y^(N-1) + tau M f^(N) + (tau/gamma) M p^(N);
    (M + tau K) p^(0) = M p^(1) + tau M g^(0) - tau M y^(0)   (Section 1, M = I)."""
    shape = y.shape[1:]
    ms = int(np.prod(shape))
    K = K_sparse(a_nodes)
    E = (sp.identity(ms) + tau * K).tocsc()
    pN = np.zeros(shape) if p_final is None else p_final
    rhs_y = y[-1] + tau * f_T + (tau / gamma) * pN
    rhs_p = p[0] + tau * g_0 - tau * y0
    yN = spla.spsolve(E, rhs_y.ravel()).reshape(shape)
    p0 = spla.spsolve(E, rhs_p.ravel()).reshape(shape)
    return yN, p0


def error_measure(y_levels, p_levels, y_exact, p_exact, h: float, d: int) -> float:
    """e_h = h^{d/2} max_{1<=j<=N} max(||y^(j) - y(t_j)||_2, ||p^(j-1) - p(t_{j-1})||_2)
    (Section 3).  ``y_levels`` holds j = 1..N, ``p_levels`` holds j-1 = 0..N-1."""
    worst = 0.0
    for j in range(len(y_levels)):
        ey = np.linalg.norm((y_levels[j] - y_exact[j]).ravel())
        ep = np.linalg.norm((p_levels[j] - p_exact[j]).ravel())
        worst = max(worst, ey, ep)
    return h ** (d / 2.0) * worst
