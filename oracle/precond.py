"""Oracle: the eps-circulant RBD preconditioner and its spatial solvers.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper taken here (each is pinned by a test against a dense
definition, not against this module itself):

* D_eps = diag(eps^{(i-1)/n}) with exponent denominator n, the size of C_{eps,n}
  (Eq. decomposition_eps; Section 2.1 prints N there).
* The transposed (upper) block.  Because C_{eps,n} is real,
  C^T = conj(C^T) = D F conj(Lambda) F^* D^{-1}, so
  (C_eps^T + alpha I (x) M)^{-1} v1 = (D F (x) I) [(conj(Lambda)+alpha I) (x) M + tau I (x) K]^{-1} (F^* D^{-1} (x) I) v1.
  The spectral form printed in Section 2.1 pairs (F^* D)^T with Lambda^*, which is
  not consistent; the form above is the one the dense P_eps of Eq. matrix_P_eps
  agrees with.
* Multigrid (Example 2 only says: one V-cycle, Gauss-Seidel pre-smoother, no
  post-smoother): V(1,0) with one red-black Gauss-Seidel sweep (red = even sum
  of 1-based indices, swept first) from a zero initial guess on every level,
  full-weighting restriction, (bi/tri)linear prolongation, coarse operators by
  rediscretisation with the nodal coefficient injected (a_c[I] = a[2I]), the
  same complex shift on every level, exact solve on the one-point level.
"""
from __future__ import annotations

import math

import numpy as np

from . import system

# ----------------------------------------------------------------------------
# eps-circulant time matrix and its diagonalisation (Eqs. matrix_C_eps_n, decomposition_eps)
# ----------------------------------------------------------------------------


def C_eps_matrix(n: int, eps: float) -> np.ndarray:
    """C_{eps,n}: B_n with -eps in the top-right corner (Eq. matrix_C_eps_n)."""
    C = system.B_matrix(n)
    C[0, n - 1] -= eps
    return C


def D_eps_diag(n: int, eps: float) -> np.ndarray:
    """Diagonal of D_eps: eps^{(i-1)/n}, i = 1..n (Eq. decomposition_eps)."""
    return eps ** (np.arange(n) / n)


def fourier_matrix(n: int) -> np.ndarray:
    """F_n = n^{-1/2} [theta^{(i-1)(j-1)}], theta = exp(2 pi i / n) (Eq. decomposition_eps)."""
    jk = np.outer(np.arange(n), np.arange(n))
    return np.exp(2j * math.pi * jk / n) / math.sqrt(n)


def eigenvalues_lambda(n: int, eps: float) -> np.ndarray:
    """lambda_k = 1 - eps^{1/n} theta^{-k}, k = 0..n-1 (Eq. decomposition_eps)."""
    k = np.arange(n)
    return 1.0 - eps ** (1.0 / n) * np.exp(-2j * math.pi * k / n)


# ----------------------------------------------------------------------------
# dense preconditioners (tiny sizes only)                  (Eqs. matrix_P, matrix_P_eps)
# ----------------------------------------------------------------------------


def _rotation(nm: int) -> np.ndarray:
    I = np.eye(nm)
    return np.block([[I, I], [-I, I]])


def P_eps_dense(K: np.ndarray, n: int, tau: float, alpha: float, eps: float) -> np.ndarray:
    """P_eps = 1/2 blockdiag(C_eps^T + alpha I(x)M, C_eps + alpha I(x)M) [[I, I], [-I, I]]
    with C_eps = C_{eps,n} (x) M + tau I_n (x) K, M = I (Eq. matrix_P_eps)."""
    ms = K.shape[0]
    Ce = np.kron(C_eps_matrix(n, eps), np.eye(ms)) + tau * np.kron(np.eye(n), K)
    I = np.eye(n * ms)
    Z = np.zeros_like(I)
    H = np.block([[Ce.T + alpha * I, Z], [Z, Ce + alpha * I]])
    return 0.5 * H @ _rotation(n * ms)


def P_dense(K: np.ndarray, n: int, tau: float, alpha: float) -> np.ndarray:
    """The ideal RBD preconditioner P of Eq. matrix_P (C_eps replaced by T)."""
    ms = K.shape[0]
    T = system.T_dense(K, n, tau)
    I = np.eye(n * ms)
    Z = np.zeros_like(I)
    H = np.block([[T.T + alpha * I, Z], [Z, T + alpha * I]])
    return 0.5 * H @ _rotation(n * ms)


# ----------------------------------------------------------------------------
# spatial solvers for ((sigma_k) I + tau K) z_k = r_k, one complex shift per k
# ----------------------------------------------------------------------------


class DenseSpatialSolver:
    """Exact solves with the dense matrix sigma I + tau K (tiny sizes)."""

    def __init__(self, a_nodes: np.ndarray, tau: float):
        self.K = system.K_sparse(a_nodes).toarray()
        self.tau = tau
        self.shape = (a_nodes.shape[0] - 2,) * a_nodes.ndim

    def __call__(self, sigma: np.ndarray, R: np.ndarray) -> np.ndarray:
        ms = self.K.shape[0]
        out = np.empty(R.shape, dtype=complex)
        for k in range(R.shape[0]):
            Mk = sigma[k] * np.eye(ms) + self.tau * self.K
            out[k] = np.linalg.solve(Mk, R[k].reshape(ms)).reshape(self.shape)
        return out


def dst1_matrix(m: int) -> np.ndarray:
    """Orthonormal DST-I matrix S_ij = sqrt(2/(m+1)) sin(pi i j/(m+1)), i,j = 1..m."""
    ij = np.outer(np.arange(1, m + 1), np.arange(1, m + 1))
    return math.sqrt(2.0 / (m + 1)) * np.sin(math.pi * ij / (m + 1))


class FSTSpatialSolver:
    """Exact solves for constant a = c by the discrete sine transform in every
    dimension (Example 1): the 1D Dirichlet second difference has eigenvectors
    the DST-I columns and eigenvalues mu_i = 4 sin^2(pi i/(2(m+1)))/h^2."""

    def __init__(self, m1: int, d: int, tau: float, coeff: float = 1.0):
        self.m1, self.d, self.tau, self.c = m1, d, tau, coeff
        self.S = dst1_matrix(m1)
        h = system.mesh_width(m1)
        mu = 4.0 * np.sin(math.pi * np.arange(1, m1 + 1) / (2 * (m1 + 1))) ** 2 / (h * h)
        lam = np.zeros((m1,) * d)
        for ax in range(d):
            shp = [1] * d
            shp[ax] = m1
            lam = lam + mu.reshape(shp)
        self.lamK = coeff * lam

    def _transform(self, R: np.ndarray) -> np.ndarray:
        out = R
        for ax in range(self.d):
            out = np.moveaxis(np.tensordot(self.S, out, axes=([1], [1 + ax])), 0, 1 + ax)
        return out

    def __call__(self, sigma: np.ndarray, R: np.ndarray) -> np.ndarray:
        Rh = self._transform(R)
        den = sigma.reshape((-1,) + (1,) * self.d) + self.tau * self.lamK[None]
        return self._transform(Rh / den)


class MGLevel:
    def __init__(self, a_nodes: np.ndarray):
        self.a = a_nodes
        self.d = a_nodes.ndim
        self.m = a_nodes.shape[0] - 2
        self.diagK = system.K_diagonal(a_nodes)
        idx = np.indices((self.m,) * self.d).sum(axis=0) + self.d   # sum of 1-based indices
        self.red = (idx % 2) == 0
        self.black = ~self.red


def restrict_full_weighting(r: np.ndarray, d: int) -> np.ndarray:
    """Full weighting: coarse point I sits on fine point 2I (1-based); the weight
    of the fine point 2I + o (o in {-1,0,1}^d) is prod_k w(o_k), w(0) = 1/2,
    w(+-1) = 1/4.  Leading axis of ``r`` is a batch axis."""
    mf = r.shape[1]
    mc = (mf - 1) // 2
    w = {-1: 0.25, 0: 0.5, 1: 0.25}
    out = np.zeros((r.shape[0],) + (mc,) * d, dtype=r.dtype)
    for off in np.ndindex(*([3] * d)):
        o = [v - 1 for v in off]
        wt = 1.0
        sl = [slice(None)]
        for k in range(d):
            wt *= w[o[k]]
            start = 1 + o[k]                 # 0-based fine index of 2I+o for I = 1
            sl.append(slice(start, start + 2 * mc - 1, 2))
        out += wt * r[tuple(sl)]
    return out


def prolong_linear(e: np.ndarray, d: int) -> np.ndarray:
    """(Bi/tri)linear interpolation, one dimension at a time: fine point 2I takes
    e_c(I); fine point 2I+1 takes (e_c(I) + e_c(I+1))/2 with zero boundary values."""
    out = e
    for k in range(d):
        axis = 1 + k
        mc = out.shape[axis]
        shp = list(out.shape)
        shp[axis] = 2 * mc + 1
        fine = np.zeros(shp, dtype=out.dtype)
        pad = [(0, 0)] * out.ndim
        pad[axis] = (1, 1)
        op = np.pad(out, pad)
        sl_odd = [slice(None)] * out.ndim
        sl_odd[axis] = slice(1, 2 * mc, 2)          # 0-based fine 2c+1  <->  coarse c
        fine[tuple(sl_odd)] = out
        sl_even = [slice(None)] * out.ndim
        sl_even[axis] = slice(0, 2 * mc + 1, 2)     # 0-based fine 2c  <->  between c-1 and c
        lo = [slice(None)] * out.ndim
        hi = [slice(None)] * out.ndim
        lo[axis] = slice(0, mc + 1)
        hi[axis] = slice(1, mc + 2)
        fine[tuple(sl_even)] = 0.5 * (op[tuple(lo)] + op[tuple(hi)])
        out = fine
    return out


class MGSpatialSolver:
    """One V(1,0) cycle per shifted system (Example 2, Section 2.1): the
    preconditioner is *defined* by this cycle, not by an exact solve.

    smoother: "red-black" (one red-black Gauss-Seidel sweep from zero, red first) or
    "lexicographic" (one sweep in the natural order, x1 fastest: every point takes its
    lower neighbours' new values and zero for the others)."""

    def __init__(self, a_nodes: np.ndarray, tau: float, smoother: str = "red-black"):
        m = a_nodes.shape[0] - 2
        if m < 1 or (m + 1) & m:
            raise ValueError("multigrid needs m1 = 2^k - 1")
        if smoother not in ("red-black", "lexicographic"):
            raise ValueError("smoother must be 'red-black' or 'lexicographic'")
        self.smoother = smoother
        self.tau = tau
        self.d = a_nodes.ndim
        self.levels = []
        a = a_nodes
        while True:
            self.levels.append(MGLevel(a))
            if a.shape[0] - 2 == 1:
                break
            a = a[(slice(None, None, 2),) * self.d]      # injection of the nodal coefficient

    def _op(self, lev: MGLevel, sigma: np.ndarray, u: np.ndarray) -> np.ndarray:
        s = sigma.reshape((-1,) + (1,) * self.d)
        return s * u + self.tau * system.apply_K(u, lev.a)

    def vcycle(self, l: int, sigma: np.ndarray, r: np.ndarray) -> np.ndarray:
        lev = self.levels[l]
        s = sigma.reshape((-1,) + (1,) * self.d)
        dg = s + self.tau * lev.diagK[None]
        if lev.m == 1:
            return r / dg
        if self.smoother == "lexicographic":
            u = self._lex_sweep(lev, dg, r)
        else:
            u = np.zeros_like(r)
            # red-black Gauss-Seidel sweep from zero: red first (its neighbours are 0) ...
            u[:, lev.red] = r[:, lev.red] / dg[:, lev.red]
            # ... then black, using the updated red values
            off = self._op(lev, sigma, u) - dg * u
            u[:, lev.black] = (r[:, lev.black] - off[:, lev.black]) / dg[:, lev.black]
        res = r - self._op(lev, sigma, u)
        rc = restrict_full_weighting(res, self.d)
        ec = self.vcycle(l + 1, sigma, rc)
        return u + prolong_linear(ec, self.d)

    def _lex_sweep(self, lev: MGLevel, dg: np.ndarray, r: np.ndarray) -> np.ndarray:
        """Gauss-Seidel sweep from zero in the natural order: u_P = (r_P + sum over the
        lower neighbours Q of w_PQ u_Q) / (sigma + d_P), w_PQ = tau (a_P + a_Q) / (2 h^2).
        Points with equal index sum do not depend on each other, so the sweep runs one
        such diagonal at a time (the result is that of the point-by-point loop)."""
        d, m, a = self.d, lev.m, lev.a
        h = system.mesh_width(m)
        inner = (slice(1, -1),) * d
        aP = a[inner]
        wlow = []  # weight towards the lower neighbour along each array axis
        for ax in range(d):
            sl = [slice(1, -1)] * d
            sl[ax] = slice(0, -2)
            wlow.append(self.tau * 0.5 * (aP + a[tuple(sl)]) / (h * h))
        u = np.zeros_like(r)
        tsum = np.indices((m,) * d).sum(axis=0)
        for t in range(d * (m - 1) + 1):
            pts = np.nonzero(tsum == t)
            acc = r[(slice(None),) + pts].copy()
            for ax in range(d):
                has = pts[ax] > 0
                if not has.any():
                    continue
                sel = tuple(p[has] for p in pts)
                nb = list(sel)
                nb[ax] = nb[ax] - 1
                acc[:, has] += wlow[ax][sel] * u[(slice(None),) + tuple(nb)]
            u[(slice(None),) + pts] = acc / dg[(slice(None),) + pts]
        return u

    def __call__(self, sigma: np.ndarray, R: np.ndarray) -> np.ndarray:
        return self.vcycle(0, sigma, R.astype(complex))


# ----------------------------------------------------------------------------
# the four-step apply of P_eps^{-1}                                   (Section 2.1)
# ----------------------------------------------------------------------------


def apply_Peps_inv(v: np.ndarray, n: int, alpha: float, eps: float, spatial) -> np.ndarray:
    """w = P_eps^{-1} v in four steps (Section 2.1):
    1. hat v = U^{-1} v:   hat v_1 = fft_t(D^{-1} v_1),  hat v_2 = fft_t(D v_2);
    2. solve per frequency k: ((conj lambda_k + alpha) I + tau K) for half 1 and
       ((lambda_k + alpha) I + tau K) for half 2;
    3. tilde w = U tilde v:  tilde w_1 = D ifft_t(.),  tilde w_2 = D^{-1} ifft_t(.);
    4. w = [[I, -I], [I, I]] tilde w.
    fft_t is the unnormalised DFT along time with kernel exp(-2 pi i jk/n)."""
    dpow = D_eps_diag(n, eps)
    bshape = (n,) + (1,) * (v.ndim - 2)
    dp = dpow.reshape(bshape)
    lam = eigenvalues_lambda(n, eps)
    v1h = np.fft.fft(v[0] / dp, axis=0)
    v2h = np.fft.fft(v[1] * dp, axis=0)
    w1h = spatial(np.conj(lam) + alpha, v1h)
    w2h = spatial(lam + alpha, v2h)
    wt1 = np.real(np.fft.ifft(w1h, axis=0)) * dp
    wt2 = np.real(np.fft.ifft(w2h, axis=0)) / dp
    return np.stack([wt1 - wt2, wt1 + wt2])


# ----------------------------------------------------------------------------
# the ideal RBD preconditioner P by block substitution in time     (Eq. matrix_P)
# ----------------------------------------------------------------------------


def apply_P_inv(v: np.ndarray, n: int, alpha: float, spatial) -> np.ndarray:
    """w = P^{-1} v for the rotated block-diagonal preconditioner of Eq. matrix_P,
    P = 1/2 blockdiag(T^T + alpha I, T + alpha I) [[I, I], [-I, I]] (M = I).
    Its inverse is [[I, -I], [I, I]] blockdiag((T^T + alpha I)^{-1}, (T + alpha I)^{-1}):
    * (T + alpha I) w2 = v2, T block lower bidiagonal (Eq. matrix_T): forward in time,
      ((1 + alpha) I + tau K) w2_j = v2_j + w2_{j-1}, w2_0 = 0;
    * (T^T + alpha I) w1 = v1: backward in time,
      ((1 + alpha) I + tau K) w1_j = v1_j + w1_{j+1}, w1_{n+1} = 0;
    then w = [w1 - w2; w1 + w2].  Each step is one spatial solve with the real shift
    1 + alpha by `spatial` (exact for the dense and sine-transform solvers, one
    V(1,0) cycle for multigrid): n sequential solves per half, the cost the
    eps-circulant P_eps removes."""
    shift = np.array([1.0 + alpha])
    w1 = np.zeros(v[0].shape)
    w2 = np.zeros(v[1].shape)
    prev = np.zeros(v[1].shape[1:])
    for j in range(n):
        w2[j] = np.real(spatial(shift, (v[1][j] + prev)[None]))[0]
        prev = w2[j]
    nxt = np.zeros(v[0].shape[1:])
    for j in reversed(range(n)):
        w1[j] = np.real(spatial(shift, (v[0][j] + nxt)[None]))[0]
        nxt = w1[j]
    return np.stack([w1 - w2, w1 + w2])


def make_spatial_solver(kind: str, a_nodes, m1: int, d: int, tau: float, smoother: str = "red-black"):
    """'dense' | 'fst' (a constant; a_nodes None means a = 1) | 'mg' (with the given smoother)."""
    if a_nodes is None:
        a_nodes = system.unit_coefficient(m1, d)
    if kind == "dense":
        return DenseSpatialSolver(a_nodes, tau)
    if kind == "fst":
        c = float(a_nodes.flat[0])
        if not np.allclose(a_nodes, c, rtol=0, atol=0):
            raise ValueError("FST needs a constant coefficient")
        return FSTSpatialSolver(m1, d, tau, c)
    if kind == "mg":
        return MGSpatialSolver(a_nodes, tau, smoother)
    raise ValueError(kind)
