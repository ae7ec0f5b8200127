"""Oracle: GMRES without restarts, left- or right-preconditioned (flexible).

TEST INFRASTRUCTURE ONLY (see the package docstring).

GMRES (Saad & Schultz, cited in Section 1) builds an orthonormal basis of the
Krylov space with Arnoldi (modified Gram-Schmidt here), reduces the Hessenberg
least-squares problem with Givens rotations, and returns the iterate that
minimises the residual over x0 + K_j (Lemma 2.1).  Section 3 runs it from a
zero initial guess with a relative tolerance of 1e-8.

* ``mode='left'``  solves P^{-1} A x = P^{-1} b and stops on
  ||P^{-1}(b - A x_j)|| <= rtol ||P^{-1} b|| (the preconditioned residual the
  theorems bound).
* ``mode='right'`` is flexible GMRES: z_j = P^{-1} v_j is stored, A z_j is
  orthogonalised, x_j = x0 + Z_j y_j, and it stops on ||b - A x_j|| <= rtol ||b||.
"""
from __future__ import annotations

import numpy as np


class GMRESResult:
    def __init__(self, x, iters, resid_history, converged):
        self.x = x
        self.iters = iters
        self.resid_history = resid_history      # relative residual estimates, index 0 = start
        self.converged = converged


def _givens(a: float, b: float):
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def gmres(apply_A, apply_Pinv, b: np.ndarray, rtol: float = 1e-8, maxit: int = 200,
          mode: str = "right", x0: np.ndarray | None = None) -> GMRESResult:
    shape = b.shape
    bf = b.ravel().astype(np.float64)
    A = lambda v: apply_A(v.reshape(shape)).ravel()
    Pi = lambda v: apply_Pinv(v.reshape(shape)).ravel()
    x = np.zeros_like(bf) if x0 is None else x0.ravel().astype(np.float64).copy()

    if mode == "left":
        r0 = Pi(bf - A(x))
        ref = np.linalg.norm(Pi(bf))
    elif mode == "right":
        r0 = bf - A(x)
        ref = np.linalg.norm(bf)
    else:
        raise ValueError(mode)
    if ref == 0.0:
        return GMRESResult(np.zeros(shape), 0, [0.0], True)
    beta = np.linalg.norm(r0)
    hist = [beta / ref]
    if beta / ref <= rtol:
        return GMRESResult(x.reshape(shape), 0, hist, True)

    V = [r0 / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    gvec = np.zeros(maxit + 1)
    gvec[0] = beta
    k = 0
    converged = False
    for j in range(maxit):
        if mode == "left":
            w = Pi(A(V[j]))
        else:
            z = Pi(V[j])
            Z.append(z)
            w = A(z)
        for i in range(j + 1):                  # modified Gram-Schmidt
            H[i, j] = np.dot(w, V[i])
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0:
            V.append(w / H[j + 1, j])
        else:
            V.append(np.zeros_like(w))
        for i in range(j):                      # previous rotations on the new column
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
        H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
        H[j + 1, j] = 0.0
        gvec[j + 1] = -sn[j] * gvec[j]
        gvec[j] = cs[j] * gvec[j]
        k = j + 1
        hist.append(abs(gvec[j + 1]) / ref)
        if hist[-1] <= rtol:
            converged = True
            break
    y = np.linalg.solve(np.triu(H[:k, :k]), gvec[:k]) if k else np.zeros(0)
    basis = V if mode == "left" else Z
    for i in range(k):
        x = x + y[i] * basis[i]
    return GMRESResult(x.reshape(shape), k, hist, converged)


def krylov_minimiser(apply_op, rhs: np.ndarray, x0: np.ndarray, j: int) -> np.ndarray:
    """Brute force of Lemma 2.1: argmin over c in x0 + K_j(op, r0) of ||rhs - op c||,
    with the Krylov space spanned by the explicit powers r0, op r0, ..., op^{j-1} r0
    (orthonormalised by QR only for conditioning) and a dense least-squares solve."""
    r0 = rhs - apply_op(x0)
    cols = [r0]
    for _ in range(1, j):
        cols.append(apply_op(cols[-1]))
    Kmat = np.stack(cols, axis=1)
    Q, _ = np.linalg.qr(Kmat)
    OQ = np.stack([apply_op(Q[:, i]) for i in range(Q.shape[1])], axis=1)
    coef, *_ = np.linalg.lstsq(OQ, r0, rcond=None)
    return x0 + Q @ coef
