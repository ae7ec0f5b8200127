"""Oracle: the discrete objective and its gradient with respect to the nodal
log-coefficient log a and the target g.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading (the paper states the continuous cost, Eq. Cost_functional_heat, and
not its discrete form): with u = p/gamma (Section 1) the discrete objective is

    J_h = h^d tau [ 1/2 sum_{j=1..n} ||y_j - g_j||^2 + 1/(2 gamma) sum_{j=1..n} ||p_j||^2 ],

whose first-order conditions under the backward-Euler constraint are exactly
the saddle-point system of Eq. matrix_A_before (the multiplier of time block j
is p_j).  Two independent routes to dJ*/dtheta at the optimum x*(theta):

* envelope (Lagrangian) form: dJ*/d log a_P = h^d tau sum_j p_j^T (dK/d log a_P) y_j,
  dJ*/dg_j = -h^d tau (y_j - g_j);
* adjoint form: A^T lam = dJ/dx, dJ/dtheta = dJ/dtheta|_x + lam^T (db/dtheta - dA/dtheta x).

With a_f = (a_P + a_Q)/2,  u^T (dK/d log a_P) v = a_P/(2 h^2) sum_{faces f of P} (u_P - u_Q)(v_P - v_Q),
with boundary values 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import system


def objective(x: np.ndarray, g: np.ndarray, tau: float, gamma: float) -> float:
    d = g.ndim - 1
    m1 = g.shape[1]
    h = system.mesh_width(m1)
    y, p = system.unscale(x, gamma)
    return h ** d * tau * (0.5 * np.sum((y - g) ** 2) + 0.5 / gamma * np.sum(p ** 2))


def objective_grad_x(x: np.ndarray, g: np.ndarray, tau: float, gamma: float) -> np.ndarray:
    """Partial derivative of J_h with respect to x = [sqrt(gamma) y; p] at fixed g."""
    d = g.ndim - 1
    h = system.mesh_width(g.shape[1])
    y, p = system.unscale(x, gamma)
    return np.stack([h ** d * tau * (y - g) / math.sqrt(gamma), h ** d * tau * p / gamma])


def stencil_derivative(u: np.ndarray, v: np.ndarray, a_nodes: np.ndarray) -> np.ndarray:
    """S_P = sum over the leading (time) axis of a_P/(2 h^2) sum_{faces f=(P,Q)} (u_P-u_Q)(v_P-v_Q),
    u = v = 0 on boundary nodes; one value per interior node P."""
    d = a_nodes.ndim
    m1 = a_nodes.shape[0] - 2
    h = system.mesh_width(m1)
    pad = [(0, 0)] + [(1, 1)] * d
    up = np.pad(u, pad)
    vp = np.pad(v, pad)
    acc = np.zeros((m1,) * d)
    centre = (slice(None),) + (slice(1, -1),) * d
    for ax in range(d):
        for shift in (-1, 1):
            nb = [slice(None)] + [slice(1, -1)] * d
            nb[1 + ax] = slice(1 + shift, m1 + 1 + shift)
            du = up[centre] - up[tuple(nb)]
            dv = vp[centre] - vp[tuple(nb)]
            acc += np.sum(du * dv, axis=0)
    a_int = a_nodes[(slice(1, -1),) * d]
    return 0.5 * a_int * acc / (h * h)


def envelope_gradient(x: np.ndarray, g: np.ndarray, a_nodes: np.ndarray, tau: float,
                      gamma: float):
    d = a_nodes.ndim
    h = system.mesh_width(a_nodes.shape[0] - 2)
    y, p = system.unscale(x, gamma)
    g_loga = h ** d * tau * stencil_derivative(p, y, a_nodes)
    g_g = -h ** d * tau * (y - g)
    return g_loga, g_g


def adjoint_gradient(x: np.ndarray, lam: np.ndarray, g: np.ndarray, a_nodes: np.ndarray,
                     tau: float, gamma: float):
    """dJ/dtheta = dJ/dtheta|_x + lam^T (db/dtheta - dA/dtheta x), A^T lam = dJ/dx.
    dA/dtheta = tau [[0, I (x) K'], [-I (x) K', 0]] and db_1/dg_j = tau I."""
    d = a_nodes.ndim
    h = system.mesh_width(a_nodes.shape[0] - 2)
    y, _ = system.unscale(x, gamma)
    lam_dA_x = tau * (stencil_derivative(lam[0], x[1], a_nodes)
                      - stencil_derivative(lam[1], x[0], a_nodes))
    g_loga = -lam_dA_x
    g_g = -h ** d * tau * (y - g) + tau * lam[0]
    return g_loga, g_g
