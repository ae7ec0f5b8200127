"""Seeded input fields for the parabolic optimal-control workloads.

Conventions shared by every consumer:

* the domain is the unit square/cube; ``m1`` interior points per dimension,
  mesh width ``h = 1/(m1+1)``; node ``(i_d, ..., i_2, i_1)`` sits at
  ``x_k = i_k h`` (``i_k = 0..m1+1``, 0 and m1+1 are boundary nodes);
* a spatial field on the interior is a C-ordered array of shape ``(m1,)*d``
  whose LAST axis is ``x1`` (so the flattened index is
  ``s = i1 + m1*i2 (+ m1^2*i3)`` with 0-based interior indices);
* a nodal coefficient field ``a`` has shape ``(m1+2,)*d`` and includes the
  boundary nodes;
* time levels of the all-at-once system are ``t_j = j*tau`` for ``j = 1..n``
  with ``tau = T/(n+1)`` (``n`` time blocks, ``N = n+1`` backward-Euler steps),
  so a space-time field has shape ``(n,) + (m1,)*d``.

Nothing here performs any step of the solver; these are only inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "Problem", "node_grid", "interior_grid", "time_levels",
    "plain_fp64_problem", "variable_2d_problem", "gaussian_field_3d_problem",
    "batched_problems", "gradient_problem",
    "example1_problem", "example1_exact", "example2_problem", "example2_exact",
    "smooth_modes_target", "random_vector",
]


@dataclass
class Problem:
    """One instance of the discrete optimal-control problem (inputs only)."""
    d: int
    m1: int
    n: int
    T: float
    gamma: float
    eps: float
    a_nodes: Optional[np.ndarray]      # (m1+2,)*d, None means a == 1
    f: np.ndarray                      # (n,)+(m1,)*d   source at t_1..t_n
    g: np.ndarray                      # (n,)+(m1,)*d   target at t_1..t_n
    y0: np.ndarray                     # (m1,)*d        initial state
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def tau(self) -> float:
        return self.T / (self.n + 1)

    @property
    def h(self) -> float:
        return 1.0 / (self.m1 + 1)

    @property
    def ms(self) -> int:
        return self.m1 ** self.d

    @property
    def unknowns(self) -> int:
        return 2 * self.ms * self.n


def node_grid(m1: int, d: int):
    """Coordinates of all nodes incl. boundary; returns (x1, x2[, x3]) arrays."""
    t = np.arange(m1 + 2) / (m1 + 1)
    axes = np.meshgrid(*([t] * d), indexing="ij")   # axes[0] varies along axis 0
    # last array axis is x1 -> x1 = axes[d-1], x2 = axes[d-2], ...
    return tuple(axes[d - 1 - k] for k in range(d))


def interior_grid(m1: int, d: int):
    t = np.arange(1, m1 + 1) / (m1 + 1)
    axes = np.meshgrid(*([t] * d), indexing="ij")
    return tuple(axes[d - 1 - k] for k in range(d))


def time_levels(T: float, n: int) -> np.ndarray:
    tau = T / (n + 1)
    return tau * np.arange(1, n + 1)


def random_vector(shape, seed: int) -> np.ndarray:
    """Standard-normal FP64 array (used as generic operator inputs in tests)."""
    return np.random.default_rng(seed).standard_normal(shape)


# ----------------------------------------------------------------------------
# configuration generators
# ----------------------------------------------------------------------------

def smooth_modes_target(m1: int, d: int, T: float, n: int, seed: int,
                        modes: int = 16) -> np.ndarray:
    """g(x,t) = sum_q c_q prod_k sin(pi k_q,k x_k) cos(pi k_q,t t), c_q ~ N(0,1),
    spatial wavenumbers in {1..4}, temporal in {0..3}; shape (n,)+(m1,)*d."""
    rng = np.random.default_rng(seed)
    xs = interior_grid(m1, d)
    t = time_levels(T, n)
    g = np.zeros((n,) + (m1,) * d)
    for _ in range(modes):
        c = rng.standard_normal()
        ks = rng.integers(1, 5, size=d)
        kt = rng.integers(0, 4)
        space = np.ones((m1,) * d)
        for k in range(d):
            space = space * np.sin(math.pi * ks[k] * xs[k])
        g += c * np.cos(math.pi * kt * t)[(slice(None),) + (None,) * d] * space[None]
    return g


def plain_fp64_problem(m1: int = 31, n: int = 32, gamma: float = 1e-2,
                       T: float = 1.0) -> Problem:
    """2D, a == 1, f = 0, y0 = 0, g = sin(pi x1) sin(pi x2) * t, eps = 0.5 sqrt(tau)."""
    d = 2
    x1, x2 = interior_grid(m1, d)
    t = time_levels(T, n)
    g = t[:, None, None] * (np.sin(math.pi * x1) * np.sin(math.pi * x2))[None]
    tau = T / (n + 1)
    return Problem(d, m1, n, T, gamma, 0.5 * math.sqrt(tau), None,
                   np.zeros_like(g), g, np.zeros((m1,) * d), name="plain-2d-a1")


def variable_2d_problem(gamma: float = 1e-4, m1: int = 255, n: int = 256,
                        T: float = 1.0, seed: int = 2410) -> Problem:
    """2D, a = 1 + 0.5 sin(2 pi x1) cos(2 pi x2), eps = sqrt(tau), f = 0, y0 = 0,
    g from 16 seeded smooth Fourier modes."""
    d = 2
    X1, X2 = node_grid(m1, d)
    a = 1.0 + 0.5 * np.sin(2 * math.pi * X1) * np.cos(2 * math.pi * X2)
    g = smooth_modes_target(m1, d, T, n, seed)
    tau = T / (n + 1)
    return Problem(d, m1, n, T, gamma, math.sqrt(tau), a, np.zeros_like(g), g,
                   np.zeros((m1,) * d), name=f"variable-2d-m{m1}-n{n}")


def _gaussian_random_field_3d(npts: int, corr_len: float, seed: int) -> np.ndarray:
    """Unit-variance stationary Gaussian field with squared-exponential
    covariance exp(-r^2/(2 l^2)) sampled on an npts^3 node grid of the unit cube.
    Generated spectrally on a doubled periodic box to suppress wrap-around."""
    rng = np.random.default_rng(seed)
    big = 2 * npts
    dx = 1.0 / (npts - 1)
    kx = 2 * math.pi * np.fft.fftfreq(big, d=dx)
    KX, KY, KZ = np.meshgrid(kx, kx, kx, indexing="ij")
    spec = np.exp(-0.25 * corr_len ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2))
    noise = rng.standard_normal((big, big, big))
    fld = np.real(np.fft.ifftn(np.fft.fftn(noise) * spec))
    fld = fld[:npts, :npts, :npts]
    fld = (fld - fld.mean()) / fld.std()
    return fld


def gaussian_field_3d_problem(m1: int = 63, n: int = 128, gamma: float = 1e-4,
                              T: float = 1.0, seed: int = 2411) -> Problem:
    """3D unit cube, a = exp(0.5 G), G a unit-variance Gaussian random field
    (correlation length 0.2), eps = sqrt(tau), 16-mode smooth target."""
    d = 3
    G = _gaussian_random_field_3d(m1 + 2, 0.2, seed)
    a = np.exp(0.5 * G)
    g = smooth_modes_target(m1, d, T, n, seed + 1)
    tau = T / (n + 1)
    return Problem(d, m1, n, T, gamma, math.sqrt(tau), a, np.zeros_like(g), g,
                   np.zeros((m1,) * d), name=f"grf-3d-m{m1}-n{n}")


def _smooth_log2_field(m1: int, rng) -> np.ndarray:
    """a = 2^{s(x)}, s an 8-mode smooth sine/cosine sum normalised to [-1, 1]."""
    X1, X2 = node_grid(m1, 2)
    s = np.zeros_like(X1)
    for _ in range(8):
        c = rng.standard_normal()
        k1, k2 = rng.integers(1, 4, size=2)
        ph1, ph2 = rng.uniform(0, 2 * math.pi, size=2)
        s += c * np.sin(math.pi * k1 * X1 + ph1) * np.cos(math.pi * k2 * X2 + ph2)
    s = s / max(np.abs(s).max(), 1e-300)
    return 2.0 ** s


def batched_problems(count: int = 64, seed: int = 2412,
                     grids=(31, 63, 127, 255), steps=(16, 64, 256, 512),
                     T: float = 1.0):
    """Independent 2D problems of uneven size: m1 and n drawn uniformly from the
    given sets, log10(gamma) ~ U[-8,-2], per-problem smooth a in [0.5, 2]."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        m1 = int(rng.choice(grids))
        n = int(rng.choice(steps))
        gamma = 10.0 ** rng.uniform(-8, -2)
        a = _smooth_log2_field(m1, rng)
        g = smooth_modes_target(m1, 2, T, n, int(rng.integers(0, 2 ** 31)))
        tau = T / (n + 1)
        out.append(Problem(2, m1, n, T, gamma, math.sqrt(tau), a, np.zeros_like(g), g,
                           np.zeros((m1, m1)), name=f"batch{q}-m{m1}-n{n}"))
    return out


def gradient_problem(m1: int = 127, n: int = 128, gamma: float = 1e-4,
                     T: float = 1.0, seed: int = 2410) -> Problem:
    """Differentiation workload: the variable-coefficient 2D generator at m1, n."""
    p = variable_2d_problem(gamma=gamma, m1=m1, n=n, T=T, seed=seed)
    p.name = f"gradient-2d-m{m1}-n{n}"
    return p


# ----------------------------------------------------------------------------
# manufactured-solution examples of the paper (Section 3, Examples 1 and 2)
# ----------------------------------------------------------------------------

def _paper_eps(tau: float) -> float:
    # the experiments of Section 3 use eps = min{1/2, tau/2}
    return min(0.5, 0.5 * tau)


def example1_exact(x1, x2, t):
    """Example 1: y = e^{-t} sin(pi x1) sin(pi x2), p = 0."""
    y = np.exp(-t) * np.sin(math.pi * x1) * np.sin(math.pi * x2)
    return y, np.zeros_like(y)


def example1_problem(m1: int, n: int, gamma: float, T: float = 1.0) -> Problem:
    """Example 1 (Section 3): a = 1, f = (2 pi^2 - 1) e^{-t} SS, g = e^{-t} SS,
    y0 = SS where SS = sin(pi x1) sin(pi x2)."""
    x1, x2 = interior_grid(m1, 2)
    t = time_levels(T, n)[:, None, None]
    ss = (np.sin(math.pi * x1) * np.sin(math.pi * x2))[None]
    f = (2 * math.pi ** 2 - 1) * np.exp(-t) * ss
    g = np.exp(-t) * ss
    tau = T / (n + 1)
    p = Problem(2, m1, n, T, gamma, _paper_eps(tau), None, f, g, ss[0].copy(),
                name=f"example1-m{m1}-n{n}")
    # source/target at t = T and t = 0 (needed by the two end-point solves)
    p.extra["f_T"] = (2 * math.pi ** 2 - 1) * math.exp(-T) * ss[0]
    p.extra["g_0"] = ss[0].copy()
    return p


def _example2_fg(x1, x2, t, gamma):
    s1, s2 = np.sin(math.pi * x1), np.sin(math.pi * x2)
    c1, c2 = np.cos(math.pi * x1), np.cos(math.pi * x2)
    sx, cx = np.sin(math.pi * x1 * x2), np.cos(math.pi * x1 * x2)
    et = np.exp(-t)
    # the bare "x" in the printed source term is read as x1
    f = (-np.sin(math.pi * t) * s1 * s2
         + et * x1 * (1 - x1) * (2e-5 * sx - x2 * (1 - x2) - 1e-5 * math.pi * cx * x1 * (1 - 2 * x2))
         + et * x2 * (1 - x2) * (2e-5 * sx - 1e-5 * math.pi * cx * x2 * (1 - 2 * x1)))
    g = (-gamma * math.pi * np.cos(math.pi * t) * s1 * s2
         + et * x1 * (1 - x1) * x2 * (1 - x2)
         - 1e-5 * gamma * math.pi ** 2 * np.sin(math.pi * t)
         * (-2 * sx * s1 * s2 + cx * (x1 * s1 * c2 + x2 * c1 * s2)))
    return f, g


def example2_exact(x1, x2, t, gamma):
    """Example 2: y = e^{-t} x1(1-x1) x2(1-x2), p = gamma sin(pi t) sin(pi x1) sin(pi x2)."""
    y = np.exp(-t) * x1 * (1 - x1) * x2 * (1 - x2)
    p = gamma * np.sin(math.pi * t) * np.sin(math.pi * x1) * np.sin(math.pi * x2)
    return y, p


def example2_problem(m1: int, n: int, gamma: float, T: float = 1.0) -> Problem:
    """Example 2 (Section 3): a = 1e-5 sin(pi x1 x2) with the manufactured f, g."""
    x1, x2 = interior_grid(m1, 2)
    X1, X2 = node_grid(m1, 2)
    a = 1e-5 * np.sin(math.pi * X1 * X2)
    t = time_levels(T, n)[:, None, None]
    f, g = _example2_fg(x1[None], x2[None], t, gamma)
    y0, _ = example2_exact(x1, x2, 0.0, gamma)
    tau = T / (n + 1)
    p = Problem(2, m1, n, T, gamma, _paper_eps(tau), a, f, g, y0,
                name=f"example2-m{m1}-n{n}")
    fT, _ = _example2_fg(x1, x2, T, gamma)
    _, g0 = _example2_fg(x1, x2, 0.0, gamma)
    p.extra["f_T"] = fT
    p.extra["g_0"] = g0
    return p
