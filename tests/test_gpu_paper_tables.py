"""The GPU solver at the paper's own sizes (n = 2^k - 1 time blocks, eps =
min{1/2, tau/2}, left-preconditioned GMRES from zero, tol 1e-8, Section 3)
reproduces the iteration counts and discretisation errors printed in Table 3
(Example 1, sine-transform solves) and Table 7 (Example 2, one V-cycle); the
end-point values y^(N), p^(0) come from the GPU too (pc_end_point_solves)."""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from oracle import system as osy

from conftest import read_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_22686_gb300 import build
    build.build()


def _printed(value, printed):
    unit = 10.0 ** (math.floor(math.log10(abs(printed))) - 2)
    return abs(value - printed) <= 0.6 * unit


def _gpu_example(ex, m1, n, gamma, smoother="red-black"):
    from paper_2410_22686_gb300 import Solver
    P = (S.example1_problem if ex == 1 else S.example2_problem)(m1, n, gamma)
    sol = Solver(2, m1, n, P.T, gamma, P.eps, P.a_nodes, spatial="fst" if ex == 1 else "mg",
                 precision="fp64", max_iter=150, smoother=smoother)
    b = sol.build_rhs(torch.from_numpy(P.f).cuda(), torch.from_numpy(P.g).cuda(), torch.from_numpy(P.y0).cuda())
    _, it_paper_mode, _ = sol.solve(b, rtol=1e-8, mode="left")
    x, _, rel = sol.solve(b, rtol=1e-12, mode="right")
    # end-point values y^(N), p^(0) on the GPU as well
    yNd, p0d, _ = sol.end_point_solves(x, f_T=torch.from_numpy(P.extra["f_T"]).cuda(),
                                       g_0=torch.from_numpy(P.extra["g_0"]).cuda(),
                                       y0=torch.from_numpy(P.y0).cuda(), rtol=1e-13)
    sol.close()
    xg = x.cpu().numpy()
    y, p = osy.unscale(xg, gamma)
    yN, p0 = yNd.cpu().numpy(), p0d.cpu().numpy()
    N = n + 1
    x1, x2 = S.interior_grid(m1, 2)
    tl = P.tau * np.arange(N + 1)
    exact = S.example1_exact if ex == 1 else (lambda u, v, t: S.example2_exact(u, v, t, gamma))
    yex = [exact(x1, x2, tl[j])[0] for j in range(1, N + 1)]
    pex = [exact(x1, x2, tl[j])[1] for j in range(0, N)]
    eh = osy.error_measure(list(y) + [yN], [p0] + list(p), yex, pex, P.h, 2)
    return it_paper_mode, eh


@pytest.mark.parametrize("row", read_golden("table3_example1.txt"))
def test_gpu_reproduces_table3(row):
    gamma, lh, lt, it, eh = float(row[0]), int(row[1]), int(row[2]), int(row[4]), float(row[5])
    iters, got = _gpu_example(1, 2 ** lh - 1, 2 ** lt - 1, gamma)
    assert _printed(got, eh), (got, eh)
    assert abs(iters - it) <= 1, (iters, it)


@pytest.mark.parametrize("row", read_golden("table7_example2.txt"))
def test_gpu_reproduces_table7(row):
    gamma, lh, lt, it, eh = float(row[0]), int(row[1]), int(row[2]), int(row[4]), float(row[5])
    iters, got = _gpu_example(2, 2 ** lh - 1, 2 ** lt - 1, gamma)
    assert _printed(got, eh), (got, eh)
    assert abs(iters - it) <= 3, (iters, it)


@pytest.mark.parametrize("row", read_golden("table7_example2.txt"))
def test_gpu_lexicographic_smoother_gives_table7_exactly(row):
    # Gauss-Seidel in the natural order: every iteration count of Table 7, e_h to the printed digit
    gamma, lh, lt, it, eh = float(row[0]), int(row[1]), int(row[2]), int(row[4]), float(row[5])
    iters, got = _gpu_example(2, 2 ** lh - 1, 2 ** lt - 1, gamma, "lexicographic")
    assert _printed(got, eh), (got, eh)
    assert iters == it, (iters, it)
