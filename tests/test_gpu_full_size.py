"""Parity at the full sizes of the timed workloads, in the launch configuration the
benchmark uses (Solver defaults: the stored tile table), against the FP64 CPU oracle.

* 3D random-field workload (63^3 interior grid, n = 128, 64 M unknowns): the FP32
  preconditioner (time FFTs, 3D multigrid V(1,0) cycle) element by element at 1e-5 and
  the all-at-once matvec at 1e-12, as in the small-size parity tests.
* Batched workload (64 problems, grids 31..255, n 16..512, 5.2e8 unknowns in all): each
  solution of the graph-launched batch, checked by the oracle's own operator: the true
  relative residual ||b - A x|| / ||b|| of every problem, with b and A x from the oracle,
  is at most the stopping tolerance (1e-8) plus the FP64 matvec's rounding.
The 255^2 x 256 variable-coefficient workload is covered in test_gpu_parity.py.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import precond as opc, system as osy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_22686_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


def test_full_size_3d_random_field_precond_and_matvec():
    from paper_2410_22686_gb300 import Solver
    P = S.gaussian_field_3d_problem()
    assert (P.m1, P.n) == (63, 128)
    tau, alpha = P.tau, osy.alpha_weight(P.T, P.n, P.gamma)
    sol = Solver(3, P.m1, P.n, P.T, P.gamma, P.eps, P.a_nodes, spatial="mg", precision="fp32", max_iter=60)
    v = S.random_vector((2, P.n) + (P.m1,) * 3, 43)
    w = sol.apply_precond(_dev(v)).cpu().numpy()
    y = sol.matvec(_dev(v)).cpu().numpy()
    sol.close()
    torch.cuda.empty_cache()
    assert _rel(y, osy.apply_A(v, P.a_nodes, tau, alpha)) <= 1e-12
    ref = opc.apply_Peps_inv(v, P.n, alpha, P.eps, opc.MGSpatialSolver(P.a_nodes, tau))
    assert _rel(w, ref) <= 1e-5


def test_full_size_batched_workload_residuals_by_oracle():
    from paper_2410_22686_gb300 import Batch, Solver
    rtol, cap, wave_gb = 1e-8, 48, 110.0
    probs = S.batched_problems(64)
    waves, cur, cur_b = [], [], 0.0
    for q in probs:  # the benchmark's memory-bounded waves
        need = q.unknowns * (12.0 * cap + 60.0) / 1e9
        if cur and cur_b + need > wave_gb:
            waves.append(cur)
            cur, cur_b = [], 0.0
        cur.append(q)
        cur_b += need
    if cur:
        waves.append(cur)
    checked = 0
    for wave in waves:
        sols, bs = [], []
        for q in wave:
            so = Solver(2, q.m1, q.n, q.T, q.gamma, q.eps, q.a_nodes, spatial="mg", precision="fp32",
                        max_iter=cap)
            bs.append(so.build_rhs(_dev(q.f), _dev(q.g), _dev(q.y0)))
            sols.append(so)
        bt = Batch(sols, bs, rtol=rtol, maxit=cap)
        iters, rels = bt.solve()
        xs = [x.cpu().numpy() for x in bt.xs]
        bt.close()
        for so in sols:
            so.close()
        del bs, sols
        torch.cuda.empty_cache()
        for q, x, it, rr in zip(wave, xs, iters, rels):
            assert rr <= rtol and 0 < it <= cap
            alpha = osy.alpha_weight(q.T, q.n, q.gamma)
            b = osy.build_rhs(q.f, q.g, q.y0, q.tau, q.gamma)
            r = b - osy.apply_A(x.reshape(b.shape), q.a_nodes, q.tau, alpha)
            assert np.linalg.norm(r) / np.linalg.norm(b) <= rtol * 1.05, (q.m1, q.n, q.gamma)
            checked += 1
    assert checked == 64
