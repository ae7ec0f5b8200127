"""Right-preconditioned GMRES reports success only when the true residual meets rtol.

The solve stops on the least-squares estimate of ||b - A x|| / ||b||.  With the FP32
preconditioner (flexible GMRES, double-float basis) the true residual formed at exit
can sit just above that estimate; the library then continues from x in a fresh Krylov
space (pc_gmres_solve, the graph-launched solve and the batch).  The contract checked
here, on the host-driven and graph-launched solves at tolerances down to the FP32
path's floor: a solve that returns without PC_ERR_NOT_CONVERGED has a true residual
<= rtol, measured independently with the oracle's A, and the solution agrees with the
oracle's.  Whether a continuation happened shows in the residual history, which then
covers only the last Krylov space (fewer entries than iterations + 1).
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import krylov as okr, precond as opc, system as osy

pytestmark = pytest.mark.gpu

RTOLS = (1e-8, 1e-9, 1e-10, 3e-11, 1e-11, 3e-12, 1e-12)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_22686_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _problem(case):
    if case == "plain":
        return S.plain_fp64_problem(), "fst"
    return S.variable_2d_problem(gamma=1e-6, m1=63, n=64), "mg"


def _oracle(prob, spatial):
    a = prob.a_nodes if prob.a_nodes is not None else np.ones((prob.m1 + 2,) * prob.d)
    tau, alpha = prob.tau, osy.alpha_weight(prob.T, prob.n, prob.gamma)
    b = osy.build_rhs(prob.f, prob.g, prob.y0, tau, prob.gamma)
    spat = opc.make_spatial_solver(spatial, prob.a_nodes, prob.m1, prob.d, tau)
    A = lambda v: osy.apply_A(v, a, tau, alpha)
    Pi = lambda v: opc.apply_Peps_inv(v, prob.n, alpha, prob.eps, spat)
    return b, A, okr.gmres(A, Pi, b, rtol=1e-13, maxit=200, mode="right")


@pytest.mark.parametrize("precision", ["fp32", "bf16s"])
@pytest.mark.parametrize("case", ["plain", "variable"])
def test_success_means_true_residual_below_rtol(case, precision):
    from paper_2410_22686_gb300 import Solver, capi
    prob, spatial = _problem(case)
    if precision == "bf16s" and spatial != "mg":
        pytest.skip("BF16 storage is a multigrid smoother variant")
    b, A, ref = _oracle(prob, spatial)
    sol = Solver(prob.d, prob.m1, prob.n, prob.T, prob.gamma, prob.eps, prob.a_nodes, spatial=spatial,
                 precision=precision, max_iter=80)
    bd = torch.from_numpy(b).cuda()
    nb = np.linalg.norm(b)
    outcomes = []
    for graph in (False, True):
        for rtol in RTOLS:
            try:
                if graph:
                    x, it, rel = sol.solve_graph(bd, rtol=rtol, maxit=80)
                else:
                    x, it, rel = sol.solve(bd, rtol=rtol, maxit=80)
            except capi.PCError as err:
                assert err.status == capi.PC_ERR_NOT_CONVERGED
                outcomes.append((graph, rtol, "not converged"))
                continue
            xg = x.cpu().numpy()
            true_rel = np.linalg.norm(b - A(xg)) / nb
            assert rel <= rtol, (graph, rtol, it, rel)
            # forming b - A x in FP64 costs ~1e-16 ||A|| ||x|| / ||b||: 1e-13 of slack
            assert true_rel <= rtol + 1e-13, (graph, rtol, it, rel, true_rel)
            assert abs(true_rel - rel) <= 1e-3 * rel + 1e-13
            if rtol <= 1e-11:
                assert np.linalg.norm(xg - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
            hist = sol.residual_history()
            outcomes.append((graph, rtol, it, len(hist) - 1 < it))
    # the strictest tolerances may end at the FP32 path's floor, the looser ones may not
    assert all(o[2] != "not converged" for o in outcomes if o[1] >= 1e-10), outcomes
    sol.close()
