"""Graph-captured solves (device-controlled WHILE loop) and batched solves of
uneven problems in one graph launch, against the host-driven solve and the oracle."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import krylov as okr, precond as opc, system as osy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_22686_gb300 import build
    build.build()


def _make(prob, precision, max_iter=60):
    from paper_2410_22686_gb300 import Solver
    sol = Solver(2, prob.m1, prob.n, prob.T, prob.gamma, prob.eps, prob.a_nodes, spatial="mg",
                 precision=precision, max_iter=max_iter)
    b = sol.build_rhs(torch.from_numpy(prob.f).cuda(), torch.from_numpy(prob.g).cuda(),
                      torch.from_numpy(prob.y0).cuda())
    return sol, b


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_solve_equals_host_driven_solve(precision):
    prob = S.variable_2d_problem(gamma=1e-4, m1=63, n=64)
    sol, b = _make(prob, precision)
    x_ref, it_ref, rr_ref = sol.solve(b, rtol=1e-10)
    for _ in range(2):  # second call replays the cached graph
        x, it, rr = sol.solve_graph(b, rtol=1e-10)
        assert it == it_ref
        assert rr <= 1e-10
        assert (x - x_ref).norm().item() <= 1e-12 * x_ref.norm().item()
    sol.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16s"])
def test_solves_are_bitwise_reproducible(precision):
    """Fixed grids and fixed reduction orders: the same solve twice gives the same bits
    (host-driven and graph-launched), and so do two preconditioner applies."""
    prob = S.variable_2d_problem(gamma=1e-4, m1=63, n=64)
    sol, b = _make(prob, precision)
    x1, it1, r1 = sol.solve(b, rtol=1e-8)
    x2, it2, r2 = sol.solve(b, rtol=1e-8)
    assert (it1, r1) == (it2, r2) and torch.equal(x1, x2)
    g1 = sol.solve_graph(b, rtol=1e-8)[0].clone()
    g2 = sol.solve_graph(b, rtol=1e-8)[0]
    assert torch.equal(g1, g2)
    w1, w2 = sol.apply_precond(b), sol.apply_precond(b)
    assert torch.equal(w1, w2)
    sol.close()


def test_residual_history_of_host_graph_and_batch_solves():
    """The history is the Givens estimate after every iteration: starts at 1 (zero
    initial guess), never increases, ends at or below rtol, one entry per iteration
    plus the start; host-driven, graph and batched solves give the same history (to
    1e-4: the two paths round the mixed-precision iteration differently, ~1e-6 relative
    in the last estimates)."""
    from paper_2410_22686_gb300 import Batch
    prob = S.variable_2d_problem(gamma=1e-6, m1=63, n=64)
    sol, b = _make(prob, "fp32")
    assert sol.residual_history() == []  # no solve yet
    x, it, rr = sol.solve(b, rtol=1e-8)
    h1 = np.array(sol.residual_history())
    assert len(h1) == it + 1 and h1[0] == 1.0
    assert np.all(np.diff(h1) <= 0) and h1[-1] <= 1e-8 < h1[-2]
    assert len(sol.residual_history(cap=3)) == 3
    xg, itg, _ = sol.solve_graph(b, rtol=1e-8)
    h2 = np.array(sol.residual_history())
    assert itg == it and np.allclose(h2, h1, rtol=1e-4, atol=0)
    bt = Batch([sol], [b], rtol=1e-8, maxit=60)
    itb, _ = bt.solve()
    h3 = np.array(sol.residual_history())
    assert itb[0] == it and np.allclose(h3, h1, rtol=1e-4, atol=0)
    bt.close()
    sol.close()


def test_batch_of_uneven_problems_matches_individual_solves_and_oracle():
    from paper_2410_22686_gb300 import Batch
    probs = [S.variable_2d_problem(gamma=1e-2, m1=15, n=16), S.variable_2d_problem(gamma=1e-6, m1=31, n=64),
             S.variable_2d_problem(gamma=1e-4, m1=63, n=32), S.gradient_problem(m1=31, n=16, gamma=1e-8)]
    precs = ["fp64", "fp32", "fp64", "bf16s"]
    made = [_make(p, q, max_iter=80) for p, q in zip(probs, precs)]
    sols, bs = [m[0] for m in made], [m[1] for m in made]
    singles = [s.solve(b, rtol=1e-10) for s, b in zip(sols, bs)]
    batch = Batch(sols, bs, rtol=1e-10, maxit=80)
    for _ in range(2):
        iters, rel = batch.solve()
        for k in range(len(probs)):
            x_ref, it_ref, _ = singles[k]
            assert iters[k] == it_ref
            assert rel[k] <= 1e-10
            assert (batch.xs[k] - x_ref).norm().item() <= 1e-12 * x_ref.norm().item()
    # the FP64 members against the oracle
    for k in (0, 2):
        p = probs[k]
        tau, alpha = p.tau, osy.alpha_weight(p.T, p.n, p.gamma)
        bo = osy.build_rhs(p.f, p.g, p.y0, tau, p.gamma)
        mg = opc.MGSpatialSolver(p.a_nodes, tau)
        ref = okr.gmres(lambda v: osy.apply_A(v, p.a_nodes, tau, alpha),
                        lambda v: opc.apply_Peps_inv(v, p.n, alpha, p.eps, mg), bo, rtol=1e-13, maxit=200)
        xg = batch.xs[k].cpu().numpy()
        assert np.linalg.norm(xg - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    batch.close()
    for s in sols:
        s.close()


def test_graph_solve_zero_rhs_and_maxit():
    from paper_2410_22686_gb300 import capi
    prob = S.variable_2d_problem(gamma=1e-4, m1=15, n=16)
    sol, b = _make(prob, "fp32")
    x, it, rr = sol.solve_graph(torch.zeros_like(b), rtol=1e-8)
    assert it == 0 and float(x.abs().max()) == 0.0
    x, it, rr = sol.solve_graph(b, rtol=1e-14, maxit=3, raise_on_nonconv=False)
    assert it == 3
    with pytest.raises(capi.PCError) as ei:
        sol.solve_graph(b, rtol=1e-14, maxit=3)
    assert ei.value.status == capi.PC_ERR_NOT_CONVERGED
    sol.close()


def test_pipelined_host_solves_equal_device_solves():
    # copies overlapped with the solves on a second stream change nothing in the results
    from paper_2410_22686_gb300 import Solver, solve_host_pipelined
    sols, hb, hx, ref = [], [], [], []
    for gamma in (1e-2, 1e-4, 1e-6):
        prob = S.variable_2d_problem(gamma=gamma, m1=31, n=16)
        sol = Solver(2, prob.m1, prob.n, prob.T, prob.gamma, prob.eps, prob.a_nodes, spatial="mg",
                     precision="mixed", max_iter=60)
        b = sol.build_rhs(torch.from_numpy(prob.f).cuda(), torch.from_numpy(prob.g).cuda(),
                          torch.from_numpy(prob.y0).cuda())
        x, it, rr = sol.solve(b, rtol=1e-8)
        sols.append(sol)
        hb.append(b.cpu().pin_memory())
        hx.append(torch.empty(b.shape, dtype=torch.float64).pin_memory())
        ref.append((x.cpu(), it, rr))
    for _ in range(2):
        res = solve_host_pipelined(list(zip(sols, hb, hx)), rtol=1e-8)
        for (xr, itr, rrr), (it, rr), xh in zip(ref, res, hx):
            assert it == itr and rr == rrr
            assert torch.equal(xh, xr)
    # the same solver listed twice gets a second pair of device buffers for that call
    hx2 = [torch.empty(hx[0].shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    res = solve_host_pipelined([(sols[0], hb[0], hx2[0]), (sols[0], hb[0], hx2[1])], rtol=1e-8)
    for (it, rr), xh in zip(res, hx2):
        assert it == ref[0][1] and rr == ref[0][2]
        assert torch.equal(xh, ref[0][0])
    # solving into a given vector equals the allocating call
    out = torch.full((sols[1].vec_len,), 7.0, dtype=torch.float64, device="cuda")
    x, it, rr = sols[1].solve(hb[1].cuda(), rtol=1e-8, out=out)
    assert x.data_ptr() == out.data_ptr() and it == ref[1][1] and torch.equal(x.cpu().reshape(ref[1][0].shape), ref[1][0])
    for s in sols:
        s.close()
