"""Tile shapes (pc_set_tiles / pc_autotune): every shape gives the oracle's result."""
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


def _rel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


SHAPES = [dict(mg_cx=8, mg_ctas=2, mv_tj=8, pro_pch=2, fft_stream=1, mg_march=0, mg_seg=0, fst_stream=1),
          dict(mg_cx=16, mg_ctas=32, mv_tj=128, pro_pch=32, fft_stream=0, mg_march=1, mg_seg=16, fst_stream=2),
          dict(mg_cx=16, mg_ctas=1, mv_tj=1, pro_pch=1, fft_stream=1, mg_march=1, mg_seg=1, fst_stream=3),
          dict(mg_cx=0, mg_ctas=0, mv_tj=0, pro_pch=0, fft_stream=0, mg_march=1, mg_seg=1024, fst_stream=0)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5), ("bf16s", 3e-2)])
@pytest.mark.parametrize("d,m1,n", [(2, 63, 16), (2, 127, 8), (3, 15, 8), (2, 31, 256), (2, 15, 512), (2, 31, 128),
                                    (2, 7, 1024)])
def test_precond_and_matvec_match_oracle_for_every_tile_shape(precision, tol, d, m1, n):
    from paper_2410_22686_gb300 import Solver
    a = np.exp(0.4 * S.random_vector((m1 + 2,) * d, 5))
    gamma, eps = 1e-4, 0.25
    sol = Solver(d, m1, n, 1.0, gamma, eps, a, spatial="mg", precision=precision, max_iter=4, tiles=None)
    v = S.random_vector((2, n) + (m1,) * d, 21)
    tau, alpha = osy.time_step(1.0, n), osy.alpha_weight(1.0, n, gamma)
    ref = opc.apply_Peps_inv(v, n, alpha, eps, opc.make_spatial_solver("mg", a, m1, d, tau))
    ref_mv = osy.apply_A(v, a, tau, alpha)
    dv = torch.from_numpy(v).cuda()
    base = sol.apply_precond(dv).cpu().numpy()
    assert _rel(base, ref) <= tol
    for shape in SHAPES:
        sol.set_tiles(**shape)
        assert sol.get_tiles() == shape
        w = sol.apply_precond(dv).cpu().numpy()
        assert _rel(w, ref) <= tol, shape
        # same arithmetic, only the work split differs
        assert _rel(w, base) <= (1e-13 if precision == "fp64" else tol), shape
        assert _rel(sol.matvec(dv).cpu().numpy(), ref_mv) <= 1e-12, shape
    sol.close()


def test_invalid_tile_shapes_are_rejected():
    from paper_2410_22686_gb300 import Solver, capi
    sol = Solver(2, 15, 8, 1.0, 1e-3, 0.3, None, spatial="fst", tiles=None)
    for bad in (dict(mg_cx=12), dict(mg_ctas=-1), dict(mv_tj=5000), dict(pro_pch=65), dict(fft_stream=2),
                dict(mg_march=2), dict(mg_seg=-1), dict(fst_stream=4), dict(fst_stream=-1)):
        with pytest.raises(capi.PCError):
            sol.set_tiles(**bad)
    with pytest.raises(ValueError):
        sol.set_tiles(nope=1)
    sol.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotune_picks_valid_shapes_and_keeps_the_solution(precision):
    from paper_2410_22686_gb300 import Solver
    # 127^2: one fine level with a fused down leg (the levels from 63^2 down run in
    # one kernel), so the down-leg shape is tuned
    prob = S.variable_2d_problem(gamma=1e-4, m1=127, n=32)
    sol = Solver(2, prob.m1, prob.n, prob.T, prob.gamma, prob.eps, prob.a_nodes, spatial="mg",
                 precision=precision, max_iter=60, tiles=None)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    b = sol.build_rhs(dev(prob.f), dev(prob.g), dev(prob.y0))
    x0, it0, rr0 = sol.solve(b, rtol=1e-8)
    t = sol.autotune(reps=2)
    assert t["mg_cx"] in (8, 16) and 1 <= t["mg_ctas"] <= 64
    # pro_pch stays 0 (default) when the handle launches no prolongation kernel:
    # at 127^2 the only fine level's correction is fused into the inverse FFT
    assert 1 <= t["mv_tj"] <= 4096 and 0 <= t["pro_pch"] <= 64 and t["fft_stream"] in (0, 1)
    assert sol.get_tiles() == t
    x1, it1, rr1 = sol.solve(b, rtol=1e-8)
    assert rr1 <= 1e-8 and abs(it1 - it0) <= 1
    x0, x1 = x0.cpu().numpy(), x1.cpu().numpy()
    assert np.linalg.norm(x1 - x0) <= 1e-7 * np.linalg.norm(x0)
    sol.close()
