"""End-point solves y^(N), p^(0) (pc_end_point_solves) against the oracle's sparse
direct solves of (I + tau K) u = rhs (Section 1), on the GPU solution itself."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import system as osy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_22686_gb300 import build
    build.build()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


CASES = [("ex1", "fst", "fp64"), ("ex2", "mg", "fp64"), ("ex2", "mg", "mixed"), ("ex2", "mg", "bf16s"),
         ("3d", "mg", "fp64"), ("3d", "mg", "mixed")]


@pytest.mark.parametrize("case,spatial,precision", CASES)
def test_end_point_solves_match_oracle(case, spatial, precision):
    from paper_2410_22686_gb300 import Solver
    if case == "3d":
        P = S.gaussian_field_3d_problem(m1=15, n=8)
        fT = S.random_vector((15,) * 3, 3)
        g0 = S.random_vector((15,) * 3, 4)
        pN = S.random_vector((15,) * 3, 5)
    else:
        P = (S.example1_problem if case == "ex1" else S.example2_problem)(31, 31, 1e-2)
        fT, g0, pN = P.extra["f_T"], P.extra["g_0"], None
    d = P.d
    sol = Solver(d, P.m1, P.n, P.T, P.gamma, P.eps, P.a_nodes, spatial=spatial, precision=precision, max_iter=80)
    b = sol.build_rhs(_dev(P.f), _dev(P.g), _dev(P.y0))
    x, _, _ = sol.solve(b, rtol=1e-10)
    yN, p0, it = sol.end_point_solves(x, f_T=_dev(fT), g_0=_dev(g0), y0=_dev(P.y0),
                                      p_N=None if pN is None else _dev(pN), rtol=1e-13)
    assert 1 <= it <= (2 if spatial == "fst" else 60)
    a = P.a_nodes if P.a_nodes is not None else osy.unit_coefficient(P.m1, d)
    y, p = osy.unscale(x.cpu().numpy(), P.gamma)
    yN_ref, p0_ref = osy.end_point_solves(y, p, a, P.tau, P.gamma, fT, g0, P.y0, p_final=pN)
    assert _rel(yN.cpu().numpy(), yN_ref) <= 1e-11
    assert _rel(p0.cpu().numpy(), p0_ref) <= 1e-11
    sol.close()


def test_end_point_solves_zero_input_and_errors():
    from paper_2410_22686_gb300 import Solver, capi
    sol = Solver(2, 15, 4, 1.0, 1e-2, 0.3, None, spatial="fst")
    x = torch.zeros(sol.vec_len, dtype=torch.float64, device="cuda")
    yN, p0, it = sol.end_point_solves(x)
    assert it == 0 and float(yN.abs().max()) == 0.0 and float(p0.abs().max()) == 0.0
    with pytest.raises(capi.PCError):
        sol.end_point_solves(x, rtol=-1.0)
    with pytest.raises(ValueError):
        sol.end_point_solves(x, f_T=torch.zeros(7, dtype=torch.float64, device="cuda"))
    sol.close()
