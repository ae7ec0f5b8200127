"""Problems whose Krylov storage is shared (pc_setup_shared) give the results of
problems with storage of their own: in one batch graph launch (the batch orders
problems whose storage overlaps), and in host-driven solves one after another."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu

CASES = [(15, 16, 1e-2), (31, 32, 1e-4), (15, 64, 1e-6), (31, 16, 1e-8), (7, 32, 1e-3)]
CAP = 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_22686_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _problems():
    return [S.variable_2d_problem(gamma=g, m1=m1, n=n) for m1, n, g in CASES]


def _solver(p, krylov=None):
    from paper_2410_22686_gb300 import Solver
    return Solver(2, p.m1, p.n, p.T, p.gamma, p.eps, p.a_nodes, spatial="mg", precision="fp32", max_iter=CAP,
                  krylov=krylov)


def _rhs(s, p):
    return s.build_rhs(torch.from_numpy(p.f).cuda(), torch.from_numpy(p.g).cuda(), torch.from_numpy(p.y0).cuda())


def _reference(probs):
    out = []
    for p in probs:
        s = _solver(p)
        x, it, rr = s.solve_graph(_rhs(s, p), rtol=1e-10, maxit=CAP)
        out.append((x.cpu().numpy(), it, rr))
        s.close()
    return out


@pytest.mark.parametrize("layout", ["one-range", "two-at-a-time", "disjoint"])
def test_batch_with_shared_krylov_storage_equals_separate_solves(layout):
    from paper_2410_22686_gb300 import Batch, krylov_bytes, pack_krylov
    probs = _problems()
    ref = _reference(probs)
    sizes = [krylov_bytes(2, p.m1, p.n, p.eps, "fp32", CAP) for p in probs]
    if layout == "one-range":      # every problem at offset 0: a chain, one after another
        pool, offs = max(sizes), [0] * len(sizes)
    elif layout == "two-at-a-time":
        pool = sorted(sizes)[-1] + sorted(sizes)[-2] + 512
        offs = pack_krylov(sizes, pool)
    else:                          # room for all: nothing overlaps, all concurrent
        pool = sum(-(-b // 256) * 256 for b in sizes)
        offs = pack_krylov(sizes, pool)
    buf = torch.empty(pool, dtype=torch.uint8, device="cuda")
    sols = [_solver(p, buf[o:o + b]) for p, o, b in zip(probs, offs, sizes)]
    bs = [_rhs(s, p) for s, p in zip(sols, probs)]
    bt = Batch(sols, bs, rtol=1e-10, maxit=CAP)
    for _ in range(2):  # a second launch reuses the graph and the storage
        its, rrs = bt.solve()
        for (xr, itr, rrr), x, it, rr in zip(ref, bt.xs, its, rrs):
            assert it == itr
            assert rr <= 1e-10
            xg = x.cpu().numpy()
            assert np.linalg.norm(xg - xr) <= 1e-12 * np.linalg.norm(xr)
    bt.close()
    # host-driven solves on the sharing handles, one after another
    for s, b, (xr, itr, _) in zip(sols, bs, ref):
        x, it, rr = s.solve(b, rtol=1e-10, maxit=CAP)
        assert it == itr and rr <= 1e-10
        assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-9 * np.linalg.norm(xr)
    for s in sols:
        s.close()


def test_shared_setup_rejects_short_or_misaligned_storage():
    from paper_2410_22686_gb300 import capi, krylov_bytes
    p = _problems()[0]
    need = krylov_bytes(2, p.m1, p.n, p.eps, "fp32", CAP)
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.PCError) as e:
        _solver(p, buf[: need - 256])
    assert e.value.status == capi.PC_ERR_ARG
    with pytest.raises(capi.PCError) as e:
        _solver(p, buf[16: 16 + need])
    assert e.value.status == capi.PC_ERR_ARG
