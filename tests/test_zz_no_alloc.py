"""The allocation-free gradient entry point, pc_grad_log_a_noalloc.

It exists for callers that may not allocate device memory (code under a
foreign memory pool or a fixed pre-allocated budget): they cannot create a
handle, so this call takes every input explicitly and keeps its scratch in a
static device array.  Its result must equal the handle-based pc_grad_log_a on
the same inputs, call after call (the shared scratch keeps the previous call's
contents, which must not leak into the next result).
"""
import ctypes

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _noalloc(lib, d, m1, n, T, a_int, x, lam, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    return lib.pc_grad_log_a_noalloc(d, m1, n, T, p(a_int), p(x), p(lam), p(out), stream)


@pytest.fixture(scope="module")
def lib():
    from paper_2410_22686_gb300 import build, capi
    build.build()
    assert torch.cuda.is_available()
    return capi.load()


def test_noalloc_gradient_equals_handle_gradient_on_consecutive_calls(lib):
    from paper_2410_22686_gb300 import Solver, capi
    # calls in a row on different problems: 3D (default time chunks); a 2D grid
    # large enough that the time chunks are coarsened to fit the scratch (8
    # blocks per chunk, all full); 1023^2 with n = 257, where only two chunks
    # fit (129 + 128 blocks, a partial last chunk)
    cases = [(3, 15, 64, 1), (2, 511, 256, 2), (2, 1023, 257, 3)]
    for d, m1, n, seed in cases:
        a_nodes = np.exp(0.3 * S.random_vector((m1 + 2,) * d, seed))
        sol = Solver(d, m1, n, 1.0, 1e-3, 0.5, a_nodes, spatial="mg", precision="fp64", max_iter=1)
        x = torch.from_numpy(S.random_vector((2, n) + (m1,) * d, 10 + seed)).cuda()
        lam = torch.from_numpy(S.random_vector((2, n) + (m1,) * d, 20 + seed)).cuda()
        a_int = torch.from_numpy(np.ascontiguousarray(a_nodes[(slice(1, -1),) * d])).cuda()
        ref = sol.grad_log_a(x, lam)
        out = torch.full((m1,) * d, float("nan"), dtype=torch.float64, device="cuda")
        capi.check(_noalloc(lib, d, m1, n, 1.0, a_int, x, lam, out))
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item() / ref.abs().max().item()
        assert err <= 1e-12, (d, m1, n, err)
        sol.close()
        del x, lam
        torch.cuda.empty_cache()


def test_noalloc_rejects_grids_beyond_the_static_scratch(lib):
    from paper_2410_22686_gb300 import capi
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 129^3 interior points exceed PC_NOALLOC_SCRATCH_DOUBLES = 2^21
    assert _noalloc(lib, 3, 129, 8, 1.0, t, t, t, t) == capi.PC_ERR_ARG
    assert b"static scratch" in lib.pc_last_error()
    assert _noalloc(lib, 4, 7, 8, 1.0, t, t, t, t) == capi.PC_ERR_ARG
    # n beyond a handle's limit
    assert _noalloc(lib, 2, 7, 4097, 1.0, t, t, t, t) == capi.PC_ERR_ARG
