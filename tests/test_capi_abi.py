"""The C-ABI library builds, loads and exports every function include/pcopt.h
declares (no GPU needed: nothing here calls into a kernel)."""
import ctypes
import subprocess

import pytest

from paper_2410_22686_gb300 import build as pbuild, capi


@pytest.fixture(scope="module")
def lib():
    path = pbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = capi.header_functions()
    for must in ("pc_setup", "pc_destroy", "pc_matvec", "pc_apply_precond", "pc_gmres_solve",
                 "pc_adjoint_solve", "pc_build_rhs", "pc_grad_log_a"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in capi.header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_function():
    assert set(capi.header_functions()) <= set(capi._SIGNATURES)


def test_exported_symbols_are_plain_c(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pbuild.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for name in capi.header_functions():
        assert name in exported, name


def test_status_strings_and_argument_errors_without_gpu():
    l = capi.load()
    assert l.pc_status_string(capi.PC_OK) == b"ok"
    assert l.pc_status_string(capi.PC_ERR_ARG) == b"invalid argument"
    # invalid parameters are rejected on the host before any device work
    h = ctypes.c_void_p()
    bad = [
        capi.pc_params(4, 7, 8, 1.0, 1e-2, 0.5, 0, 0, 10),     # dim
        capi.pc_params(2, 7, 5000, 1.0, 1e-2, 0.5, 0, 0, 10),  # n too large
        capi.pc_params(2, 7, 8, 1.0, 0.0, 0.5, 0, 0, 10),      # gamma
        capi.pc_params(2, 7, 8, 1.0, 1e-2, 0.0, 0, 0, 10),     # eps
        capi.pc_params(2, 7, 8, 1.0, 1e-2, 1.5, 0, 0, 10),     # eps
        capi.pc_params(2, 6, 8, 1.0, 1e-2, 0.5, 2, 0, 10),     # MG needs 2^k - 1
        capi.pc_params(2, 7, 8, -1.0, 1e-2, 0.5, 0, 0, 10),    # T
        capi.pc_params(2, 7, 8, 1.0, 1e-2, 0.5, 0, 0, 0),      # max_iter
        capi.pc_params(2, 7, 8, 1.0, 1e-2, 0.5, 0, 0, 10, 2),  # space
    ]
    for p in bad:
        assert l.pc_setup(ctypes.byref(p), None, None, ctypes.byref(h)) == capi.PC_ERR_ARG
        assert len(l.pc_last_error()) > 0
    # coefficient: > 0 inside, >= 0 on the boundary, finite everywhere
    import numpy as np
    p = capi.pc_params(2, 7, 8, 1.0, 1e-2, 0.5, 2, 0, 10)
    for (i, j, v) in [(3, 3, -1.0), (3, 3, 0.0), (0, 4, -1e-9), (8, 8, np.inf), (4, 0, np.nan)]:
        a = np.ones((9, 9))
        a[i, j] = v
        assert l.pc_setup(ctypes.byref(p), a.ctypes.data_as(ctypes.c_void_p), None,
                          ctypes.byref(h)) == capi.PC_ERR_ARG, (i, j, v)
        assert b"boundary" in l.pc_last_error()
    # finite elements: the element multigrid (2D and 3D) smooths in colour order only and
    # has no BF16 storage
    a = np.ones((9, 9, 9))
    a[4, 4, 4] = 2.0
    a2 = np.ones((9, 9))
    a2[4, 4] = 2.0
    for p, a_ptr in [(capi.pc_params(3, 7, 8, 1.0, 1e-2, 0.5, 2, 2, 10, 1), a.ctypes.data_as(ctypes.c_void_p)),
                     (capi.pc_params(3, 7, 8, 1.0, 1e-2, 0.5, 2, 0, 10, 1, 1), a.ctypes.data_as(ctypes.c_void_p)),
                     (capi.pc_params(2, 7, 8, 1.0, 1e-2, 0.5, 2, 2, 10, 1), a2.ctypes.data_as(ctypes.c_void_p)),
                     (capi.pc_params(2, 7, 8, 1.0, 1e-2, 0.5, 2, 0, 10, 1, 1), a2.ctypes.data_as(ctypes.c_void_p))]:
        assert l.pc_setup(ctypes.byref(p), a_ptr, None, ctypes.byref(h)) == capi.PC_ERR_UNSUPPORTED
        assert b"finite elements" in l.pc_last_error()
    assert l.pc_destroy(None) == capi.PC_OK


def test_noalloc_gradient_rejects_bad_sizes_without_gpu():
    """The allocation-free gradient checks its sizes on the host, before it looks
    up its scratch or launches anything."""
    l = capi.load()
    nul = ctypes.c_void_p(0)
    one = ctypes.c_void_p(8)  # never dereferenced: every case fails its size check first
    cases = [(4, 7, 8), (2, 0, 8), (2, 7, 0), (2, 7, 4097), (2, 7, 1 << 30), (3, 129, 8), (2, 1449, 8)]
    for d, m1, n in cases:
        assert l.pc_grad_log_a_noalloc(d, m1, n, 1.0, one, one, one, one, nul) == capi.PC_ERR_ARG, (d, m1, n)
        assert len(l.pc_last_error()) > 0
    assert l.pc_grad_log_a_noalloc(2, 7, 8, 1.0, nul, one, one, one, nul) == capi.PC_ERR_ARG
    assert b"null" in l.pc_last_error()


def test_debug_build_compiles_and_exports_the_boundary():
    """The checked build (-DPCOPT_DEBUG: index checks that record a code instead of
    trapping) compiles for sm_103a and exports the same C ABI; the release build
    answers pc_debug_status with PC_ERR_UNSUPPORTED and code 0 (no GPU needed)."""
    path = pbuild.build(debug=True)
    assert path.endswith("libpcopt_debug.so")
    dbg = ctypes.CDLL(path)
    for name in capi.header_functions():
        assert hasattr(dbg, name), name
    l = capi.load()
    code = ctypes.c_int(-7)
    assert l.pc_debug_status(0, ctypes.byref(code)) == capi.PC_ERR_UNSUPPORTED
    assert code.value == 0
