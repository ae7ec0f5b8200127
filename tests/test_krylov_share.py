"""Shared Krylov storage (pc_krylov_bytes, pc_setup_shared, pack_krylov): the host
side, no GPU needed (nothing here reaches device memory)."""
import ctypes

import pytest

from paper_2410_22686_gb300 import capi
from paper_2410_22686_gb300.solver import pack_krylov


def _params(dim=2, m1=31, n=32, precision=capi.PC_PREC_MIXED_FP32, max_iter=20, eps=0.1):
    return capi.pc_params(dim, m1, n, 1.0, 1e-2, eps, capi.PC_SPATIAL_AUTO, precision, max_iter,
                          capi.PC_SPACE_FD, capi.PC_SMOOTHER_RED_BLACK)


def _bytes(p):
    out = ctypes.c_size_t(0)
    st = capi.load().pc_krylov_bytes(ctypes.byref(p), ctypes.byref(out))
    return st, out.value


@pytest.mark.parametrize("dim,m1,n,prec,cap", [(2, 31, 32, capi.PC_PREC_MIXED_FP32, 20),
                                               (2, 255, 256, capi.PC_PREC_MIXED_FP32, 48),
                                               (3, 7, 16, capi.PC_PREC_FP64, 5),
                                               (2, 3, 1, capi.PC_PREC_MIXED_BF16S, 1)])
def test_krylov_bytes_counts_basis_and_preconditioned_vectors(dim, m1, n, prec, cap):
    U = 2 * n * m1 ** dim
    r256 = lambda b: -(-b // 256) * 256
    # basis: cap + 1 vectors padded to whole tiles of 512 unknowns, 8 bytes each;
    # then cap preconditioned vectors of 4 (FP32 preconditioner) or 8 bytes per unknown
    basis = r256((cap + 1) * (-(-U // 512) * 512) * 8)
    zvec = r256(cap * U * (8 if prec == capi.PC_PREC_FP64 else 4))
    st, b = _bytes(_params(dim, m1, n, prec, cap))
    assert st == capi.PC_OK
    assert b == basis + zvec


def test_krylov_bytes_resolves_automatic_precision_by_eps():
    _, b32 = _bytes(_params(precision=capi.PC_PREC_MIXED_FP32))
    _, b64 = _bytes(_params(precision=capi.PC_PREC_FP64))
    _, big = _bytes(_params(precision=capi.PC_PREC_AUTO, eps=0.9))
    _, small = _bytes(_params(precision=capi.PC_PREC_AUTO, eps=1e-6))
    assert {big, small} == {b32, b64}


def test_krylov_bytes_and_shared_setup_reject_bad_arguments_on_the_host():
    lib = capi.load()
    assert _bytes(_params(dim=4))[0] == capi.PC_ERR_ARG
    assert _bytes(_params(max_iter=0))[0] == capi.PC_ERR_ARG
    assert _bytes(_params(n=5000))[0] == capi.PC_ERR_ARG
    assert lib.pc_krylov_bytes(None, None) == capi.PC_ERR_ARG
    p = _params()
    _, need = _bytes(p)
    h = ctypes.c_void_p()
    # null, misaligned and too small workspaces fail before any device work
    assert lib.pc_setup_shared(ctypes.byref(p), None, None, need, None, ctypes.byref(h)) == capi.PC_ERR_ARG
    assert lib.pc_setup_shared(ctypes.byref(p), None, ctypes.c_void_p(4096 + 16), need, None,
                               ctypes.byref(h)) == capi.PC_ERR_ARG
    assert lib.pc_setup_shared(ctypes.byref(p), None, ctypes.c_void_p(4096), need - 1, None,
                               ctypes.byref(h)) == capi.PC_ERR_ARG
    assert b"needed" in lib.pc_last_error()
    assert not h.value


def test_pack_krylov_fills_waves_in_order():
    sizes = [100, 300, 250, 10, 600, 5]
    offs = pack_krylov(sizes, 1024, align=256)
    # 256 + 512 + 256 fill the first 1024 bytes, the fourth starts the next wave
    assert offs == [0, 256, 768, 0, 256, 0]
    with pytest.raises(ValueError):
        pack_krylov([2000], 1024)
    # within a wave (between two returns to offset 0) the ranges never overlap
    sizes = [37, 1000, 999, 4096, 1, 512, 3000, 77]
    offs = pack_krylov(sizes, 8192)
    wave, waves = [], []
    for o, b in zip(offs, sizes):
        if o == 0 and wave:
            waves.append(wave)
            wave = []
        wave.append((o, -(-b // 256) * 256))
    waves.append(wave)
    for w in waves:
        for (o1, b1), (o2, b2) in zip(w, w[1:]):
            assert o1 + b1 <= o2
        assert w[-1][0] + w[-1][1] <= 8192
