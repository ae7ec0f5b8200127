"""ctypes binding of libpcopt (include/pcopt.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  Vectors are torch CUDA tensors (float64, contiguous); their device
pointers and torch's current CUDA stream are handed to the C functions.  If
the library has not been built, or cannot be loaded, ``load()`` raises: there
is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpcopt.so")
# the checked build (compiled with -DPCOPT_DEBUG); PCOPT_LIBRARY=debug selects it
DEBUG_LIB_PATH = os.path.join(HERE, "libpcopt_debug.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pcopt.h")

(PC_OK, PC_ERR_ARG, PC_ERR_CUDA, PC_ERR_OOM, PC_ERR_NOT_CONVERGED, PC_ERR_BREAKDOWN, PC_ERR_UNSUPPORTED,
 PC_ERR_TIMEOUT) = range(8)
PC_SPATIAL_AUTO, PC_SPATIAL_FST, PC_SPATIAL_MG = 0, 1, 2
PC_PREC_FP64, PC_PREC_MIXED_FP32, PC_PREC_MIXED_BF16S, PC_PREC_AUTO = 0, 1, 2, 3
PC_GMRES_RIGHT, PC_GMRES_LEFT = 0, 1
PC_SPACE_FD, PC_SPACE_FE = 0, 1
PC_SMOOTHER_RED_BLACK, PC_SMOOTHER_LEXICOGRAPHIC = 0, 1
PC_PRECOND_EPS_CIRCULANT, PC_PRECOND_IDEAL_RBD = 0, 1
PC_ARNOLDI_AUTO, PC_ARNOLDI_FP64, PC_ARNOLDI_FP64_STRICT, PC_ARNOLDI_DOUBLE_FLOAT = 0, 1, 2, 3


class pc_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("m1", ctypes.c_int), ("n", ctypes.c_int),
                ("T", ctypes.c_double), ("gamma", ctypes.c_double), ("eps", ctypes.c_double),
                ("spatial", ctypes.c_int), ("precision", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("space", ctypes.c_int), ("smoother", ctypes.c_int)]


class pc_tiles(ctypes.Structure):
    _fields_ = [("mg_cx", ctypes.c_int), ("mg_ctas", ctypes.c_int), ("mv_tj", ctypes.c_int),
                ("pro_pch", ctypes.c_int), ("fft_stream", ctypes.c_int), ("mg_march", ctypes.c_int),
                ("mg_seg", ctypes.c_int), ("fst_stream", ctypes.c_int)]


class pc_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class PCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pcopt status {status}: {msg}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_ip = ctypes.POINTER(ctypes.c_int)
_dpp = ctypes.POINTER(ctypes.c_double)

_SIGNATURES = {
    "pc_setup": (_i, [ctypes.POINTER(pc_params), _vp, _vp, ctypes.POINTER(_vp)]),
    "pc_krylov_bytes": (_i, [ctypes.POINTER(pc_params), ctypes.POINTER(ctypes.c_size_t)]),
    "pc_setup_shared": (_i, [ctypes.POINTER(pc_params), _vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "pc_destroy": (_i, [_vp]),
    "pc_set_coefficient": (_i, [_vp, _vp, _vp]),
    "pc_matvec": (_i, [_vp, _dp, _dp, _vp]),
    "pc_matvec_transpose": (_i, [_vp, _dp, _dp, _vp]),
    "pc_matvec_f32": (_i, [_vp, _vp, _dp, _vp]),
    "pc_apply_precond": (_i, [_vp, _dp, _dp, _vp]),
    "pc_build_rhs": (_i, [_vp, _dp, _dp, _dp, _dp, _vp]),
    "pc_gmres_solve": (_i, [_vp, _dp, _dp, _d, _i, _i, _ip, _dpp, _vp]),
    "pc_gmres_solve_graph": (_i, [_vp, _dp, _dp, _d, _i, _ip, _dpp, _vp]),
    "pc_residual_history": (_i, [_vp, _dpp, _i, _ip, _vp]),
    "pc_batch_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _i,
                             ctypes.POINTER(_vp)]),
    "pc_batch_solve": (_i, [_vp, _ip, _dpp, _vp]),
    "pc_batch_destroy": (_i, [_vp]),
    "pc_adjoint_solve": (_i, [_vp, _dp, _dp, _d, _i, _i, _ip, _dpp, _vp]),
    "pc_grad_log_a": (_i, [_vp, _dp, _dp, _dp, _vp]),
    "pc_grad_log_a_noalloc": (_i, [_i, _i, _i, _d, _dp, _dp, _dp, _dp, _vp]),
    "pc_set_log_coefficient": (_i, [_vp, _dp, _vp]),
    "pc_set_preconditioner": (_i, [_vp, _i]),
    "pc_set_arnoldi": (_i, [_vp, _i]),
    "pc_grad_g": (_i, [_vp, _dp, _dp, _vp]),
    "pc_objective": (_i, [_vp, _dp, _dp, _dp, _vp]),
    "pc_objective_grad": (_i, [_vp, _dp, _dp, _dp, _dp, _dp, _vp]),
    "pc_sizes": (_i, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "pc_precision_of": (_i, [_vp, _ip]),
    "pc_end_point_solves": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_double, _i, _ip, _vp]),
    "pc_get_tiles": (_i, [_vp, ctypes.POINTER(pc_tiles)]),
    "pc_set_tiles": (_i, [_vp, ctypes.POINTER(pc_tiles)]),
    "pc_autotune": (_i, [_vp, _i, ctypes.POINTER(pc_tiles), _vp]),
    "pc_profile": (_i, [_vp, _i]),
    "pc_stats": (_i, [_vp, ctypes.POINTER(pc_kernel_stat), _i, _ip]),
    "pc_stats_reset": (_i, [_vp]),
    "pc_profile_classes": (_i, [_vp, ctypes.c_char_p]),
    "pc_launch_count": (ctypes.c_int64, [_vp]),
    "pc_measure_peaks": (_i, [_dpp, _dpp, _vp]),
    "pc_selftest_wait_timeout": (_i, [_d, _vp]),
    "pc_debug_status": (_i, [_i, _ip]),
    "pc_last_error": (ctypes.c_char_p, []),
    "pc_status_string": (ctypes.c_char_p, [_i]),
}


def header_functions():
    """Names of the functions declared in include/pcopt.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", text)))


def load(path: str | None = None):
    """Load libpcopt.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or (DEBUG_LIB_PATH if os.environ.get("PCOPT_LIBRARY") == "debug" else LIB_PATH)
    if not os.path.exists(p):
        raise RuntimeError(f"{p} not found: the CUDA library must be built (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status: int):
    if status != PC_OK:
        lib = load()
        raise PCError(status, lib.pc_last_error().decode())
    return status
