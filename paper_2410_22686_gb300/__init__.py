"""GB300-native eps-circulant RBD-preconditioned GMRES for the all-at-once
system of parabolic optimal control (Hon, Fung & Lin, arXiv 2410.22686).

The solver is the CUDA C-ABI library ``libpcopt.so`` (``include/pcopt.h``);
this package only binds it (``capi``), wraps a handle (``Solver``) and adds a
``torch.autograd.Function`` over the solve (``autograd``).
"""
from . import capi  # noqa: F401
from .solver import Batch, Solver, krylov_bytes, measure_peaks, pack_krylov, solve_host_pipelined  # noqa: F401

__all__ = ["capi", "Solver", "Batch", "krylov_bytes", "measure_peaks", "pack_krylov", "solve_host_pipelined"]
