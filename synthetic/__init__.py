"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package only *generates input fields* (coefficients, targets, sources,
initial states) on the grid.  It holds none of the solver's arithmetic: no
stencil, no FFT of the method, no preconditioner, no Krylov step.
"""
from .fields import *  # noqa: F401,F403
