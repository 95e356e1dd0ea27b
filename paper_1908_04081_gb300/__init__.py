"""Adaptive s-step conjugate gradient (Carson 2019, Algorithm 5) on GB300.

The solver is the C-ABI library ``libsscg.so`` (CUDA kernels for sm_103a,
declared in ``include/sscg.h``); ``sscg`` is its thin ctypes binding.  Import
is lazy: nothing is loaded until a binding function is called.
"""
from . import sscg  # noqa: F401
from .sscg import Solver, SscgError, load_library  # noqa: F401

__all__ = ["sscg", "Solver", "SscgError", "load_library"]
