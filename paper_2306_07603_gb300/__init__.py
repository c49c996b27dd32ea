"""GB300 (sm_103a) IFDLBM library: power-law fluid in a lid-driven trapezoidal cavity.

``capi`` is the ctypes binding of include/ifdlbm.h; ``solver.Solver`` is a
thin owner of one handle. All computation happens in libifdlbm.so.
"""
from . import capi  # noqa: F401

__all__ = ["capi"]
