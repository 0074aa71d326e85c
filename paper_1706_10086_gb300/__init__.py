"""GB300 (sm_103a) double-precision GEMM library: C = alpha*A*B + beta*C.

The compute path is ``libalp.so`` (CUDA kernels behind the C-ABI of
``include/alp.h``); :mod:`.alp` is its ctypes binding.  :mod:`.inputs` holds
the seeded synthetic input generators.
"""
from . import alp  # noqa: F401
from .alp import *  # noqa: F401,F403


def build(verbose: bool = False) -> str:
    """Compiles ``libalp.so`` for sm_103a (no-op when up to date)."""
    from ._build import build as _b
    return _b(verbose=verbose)
