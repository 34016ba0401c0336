"""GB300 (sm_103a) row-sampling SGS-preconditioned PCG for overdetermined least squares.

Chen & Wu, "A Preconditioner based on Non-uniform Row Sampling for Linear Least Squares
Problems" (arXiv:1806.02968), Alg. 1-3.  All computation runs in the CUDA library
``liblsq.so`` (C ABI in ``include/lsq.h``); this package only marshals arguments.
"""
from .build import build  # noqa: F401

__all__ = ["build"]
