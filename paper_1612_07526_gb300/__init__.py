"""GB300 (sm_103a) divide-and-conquer eigensolver for symmetric tridiagonal matrices.

The merge step of Cuppen's method -- deflation, FP64 secular roots, the Loewner
recomputation of z and the eigenvector product -- runs in hand-written CUDA kernels
behind the C ABI of include/tdc.h (libtdc.so); this package is the thin Python
binding.  Import ``paper_1612_07526_gb300.api`` for the PyTorch wrappers.
"""
from . import _lib  # noqa: F401

__all__ = ["_lib"]
