"""GB300-native (sm_103a) closest point method with interior boundary conditions.

The hot path -- the band, the crossing-test stencils, the fused matrix-free
operator A = mI + n[diag L + (L - diag L)E] and the Krylov solves -- runs in the
CUDA library libcpm_gb300.so behind the C ABI of include/cpm.h.  This package is
the thin Python binding (torch tensors for device memory and streams).
"""
from ._lib import CpmError, load  # noqa: F401

__all__ = ["Band", "CpmError", "load"]


def __getattr__(name):
    if name == "Band":
        from .cpm import Band
        return Band
    raise AttributeError(name)
