"""ctypes declarations of the C ABI in include/cpm.h.

The shared library is built in-tree (paper_2305_04711_gb300/libcpm_gb300.so) by
`build.py`; importing this module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcpm_gb300.so")

CPM_OK = 0
STATUS = {0: "CPM_OK", 1: "CPM_ERR_ARG", 2: "CPM_ERR_OOM", 3: "CPM_ERR_CUDA", 4: "CPM_ERR_CAPACITY",
          5: "CPM_ERR_CP_FAILED", 6: "CPM_ERR_OVERLAP", 7: "CPM_ERR_BREAKDOWN", 8: "CPM_ERR_NOT_CONVERGED",
          9: "CPM_ERR_TIMEOUT", 10: "CPM_ERR_STATE"}
PREC_FP64, PREC_FP32 = 0, 1
SOLVE_FP64, SOLVE_FP32_IR = 0, 1
NORM_PLAIN, NORM_SCALED = 0, 1
RESERVE_FP64, RESERVE_FP32_IR = 1, 2

# every entry point that include/cpm.h declares
EXPORTS = ["cpm_band_build", "cpm_band_info", "cpm_export_band", "cpm_set_boundary", "cpm_export_boundary",
           "cpm_rhs", "cpm_apply", "cpm_apply_transpose", "cpm_extend", "cpm_solve", "cpm_solve_adjoint",
           "cpm_boundary_grad", "cpm_destroy", "cpm_status_str", "cpm_diagnostics", "cpm_profile",
           "cpm_apply_noalloc", "cpm_apply_noalloc_max_bytes", "cpm_surface_gradient", "cpm_surface_divergence",
           "cpm_reserve", "cpm_autotune", "cpm_set_tune", "cpm_measure_fma_peak"]


class ShapeDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dim", ctypes.c_int), ("R", ctypes.c_double), ("rt", ctypes.c_double),
                ("K", ctypes.c_int), ("amp", ctypes.c_double), ("width", ctypes.c_double),
                ("a", ctypes.POINTER(ctypes.c_double)), ("c", ctypes.POINTER(ctypes.c_double)),
                ("seed", ctypes.c_double * 3)]


class CurveDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("bc", ctypes.c_int), ("p", ctypes.c_double * 3),
                ("nu", ctypes.c_double * 3), ("rad", ctypes.c_double), ("ref", ctypes.c_double * 3),
                ("two_sided", ctypes.c_int), ("n_samples", ctypes.c_int), ("bc_minus", ctypes.c_int),
                ("projected", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("mode", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int), ("check_every", ctypes.c_int),
                ("norm", ctypes.c_int), ("inner_maxit", ctypes.c_int)]


class TuneInfo(ctypes.Structure):
    _fields_ = [("cells_xh", ctypes.c_int), ("cells_blocks_per_sm", ctypes.c_int),
                ("combine_warps_per_sm", ctypes.c_int), ("vec_blocks_per_sm", ctypes.c_int),
                ("single_mode", ctypes.c_int),
                ("product_ms", ctypes.c_double), ("product_ms_default", ctypes.c_double),
                ("vector_ms", ctypes.c_double)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int), ("restarts", ctypes.c_int),
                ("relres", ctypes.c_double), ("status", ctypes.c_int), ("fp64_iterations", ctypes.c_int),
                ("relres_floor", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (no fallback: a missing library is an error)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run build.py / __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P, d, i, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
    pi64 = ctypes.POINTER(i64)
    L.cpm_band_build.argtypes = [ctypes.POINTER(ShapeDesc), d, i, d, P, ctypes.POINTER(P)]
    L.cpm_band_info.argtypes = [P, pi64, pi64, ctypes.POINTER(d), pi64]
    L.cpm_export_band.argtypes = [P, P, P, P]
    L.cpm_set_boundary.argtypes = [P, ctypes.POINTER(CurveDesc), i]
    L.cpm_export_boundary.argtypes = [P, P, P, P, P, P, P, P]
    L.cpm_rhs.argtypes = [P, P, P, P, P, i, i64, P]
    L.cpm_apply.argtypes = [P, d, d, i, P, P, i, i64, P]
    L.cpm_apply_transpose.argtypes = [P, d, d, i, P, P, i, i64, P]
    L.cpm_apply_noalloc.argtypes = [P, d, d, i, P, P, i, i64, P]
    L.cpm_apply_noalloc_max_bytes.argtypes = []
    L.cpm_apply_noalloc_max_bytes.restype = ctypes.c_size_t
    L.cpm_extend.argtypes = [P, P, P, i, i64, P]
    L.cpm_surface_gradient.argtypes = [P, P, P, i, P]
    L.cpm_surface_divergence.argtypes = [P, P, P, P]
    L.cpm_solve.argtypes = [P, d, d, P, P, i, i64, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), P]
    L.cpm_solve_adjoint.argtypes = [P, d, d, P, P, i, i64, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), P]
    L.cpm_boundary_grad.argtypes = [P, P, P, i, i64, P]
    L.cpm_destroy.argtypes = [P]
    L.cpm_destroy.restype = None
    L.cpm_status_str.argtypes = [i]
    L.cpm_status_str.restype = ctypes.c_char_p
    L.cpm_diagnostics.argtypes = [P, pi64, pi64]
    L.cpm_profile.argtypes = [P, i, ctypes.POINTER(d), pi64, pi64, pi64]
    L.cpm_reserve.argtypes = [P, i64, i]
    L.cpm_autotune.argtypes = [P, i, i64, i, ctypes.POINTER(TuneInfo), P]
    L.cpm_set_tune.argtypes = [P, i, i, ctypes.POINTER(TuneInfo)]
    L.cpm_measure_fma_peak.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3
    for name in EXPORTS:
        if name not in ("cpm_destroy", "cpm_status_str", "cpm_apply_noalloc_max_bytes"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class CpmError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code
        self.status = STATUS.get(code, str(code))


def check(code: int, where: str) -> None:
    if code != CPM_OK:
        raise CpmError(code, where)
