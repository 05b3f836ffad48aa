"""Python face of the CPM library: the C ABI's calls with torch tensors.

Every call here only marshals arguments (device pointers of CUDA tensors, the
current torch stream) into the sm_103a library; all arithmetic of the method
runs in the library's kernels.  Names follow include/cpm.h.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

CURVE_POINT, CURVE_CIRCLE = 1, 2


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[ctypes.c_void_p]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor required")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor required")
    return ctypes.c_void_p(t.data_ptr())


def _layout(t: torch.Tensor, N: int):
    """(nrhs, ld) of an [N] or [N, nrhs] tensor."""
    if t.dim() == 1:
        if t.shape[0] != N:
            raise ValueError(f"expected length {N}, got {t.shape[0]}")
        return 1, 1
    if t.dim() == 2 and t.shape[0] == N:
        return int(t.shape[1]), int(t.stride(0))
    raise ValueError(f"expected [N] or [N, nrhs] with N={N}, got {tuple(t.shape)}")


@dataclasses.dataclass
class SolveStats:
    iterations: int
    refinements: int
    restarts: int
    relres: float
    status: str
    fp64_iterations: int = 0
    relres_floor: float = 0.0


def shape_desc(shape) -> tuple:
    """Build the C descriptor from any object with the shape fields (kind, dim, R,
    rt, a, c, amp, width, seed_point)."""
    d = L.ShapeDesc()
    d.kind, d.dim = int(shape.kind), int(shape.dim)
    d.R, d.rt = float(shape.R), float(getattr(shape, "rt", 0.0))
    a = getattr(shape, "a", None)
    keep = []
    d.K = 0 if a is None else int(len(a))
    d.amp, d.width = float(getattr(shape, "amp", 0.0)), float(getattr(shape, "width", 1.0))
    if d.K:
        aa = np.ascontiguousarray(a, dtype=np.float64)
        cc = np.ascontiguousarray(shape.c, dtype=np.float64).reshape(-1)
        keep += [aa, cc]
        d.a = aa.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.c = cc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    sp = list(shape.seed_point) + [0.0] * 3
    for k in range(3):
        d.seed[k] = float(sp[k])
    return d, keep


def curve_descs(curves: Sequence, n_samples: Optional[Sequence[int]] = None):
    arr = (L.CurveDesc * max(1, len(curves)))()
    for i, cv in enumerate(curves):
        c = arr[i]
        c.kind, c.bc = int(cv.kind), int(cv.bc)
        for k in range(3):
            c.p[k] = float(cv.p[k]); c.nu[k] = float(cv.nu[k]); c.ref[k] = float(cv.ref[k])
        c.rad = float(cv.rad)
        c.two_sided = int(bool(getattr(cv, "two_sided", False)))
        c.n_samples = int(n_samples[i]) if n_samples is not None else 1
        c.bc_minus = int(getattr(cv, "bc_minus", 0) or 0)
        c.projected = int(bool(getattr(cv, "projected", False)))
    return arr


def measure_fma_peak() -> dict:
    """cpm_measure_fma_peak: the device's FP32 (scalar and packed-pair) and FP64
    FMA throughput in TFLOP/s."""
    lib = L.load()
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    L.check(lib.cpm_measure_fma_peak(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "cpm_measure_fma_peak")
    return {"fp32_fma_tflops": a.value, "fp32_pair_fma_tflops": b.value, "fp64_fma_tflops": c.value}


class Band:
    """A band Omega(S) with its operator (one cpm_ctx)."""

    def __init__(self, shape, h: float, r_band: float = -1.0, p: int = 3):
        self._lib = L.load()
        self._h = ctypes.c_void_p()
        d, keep = shape_desc(shape)
        L.check(self._lib.cpm_band_build(ctypes.byref(d), float(h), int(p), float(r_band), _stream(),
                                         ctypes.byref(self._h)), "cpm_band_build")
        self.h = float(h)
        self.p = int(p)
        self.dim = int(shape.dim)
        self._sizes()
        self.n_samples = []

    def _sizes(self):
        ns, nc, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rb = ctypes.c_double()
        L.check(self._lib.cpm_band_info(self._h, ctypes.byref(ns), ctypes.byref(nc), ctypes.byref(rb),
                                        ctypes.byref(nb)), "cpm_band_info")
        self.NS, self.NC, self.r_band, self.n_bricks = ns.value, nc.value, rb.value, nb.value

    @property
    def N(self) -> int:
        return self.NS + self.NC

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize()
            self._lib.cpm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- band / boundary ------------------------------------------------------
    def export_band(self):
        ijk = torch.empty((self.NS, 3), dtype=torch.int32, device="cuda")
        cp = torch.empty((self.NS, 3), dtype=torch.float64, device="cuda")
        L.check(self._lib.cpm_export_band(self._h, _ptr(ijk), _ptr(cp), _stream()), "cpm_export_band")
        return ijk, cp

    def set_boundary(self, curves: Sequence, n_samples: Optional[Sequence[int]] = None):
        arr = curve_descs(curves, n_samples)
        L.check(self._lib.cpm_set_boundary(self._h, arr, len(curves)), "cpm_set_boundary")
        self.n_samples = list(n_samples) if n_samples is not None else [1] * len(curves)
        self.curves = list(curves)
        self._sizes()
        self._reserved = (1, L.RESERVE_FP64 | L.RESERVE_FP32_IR)  # what cpm_set_boundary reserves
        return self

    def reserve(self, ld: int, fp32_ir: bool = True):
        """cpm_reserve: workspaces for leading dimension `ld` (products, and the
        FP64 and, with fp32_ir, FP32+refinement solves).  The calls below reserve
        on demand; calling this first keeps the allocation out of timed work."""
        flags = L.RESERVE_FP64 | (L.RESERVE_FP32_IR if fp32_ir else 0)
        ld0, f0 = getattr(self, "_reserved", (0, 0))
        if ld <= ld0 and (f0 | flags) == f0:
            return self
        L.check(self._lib.cpm_reserve(self._h, int(max(ld, ld0)), int(f0 | flags)), "cpm_reserve")
        self._reserved = (max(ld, ld0), f0 | flags)
        return self

    def export_boundary(self):
        n = max(self.NC, 1)
        twin = torch.empty(n, dtype=torch.int64, device="cuda")
        curve = torch.empty(n, dtype=torch.int32, device="cuda")
        cpc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        side = torch.empty(n, dtype=torch.int32, device="cuda")
        param = torch.empty(n, dtype=torch.float64, device="cuda")
        btype = torch.empty(n, dtype=torch.int32, device="cuda")
        L.check(self._lib.cpm_export_boundary(self._h, _ptr(twin), _ptr(curve), _ptr(cpc), _ptr(side), _ptr(param),
                                              _ptr(btype), _stream()), "cpm_export_boundary")
        k = self.NC
        return {"twin": twin[:k], "curve": curve[:k], "cpc": cpc[:k], "side": side[:k], "param": param[:k],
                "type": btype[:k]}

    def profile(self, enable: bool):
        """Start (True) or stop (False) the library's product timing; stopping
        returns {apply_ms, applies, launches, row_rhs}."""
        ms, calls, launches, rr = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        L.check(self._lib.cpm_profile(self._h, 1 if enable else 0, ctypes.byref(ms), ctypes.byref(calls),
                                      ctypes.byref(launches), ctypes.byref(rr)), "cpm_profile")
        return None if enable else {"apply_ms": ms.value, "applies": calls.value, "launches": launches.value,
                                    "row_rhs": rr.value}

    def autotune(self, nrhs: int, dtype=torch.float32) -> dict:
        """cpm_autotune: time the launch-shape candidates for nrhs columns of
        dtype on this band and keep the fastest; returns the choices."""
        prec = {torch.float64: L.PREC_FP64, torch.float32: L.PREC_FP32}[dtype]
        self.reserve(nrhs, fp32_ir=(dtype == torch.float32))
        info = L.TuneInfo()
        L.check(self._lib.cpm_autotune(self._h, int(nrhs), int(nrhs), prec, ctypes.byref(info), _stream()),
                "cpm_autotune")
        return {k: getattr(info, k) for k, _ in L.TuneInfo._fields_}

    def set_tune(self, nrhs: int, dtype=torch.float32, **shapes) -> "Band":
        """cpm_set_tune: fix the launch shapes (the keys of autotune's report;
        a missing key or 0 is the default)."""
        prec = L.PREC_FP32 if dtype == torch.float32 else L.PREC_FP64
        info = L.TuneInfo()
        for k, v in shapes.items():
            setattr(info, k, v)
        L.check(self._lib.cpm_set_tune(self._h, int(nrhs), prec, ctypes.byref(info)), "cpm_set_tune")
        return self

    def diagnostics(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        L.check(self._lib.cpm_diagnostics(self._h, ctypes.byref(a), ctypes.byref(b)), "cpm_diagnostics")
        return {"noflip_twin": a.value, "special_rows": b.value}

    # -- operator -------------------------------------------------------------
    def rhs(self, s: Optional[torch.Tensor] = None, g: Optional[torch.Tensor] = None,
            samples: Optional[torch.Tensor] = None, nrhs: int = 1) -> torch.Tensor:
        shape = (self.N,) if nrhs == 1 else (self.N, nrhs)
        f = torch.empty(shape, dtype=torch.float64, device="cuda")
        ld = 1 if nrhs == 1 else nrhs
        L.check(self._lib.cpm_rhs(self._h, _ptr(s), _ptr(g), _ptr(samples), _ptr(f), nrhs, ld, _stream()), "cpm_rhs")
        return f

    def apply(self, m: float, n: float, u: torch.Tensor, out: Optional[torch.Tensor] = None,
              transpose: bool = False) -> torch.Tensor:
        nrhs, ld = _layout(u, self.N)
        prec = {torch.float64: L.PREC_FP64, torch.float32: L.PREC_FP32}[u.dtype]
        v = torch.empty_like(u) if out is None else out
        self.reserve(ld, fp32_ir=False)
        fn = self._lib.cpm_apply_transpose if transpose else self._lib.cpm_apply
        L.check(fn(self._h, float(m), float(n), prec, _ptr(u), _ptr(v), nrhs, ld, _stream()),
                "cpm_apply_transpose" if transpose else "cpm_apply")
        return v

    def apply_noalloc(self, m: float, n: float, u: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        """cpm_apply_noalloc: the product with the library's fixed intermediate
        array (no allocation inside the call; `out` is the caller's)."""
        nrhs, ld = _layout(u, self.N)
        prec = {torch.float64: L.PREC_FP64, torch.float32: L.PREC_FP32}[u.dtype]
        L.check(self._lib.cpm_apply_noalloc(self._h, float(m), float(n), prec, _ptr(u), _ptr(out), nrhs, ld,
                                            _stream()), "cpm_apply_noalloc")
        return out

    def extend(self, u: torch.Tensor) -> torch.Tensor:
        nrhs, ld = _layout(u, self.N)
        a = torch.empty((self.NS,) if nrhs == 1 else (self.NS, nrhs), dtype=torch.float64, device="cuda")
        self.reserve(max(ld, nrhs), fp32_ir=False)
        L.check(self._lib.cpm_extend(self._h, _ptr(u), _ptr(a), nrhs, ld, _stream()), "cpm_extend")
        return a

    def surface_gradient(self, u: torch.Tensor, normalize: bool = False) -> torch.Tensor:
        """cpm_surface_gradient: [N, 3] central-difference gradient of the CP
        extension of u ([N]); normalize gives X = -g / |g|."""
        _layout(u, self.N)
        X = torch.empty((self.N, 3), dtype=torch.float64, device="cuda")
        L.check(self._lib.cpm_surface_gradient(self._h, _ptr(u), _ptr(X), 1 if normalize else 0, _stream()),
                "cpm_surface_gradient")
        return X

    def surface_divergence(self, X: torch.Tensor) -> torch.Tensor:
        """cpm_surface_divergence: [N_S] divergence of the CP extension of X ([N, 3])."""
        if tuple(X.shape) != (self.N, 3):
            raise ValueError(f"expected [{self.N}, 3]")
        b = torch.empty(self.NS, dtype=torch.float64, device="cuda")
        L.check(self._lib.cpm_surface_divergence(self._h, _ptr(X), _ptr(b), _stream()), "cpm_surface_divergence")
        return b

    def solve(self, m: float, n: float, f: torch.Tensor, x0: Optional[torch.Tensor] = None, tol: float = 1e-10,
              maxit: int = 20000, mode: str = "fp64", inner_tol: float = 0.0, max_refine: int = 0,
              check_every: int = 16, adjoint: bool = False, raise_on_error: bool = True, norm: str = "plain",
              inner_maxit: int = 0):
        nrhs, ld = _layout(f, self.N)
        self.reserve(ld, fp32_ir=(mode != "fp64"))
        x = torch.zeros_like(f) if x0 is None else x0.clone()
        o = L.SolveOpts(tol, maxit, L.SOLVE_FP64 if mode == "fp64" else L.SOLVE_FP32_IR, inner_tol, max_refine,
                        check_every, L.NORM_SCALED if norm == "scaled" else L.NORM_PLAIN, inner_maxit)
        st = L.SolveStats()
        fn = self._lib.cpm_solve_adjoint if adjoint else self._lib.cpm_solve
        rc = fn(self._h, float(m), float(n), _ptr(f), _ptr(x), nrhs, ld, ctypes.byref(o), ctypes.byref(st),
                _stream())
        stats = SolveStats(st.iterations, st.refinements, st.restarts, st.relres, L.STATUS.get(rc, str(rc)),
                           st.fp64_iterations, st.relres_floor)
        if raise_on_error:
            L.check(rc, "cpm_solve_adjoint" if adjoint else "cpm_solve")
        return x, stats

    def boundary_grad(self, lam: torch.Tensor) -> torch.Tensor:
        nrhs, ld = _layout(lam, self.N)
        tot = 0
        for cv, ns in zip(self.curves, self.n_samples):
            tot += ns * (2 if getattr(cv, "two_sided", False) else 1)
        out = torch.zeros((tot,) if nrhs == 1 else (tot, nrhs), dtype=torch.float64, device="cuda")
        L.check(self._lib.cpm_boundary_grad(self._h, _ptr(lam), _ptr(out), nrhs, ld, _stream()), "cpm_boundary_grad")
        return out
