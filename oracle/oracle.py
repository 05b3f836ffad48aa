"""Python face of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this module.  It wraps the plain-C FP64 oracle (cpm_oracle.c) with ctypes and
uses scipy for the sparse algebra a reader can check by eye:

  * M = diag(L) + (L - diag L) E        (Sec. 5.3)
  * A = m I + n M on PDE rows; BC rows   (Sec. 5.4; BC rows per Sec. 4.3)
  * direct solves with scipy's SuperLU    (the paper uses Eigen's SparseLU, Sec. 6.1)
  * the adjoint through A^T               (a CSR transpose)
  * Dirichlet data: f_alpha = c_alpha g(cp_C(x_alpha)) with c = 1 (1st order)
    or 2 (2nd order), g taken from the side opposite cp_S(x_alpha) (Sec. 4.3);
    zero-Neumann rows carry no data (c = 0)

It shares no code with the CUDA library and never imports it.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

sys.path.insert(0, os.path.dirname(_HERE))
import cpm_inputs as ci  # noqa: E402


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dim", ctypes.c_int), ("R", ctypes.c_double),
                ("rt", ctypes.c_double), ("K", ctypes.c_int), ("amp", ctypes.c_double),
                ("width", ctypes.c_double), ("a", ctypes.POINTER(ctypes.c_double)),
                ("c", ctypes.POINTER(ctypes.c_double)), ("seed", ctypes.c_double * 3)]


class _Curve(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("bc", ctypes.c_int), ("p", ctypes.c_double * 3),
                ("nu", ctypes.c_double * 3), ("rad", ctypes.c_double), ("ref", ctypes.c_double * 3),
                ("two_sided", ctypes.c_int), ("bc_minus", ctypes.c_int), ("projected", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        L.orc_build.argtypes = [ctypes.POINTER(_Shape), d, i32, d, ctypes.POINTER(P)]
        L.orc_destroy.argtypes = [P]
        L.orc_ns.argtypes = [P]; L.orc_ns.restype = i64
        L.orc_nc.argtypes = [P]; L.orc_nc.restype = i64
        L.orc_rband.argtypes = [P]; L.orc_rband.restype = d
        L.orc_tube_radius.argtypes = [i32, i32, d]; L.orc_tube_radius.restype = d
        L.orc_export_band.argtypes = [P, P, P]
        L.orc_lookup.argtypes = [P, i32, i32, i32]; L.orc_lookup.restype = i64
        L.orc_set_curves.argtypes = [P, ctypes.POINTER(_Curve), i32]
        L.orc_export_bc.argtypes = [P, P, P, P, P, P]
        L.orc_export_near.argtypes = [P, P, P]
        L.orc_assemble.argtypes = [P]
        L.orc_noflip_twin.argtypes = [P]; L.orc_noflip_twin.restype = i64
        L.orc_csr_dims.argtypes = [P, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.orc_csr_export.argtypes = [P, i32, P, P, P]
        L.orc_apply.argtypes = [P, d, d, P, P, P]
        L.orc_extend.argtypes = [P, P, P]
        L.orc_bicgstab.argtypes = [P, d, d, P, P, d, i32, ctypes.POINTER(i32), ctypes.POINTER(d)]
        L.orc_band_bruteforce.argtypes = [ctypes.POINTER(_Shape), d, i32, d, P, P, P, i64]
        L.orc_band_bruteforce.restype = i64
        L.orc_cp.argtypes = [ctypes.POINTER(_Shape), P, P]
        L.orc_bumpy_phi.argtypes = [ctypes.POINTER(_Shape), P, P, P, P]
        L.orc_cpc.argtypes = [ctypes.POINTER(_Curve), P, P]
        L.orc_crossing_vector.argtypes = [P, i32, i64, P]
        L.orc_bary_weights.argtypes = [i32, d, P]
        L.orc_num_threads.restype = i32
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_shape(sh: ci.Shape):
    """Convert a shape description; returns (struct, keep-alive arrays)."""
    keep = []
    s = _Shape()
    s.kind, s.dim, s.R, s.rt = sh.kind, sh.dim, sh.R, sh.rt
    s.K, s.amp, s.width = sh.K, sh.amp, sh.width
    if sh.K:
        a = np.ascontiguousarray(sh.a, dtype=np.float64)
        c = np.ascontiguousarray(sh.c, dtype=np.float64).reshape(-1)
        keep += [a, c]
        s.a = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s.c = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for k in range(3):
        s.seed[k] = float(sh.seed_point[k]) if k < len(sh.seed_point) else 0.0
    return s, keep


def make_curves(curves: Sequence[ci.Curve]):
    arr = (_Curve * max(1, len(curves)))()
    for i, cv in enumerate(curves):
        c = arr[i]
        c.kind, c.bc = cv.kind, cv.bc
        for k in range(3):
            c.p[k] = float(cv.p[k]); c.nu[k] = float(cv.nu[k]); c.ref[k] = float(cv.ref[k])
        c.rad = cv.rad
        c.two_sided = int(cv.two_sided)
        c.bc_minus = int(getattr(cv, "bc_minus", 0) or 0)
        c.projected = int(bool(getattr(cv, "projected", False)))
    return arr


def tube_radius(dim: int, h: float, p: int = 3) -> float:
    return lib().orc_tube_radius(dim, p, h)


def bary_weights(t: float, p: int = 3) -> np.ndarray:
    w = np.zeros(4)
    lib().orc_bary_weights(p, t, _ptr(w))
    return w[:p + 1]


def closest_point(sh: ci.Shape, x) -> np.ndarray:
    s, keep = make_shape(sh)
    xx = np.zeros(3); xx[:len(x)] = x
    out = np.zeros(3)
    if lib().orc_cp(ctypes.byref(s), _ptr(xx), _ptr(out)):
        raise RuntimeError("closest point failed")
    return out


def bumpy_phi(sh: ci.Shape, x):
    s, keep = make_shape(sh)
    xx = np.asarray(x, dtype=np.float64)
    phi = np.zeros(1); g = np.zeros(3); H = np.zeros(9)
    lib().orc_bumpy_phi(ctypes.byref(s), _ptr(xx), _ptr(phi), _ptr(g), _ptr(H))
    return phi[0], g, H.reshape(3, 3)


def curve_cp(cv: ci.Curve, x) -> np.ndarray:
    arr = make_curves([cv])
    xx = np.zeros(3); xx[:len(x)] = x
    out = np.zeros(3)
    lib().orc_cpc(arr, _ptr(xx), _ptr(out))
    return out


def band_bruteforce(sh: ci.Shape, h: float, lo, hi, rband: float = -1.0, p: int = 3) -> np.ndarray:
    s, keep = make_shape(sh)
    lo = np.array(list(lo) + [0] * (3 - len(lo)), dtype=np.int32)
    hi = np.array(list(hi) + [0] * (3 - len(hi)), dtype=np.int32)
    n = lib().orc_band_bruteforce(ctypes.byref(s), h, p, rband, _ptr(lo), _ptr(hi), None, 0)
    out = np.zeros((max(n, 1), 3), dtype=np.int32)
    lib().orc_band_bruteforce(ctypes.byref(s), h, p, rband, _ptr(lo), _ptr(hi), _ptr(out), n)
    return out[:n]


class OracleError(RuntimeError):
    pass


_ERRS = {1: "ARG", 2: "OOM", 3: "CP_FAILED", 4: "OVERLAP", 5: "STATE", 6: "BREAKDOWN", 7: "NOT_CONVERGED"}


def _check(rc):
    if rc:
        raise OracleError(_ERRS.get(rc, str(rc)))


class Oracle:
    """The discrete CPM of the paper on one band; FP64 throughout."""

    def __init__(self, shape: ci.Shape, h: float, rband: float = -1.0, p: int = 3):
        self.shape, self.h, self.p = shape, h, p
        self.dim = shape.dim
        s, self._keep = make_shape(shape)
        self._h = ctypes.c_void_p()
        _check(lib().orc_build(ctypes.byref(s), h, p, rband, ctypes.byref(self._h)))
        self.NS = lib().orc_ns(self._h)
        self.NC = 0
        self.rband = lib().orc_rband(self._h)
        self.ijk = np.zeros((self.NS, 3), dtype=np.int32)
        self.cp = np.zeros((self.NS, 3), dtype=np.float64)
        lib().orc_export_band(self._h, _ptr(self.ijk), _ptr(self.cp))
        self.curves: List[ci.Curve] = []
        self._assembled = False

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_destroy(h)
            self._h = None

    @property
    def N(self) -> int:
        return self.NS + self.NC

    def x(self) -> np.ndarray:
        """Grid node coordinates of the PDE DOFs."""
        out = self.ijk.astype(np.float64) * self.h
        if self.dim == 2:
            out[:, 2] = 0.0
        return out

    def set_curves(self, curves: Sequence[ci.Curve]):
        self.curves = list(curves)
        arr = make_curves(self.curves)
        _check(lib().orc_set_curves(self._h, arr, len(self.curves)))
        self.NC = lib().orc_nc(self._h)
        nc = max(self.NC, 1)
        self.twin = np.zeros(nc, dtype=np.int64)
        self.bc_curve = np.zeros(nc, dtype=np.int32)
        self.cpc = np.zeros((nc, 3), dtype=np.float64)
        self.bc_side = np.zeros(nc, dtype=np.int32)
        self.bc_type = np.zeros(nc, dtype=np.int32)
        lib().orc_export_bc(self._h, _ptr(self.twin), _ptr(self.bc_curve), _ptr(self.cpc), _ptr(self.bc_side),
                            _ptr(self.bc_type))
        self.twin, self.bc_curve = self.twin[:self.NC], self.bc_curve[:self.NC]
        self.cpc, self.bc_side = self.cpc[:self.NC], self.bc_side[:self.NC]
        self.bc_type = self.bc_type[:self.NC]
        self.near_c = np.zeros(self.NS, dtype=np.int32)
        self.bc_of = np.zeros(self.NS, dtype=np.int64)
        lib().orc_export_near(self._h, _ptr(self.near_c), _ptr(self.bc_of))
        _check(lib().orc_assemble(self._h))
        self._assembled = True
        self.noflip_twin = lib().orc_noflip_twin(self._h)
        self.E = self._csr(0, self.NS)
        self.Loff = self._csr(1, self.NS)
        self.B = self._csr(2, self.NC)
        return self

    def _csr(self, which, nrows):
        nr, nnz = ctypes.c_int64(), ctypes.c_int64()
        lib().orc_csr_dims(self._h, which, ctypes.byref(nr), ctypes.byref(nnz))
        ptr = np.zeros(nr.value + 1, dtype=np.int64)
        col = np.zeros(max(nnz.value, 1), dtype=np.int64)
        val = np.zeros(max(nnz.value, 1), dtype=np.float64)
        lib().orc_csr_export(self._h, which, _ptr(ptr), _ptr(col), _ptr(val))
        return sp.csr_matrix((val[:nnz.value], col[:nnz.value], ptr), shape=(nrows, self.N))

    # -- operators -------------------------------------------------------
    def diagL(self) -> float:
        return -2.0 * self.dim / (self.h * self.h)

    def M(self) -> sp.csr_matrix:
        """PDE rows of M = diag(L) + (L - diag L) E  (N_S x N).  E's BC rows are
        the identity, so (L - diag L) E = Loff[:, :NS] E + Loff[:, NS:]."""
        NS = self.NS
        D = sp.eye(NS, self.N, format="csr") * self.diagL()
        Efull = sp.vstack([self.E, sp.hstack([sp.csr_matrix((self.NC, NS)), sp.eye(self.NC)])]).tocsr()
        return (D + self.Loff @ Efull).tocsr()

    def A(self, m: float, n: float) -> sp.csr_matrix:
        NS = self.NS
        top = (m * sp.eye(NS, self.N, format="csr") + n * self.M()).tocsr()
        return sp.vstack([top, self.B]).tocsr()

    def apply(self, m: float, n: float, u: np.ndarray) -> np.ndarray:
        """The paper's four-step matrix-free product, in C (OpenMP)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        v = np.zeros(self.N)
        work = np.zeros(self.N)
        _check(lib().orc_apply(self._h, m, n, _ptr(u), _ptr(v), _ptr(work)))
        return v

    def extend(self, u: np.ndarray) -> np.ndarray:
        """(E u) on the PDE rows: side-correct surface values at cp_S(x_i)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        a = np.zeros(self.NS)
        _check(lib().orc_extend(self._h, _ptr(u), _ptr(a)))
        return a

    def fd_neighbours(self) -> np.ndarray:
        """[NS, 6] FD neighbour columns of each PDE row in the order x-, x+, y-,
        y+, z-, z+ as the Laplacian rows use them (Eq. 2 with the flips of
        Eq. 11): the PDE DOF at x_i +- h e_d, or its BC twin where the row's
        stencil was flipped to it; -1 where the node is not in the band."""
        if getattr(self, "_nb", None) is not None:
            return self._nb
        ijk = self.ijk.astype(np.int64)
        lo = ijk.min(axis=0) - 2
        ext = ijk.max(axis=0) - lo + 3
        def key(p):
            q = p - lo
            return (q[:, 2] * ext[1] + q[:, 1]) * ext[0] + q[:, 0]
        keys = key(ijk)
        order = np.argsort(keys)
        skeys = keys[order]
        # flipped FD entries: Loff entries (i, alpha >= NS) replace node twin[alpha]
        Lo = self.Loff.tocoo()
        sel = Lo.col >= self.NS
        flip = {(int(i), int(self.twin[c - self.NS])): int(c) for i, c in zip(Lo.row[sel], Lo.col[sel])}
        out = -np.ones((self.NS, 6), dtype=np.int64)
        for d in range(self.dim):
            for sg, slot in ((-1, 2 * d), (1, 2 * d + 1)):
                q = ijk.copy()
                q[:, d] += sg
                kq = key(q)
                pos = np.clip(np.searchsorted(skeys, kq), 0, len(skeys) - 1)
                found = skeys[pos] == kq
                out[:, slot] = np.where(found, order[pos], -1)
        for (i, j), c in flip.items():
            row = out[i]
            row[row == j] = c
        self._nb = out
        return out

    def _central(self, at: np.ndarray, a: np.ndarray, nb: np.ndarray, d: int) -> np.ndarray:
        vp = np.where(nb[:, 2 * d + 1] >= 0, at[np.maximum(nb[:, 2 * d + 1], 0)], a)
        vm = np.where(nb[:, 2 * d] >= 0, at[np.maximum(nb[:, 2 * d], 0)], a)
        return (vp - vm) / (2.0 * self.h)

    def surface_gradient(self, u: np.ndarray, normalize: bool = False) -> np.ndarray:
        """Central differences of the CP extension (Sec. 7.2, step 2): at PDE row
        i, g_d = (a(n+) - a(n-)) / 2h over its FD neighbours, with a = E u on PDE
        DOFs and u itself on BC DOFs; a missing neighbour takes a_i.  normalize:
        X = -g / |g| (0 where g = 0).  BC DOFs take their twin node's value.
        Returns [N, 3]."""
        u = np.asarray(u, dtype=np.float64)
        a = self.extend(u)
        at = np.concatenate([a, u[self.NS:]])
        nb = self.fd_neighbours()
        g = np.zeros((self.NS, 3))
        for d in range(self.dim):
            g[:, d] = self._central(at, a, nb, d)
        if normalize:
            nrm = np.sqrt(np.sum(g * g, axis=1))
            g = np.where(nrm[:, None] > 0, -g / np.where(nrm > 0, nrm, 1.0)[:, None], 0.0)
        return np.concatenate([g, g[self.twin]]) if self.NC else g

    def surface_divergence(self, X: np.ndarray) -> np.ndarray:
        """Central-difference divergence of the CP extension of the field X
        ([N, 3]) at the PDE rows (the right-hand side of Sec. 7.2, step 3)."""
        X = np.asarray(X, dtype=np.float64)
        nb = self.fd_neighbours()
        b = np.zeros(self.NS)
        for d in range(self.dim):
            a = self.extend(np.ascontiguousarray(X[:, d]))
            at = np.concatenate([a, X[self.NS:, d]])
            b += self._central(at, a, nb, d)
        return b

    def heat_cn(self, u0: np.ndarray, dt: float, nsteps: int, g_bc=None) -> np.ndarray:
        """Crank-Nicolson steps of u_t = Delta_S u (the time stepping of the
        convergence studies, Sec. 6.2): (I - dt/2 M) u^{k+1} = (I + dt/2 M) u^k on
        the PDE rows, while the BC rows of step k+1 are the BC equations with the
        data of time t_{k+1}: right-hand side c_alpha g_alpha(t_{k+1}) (c = 1, 2
        for first- and second-order Dirichlet rows, 0 for zero-Neumann rows).
        g_bc: per BC DOF values, an array held fixed in time or a function of t;
        None means zero data."""
        lu = spla.splu(self.A(1.0, -0.5 * dt).tocsc())
        Ap = self.A(1.0, 0.5 * dt)
        cb = self.bc_scale() if self.NC else np.zeros(0)
        u = np.asarray(u0, dtype=np.float64).copy()
        for k in range(nsteps):
            rhs = Ap @ u
            if callable(g_bc):
                g = np.asarray(g_bc((k + 1) * dt), dtype=np.float64)
            else:
                g = np.zeros(self.NC) if g_bc is None else np.asarray(g_bc, dtype=np.float64)
            rhs[self.NS:] = cb * g
            u = lu.solve(rhs)
        return u

    def heat_geodesic(self, dt: float, extra: int = 0) -> np.ndarray:
        """The heat method of Sec. 7.2 with the curves as the distance source:
        (1) one implicit Euler step (I - dt M) v = 0 off C, v = 1 on C;
        (2) X = -grad v / |grad v|; (3) M phi = div X with phi = 0 on C.
        `extra` repeats (2)-(3) with X = grad phi / |grad phi|.  Direct solves."""
        v = self.solve_direct(1.0, -dt, self.rhs(None, np.ones(self.NC)))
        X = self.surface_gradient(v, normalize=True)
        for _ in range(extra + 1):
            b = self.surface_divergence(X)
            phi = self.solve_direct(0.0, 1.0, self.rhs(b, np.zeros(self.NC)))
            X = self.surface_gradient(-phi, normalize=True)
        return phi

    def precond(self, m: float, n: float) -> np.ndarray:
        d = np.ones(self.N)
        d[:self.NS] = 1.0 / (m + n * self.diagL())
        return d

    def crossing_vector(self, k: int, i: int) -> np.ndarray:
        """The crossing vector cp_{S-C}(x_i) for curve k as the crossing test uses
        it (tie-resolved; projected when the curve asks for Sec. 4.7's test)."""
        z = np.zeros(3)
        _check(lib().orc_crossing_vector(self._h, int(k), int(i), _ptr(z)))
        return z

    def solve_direct(self, m: float, n: float, f: np.ndarray) -> np.ndarray:
        lu = spla.splu(self.A(m, n).tocsc())
        return lu.solve(np.asarray(f, dtype=np.float64))

    def solve_adjoint_direct(self, m: float, n: float, y: np.ndarray) -> np.ndarray:
        lu = spla.splu(self.A(m, n).T.tocsc())
        return lu.solve(np.asarray(y, dtype=np.float64))

    def bicgstab(self, m: float, n: float, f: np.ndarray, tol: float = 1e-13, maxit: int = 20000,
                 x0: Optional[np.ndarray] = None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros(self.N) if x0 is None else np.array(x0, dtype=np.float64)
        it, rr = ctypes.c_int(), ctypes.c_double()
        rc = lib().orc_bicgstab(self._h, m, n, _ptr(f), _ptr(x), tol, maxit, ctypes.byref(it), ctypes.byref(rr))
        if rc not in (0,):
            raise OracleError(f"{_ERRS.get(rc, rc)} after {it.value} iterations, relres {rr.value:.3e}")
        return x, it.value, rr.value

    # -- boundary data (Sec. 4.3, Sec. 5.2) ------------------------------
    def curve_param(self) -> np.ndarray:
        """Angle of cp_C(x_alpha) around its circle (0 for points), in [0, 2pi)."""
        out = np.zeros(self.NC)
        for a in range(self.NC):
            cv = self.curves[self.bc_curve[a]]
            if cv.kind != ci.CV_CIRCLE:
                continue
            q = self.cpc[a] - np.asarray(cv.p)
            e1 = np.asarray(cv.ref, dtype=np.float64)
            e2 = np.cross(np.asarray(cv.nu, dtype=np.float64), e1)
            ang = math.atan2(float(q @ e2), float(q @ e1))
            out[a] = ang % (2.0 * math.pi)
        return out

    def bc_scale(self) -> np.ndarray:
        """c_alpha: 1 for first-order and 2 for second-order Dirichlet rows, 0 for
        zero-Neumann rows (per BC DOF: the type of the side it stands in for)."""
        return np.array([{ci.BC_DIR1: 1.0, ci.BC_DIR2: 2.0}.get(int(t), 0.0) for t in self.bc_type])

    def sample_matrix(self, nsamples: Sequence[int]) -> sp.csr_matrix:
        """B: per-curve periodic linear interpolation of samples (taken at angles
        2 pi k / n_s) to the BC DOFs; for two-sided curves the sample block of the
        side opposite cp_S(x_alpha) is used (both blocks averaged on C itself).
        Column layout: curves in order; each curve has n_s columns, or 2 n_s
        (plus-side block then minus-side block) when two-sided."""
        offs, tot = [], 0
        for k, cv in enumerate(self.curves):
            offs.append(tot)
            tot += nsamples[k] * (2 if cv.two_sided else 1)
        ang = self.curve_param()
        rows, cols, vals = [], [], []
        for a in range(self.NC):
            k = int(self.bc_curve[a]); cv = self.curves[k]; ns = nsamples[k]
            s = ang[a] / (2.0 * math.pi) * ns
            i0 = int(math.floor(s)) % ns
            fr = s - math.floor(s)
            i1 = (i0 + 1) % ns
            if cv.two_sided:
                side = int(self.bc_side[a])
                blocks = [(offs[k] + ns, 1.0)] if side > 0 else [(offs[k], 1.0)] if side < 0 else \
                    [(offs[k], 0.5), (offs[k] + ns, 0.5)]
            else:
                blocks = [(offs[k], 1.0)]
            for b0, wb in blocks:
                rows += [a, a]; cols += [b0 + i0, b0 + i1]; vals += [wb * (1.0 - fr), wb * fr]
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.NC, tot))

    def rhs(self, s_pde: Optional[np.ndarray], g_bc: np.ndarray) -> np.ndarray:
        """f = [s ; c_alpha g_alpha] (g_alpha: the prescribed value per BC DOF)."""
        f = np.zeros(self.N)
        if s_pde is not None:
            f[:self.NS] = s_pde
        f[self.NS:] = self.bc_scale() * np.asarray(g_bc, dtype=np.float64)
        return f


def n_threads() -> int:
    return lib().orc_num_threads()
