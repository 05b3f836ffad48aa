"""Failure paths of the library, each provoked on the host side or by ordinary
inputs (no kernel is made to fault, trap or hang): every one must come back as
a status code, with the context still usable afterwards."""
import ctypes
import os

import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    return need_gpu()


def _band(w):
    from paper_2305_04711_gb300.cpm import Band
    return Band(w.shape, w.h).set_boundary(w.curves)


def test_maxit_reports_not_converged_with_stats(torch_mod):
    torch = torch_mod
    band = _band(ci.config2(1 / 16, ci.BC_DIR1))
    f = band.rhs(g=torch.tensor(np.where(np.arange(band.NC) % 2 == 0, 0.0, 1.0), device="cuda"))
    for mode in ("fp64", "fp32_ir"):
        x, st = band.solve(0.0, 1.0, f, tol=1e-12, maxit=1, mode=mode, raise_on_error=False)
        assert st.status == "CPM_ERR_NOT_CONVERGED", st
        # one BiCGSTAB step need not reduce the residual; it is reported as is
        assert st.iterations >= 1 and np.isfinite(st.relres) and st.relres > 1e-12, st
    # the context still solves afterwards
    x, st = band.solve(0.0, 1.0, f, tol=1e-10)
    assert st.status == "CPM_OK" and st.relres <= 1e-10


def test_nonfinite_right_hand_side_is_rejected(torch_mod):
    torch = torch_mod
    band = _band(ci.config2(1 / 16, ci.BC_DIR1))
    f = band.rhs(g=torch.ones(band.NC, dtype=torch.float64, device="cuda"))
    f[17] = float("nan")
    for mode in ("fp64", "fp32_ir"):
        x, st = band.solve(0.0, 1.0, f, mode=mode, raise_on_error=False)
        assert st.status == "CPM_ERR_ARG", st
    f[17] = 0.0
    x, st = band.solve(0.0, 1.0, f, tol=1e-10)
    assert st.status == "CPM_OK"


def test_brick_hash_overflow_retries_then_reports_capacity(torch_mod, monkeypatch):
    """A forced tiny initial brick-hash capacity: the build retries with a
    fourfold larger table and gets the same band; when even the last retry is too
    small the build returns CPM_ERR_CAPACITY."""
    from paper_2305_04711_gb300.cpm import Band
    from paper_2305_04711_gb300._lib import CpmError
    ref = Band(ci.sphere(), 1 / 12)
    ijk0, _ = ref.export_band()
    monkeypatch.setenv("CPM_HASH_CAP_INIT", "16")
    band = Band(ci.sphere(), 1 / 12)
    ijk1, _ = band.export_band()
    assert torch_mod.equal(ijk0, ijk1)
    with pytest.raises(CpmError, match="CPM_ERR_CAPACITY"):
        Band(ci.sphere(), 1 / 96)
    monkeypatch.delenv("CPM_HASH_CAP_INIT")
    assert Band(ci.sphere(), 1 / 16).NS > 0


def test_newton_failure_near_the_surface_is_reported(torch_mod, monkeypatch):
    """The App. A projection converges on every bumpy shape tried near S, so its
    failure is provoked with a forced iteration cap of 2: nodes whose level-set
    distance estimate puts them in the band then fail, and the build reports
    CPM_ERR_CP_FAILED; without the cap the same shape builds."""
    from paper_2305_04711_gb300.cpm import Band
    from paper_2305_04711_gb300._lib import CpmError
    sh = ci.bumpy_sphere(16, seed=0)
    # at h = 1/24 the band (radius about 0.1) stays clear of the bumps' medial
    # axes, where closest points stop being unique and the projection may fail
    monkeypatch.setenv("CPM_NEWTON_MAXIT", "2")
    with pytest.raises(CpmError, match="CPM_ERR_CP_FAILED"):
        Band(sh, 1 / 24)
    monkeypatch.delenv("CPM_NEWTON_MAXIT")
    assert Band(sh, 1 / 24).NS > 0


def test_unreserved_width_is_a_capacity_error_not_an_allocation(torch_mod):
    """Products and solves allocate nothing: through the raw C ABI, a batch wider
    than the reserved workspace returns CPM_ERR_CAPACITY; after cpm_reserve it
    runs."""
    torch = torch_mod
    from paper_2305_04711_gb300 import _lib as L
    band = _band(ci.config2(1 / 16, ci.BC_DIR1))
    lib = L.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    u = torch.rand((band.N, 8), dtype=torch.float64, device="cuda")
    v = torch.empty_like(u)
    rc = lib.cpm_apply(band._h, 0.0, 1.0, L.PREC_FP64, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                       8, 8, stream)
    assert L.STATUS[rc] == "CPM_ERR_CAPACITY"
    o = L.SolveOpts(1e-10, 5000, L.SOLVE_FP64, 0.0, 0, 16, L.NORM_PLAIN, 0)
    st = L.SolveStats()
    rc = lib.cpm_solve(band._h, 0.0, 1.0, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), 8, 8,
                       ctypes.byref(o), ctypes.byref(st), stream)
    assert L.STATUS[rc] == "CPM_ERR_CAPACITY"
    assert L.STATUS[lib.cpm_reserve(band._h, 8, L.RESERVE_FP64)] == "CPM_OK"
    rc = lib.cpm_apply(band._h, 0.0, 1.0, L.PREC_FP64, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                       8, 8, stream)
    assert L.STATUS[rc] == "CPM_OK"
    f = band.rhs(g=torch.ones((band.NC, 8), dtype=torch.float64, device="cuda"), nrhs=8)
    x = torch.zeros_like(f)
    rc = lib.cpm_solve(band._h, 0.0, 1.0, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(x.data_ptr()), 8, 8,
                       ctypes.byref(o), ctypes.byref(st), stream)
    assert L.STATUS[rc] == "CPM_OK" and st.relres <= 1e-10
