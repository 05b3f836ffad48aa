"""Parity at full size: the unit sphere at h = 1/128 with the two Dirichlet
latitude circles (1.76M DOFs) in the batched launch configuration (64
right-hand sides: batched FP32 and FP64 products) and the single-RHS one.  Band,
DOF order, closest points and twins are compared bit for bit; products on
sampled rows, which the oracle evaluates one by one from its assembled rows
(random rows plus rows next to the curves); solutions against the oracle's own
BiCGSTAB."""
import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import need_gpu, rel_inf

pytestmark = pytest.mark.gpu


def sampled_product(ref, rows, m, n, U):
    """(A U)[rows] from the oracle's assembled E, L - diag L and B rows."""
    U = np.asarray(U, dtype=np.float64)
    pde_rows = rows[rows < ref.NS]
    bc_rows = rows[rows >= ref.NS] - ref.NS
    Lo = ref.Loff[pde_rows]
    cols = np.unique(Lo.indices)
    pde, bc = cols[cols < ref.NS], cols[cols >= ref.NS]
    a = np.zeros((ref.N,) + U.shape[1:])
    a[pde] = ref.E[pde] @ U
    a[bc] = U[bc]
    out = np.zeros((len(rows),) + U.shape[1:])
    out[:len(pde_rows)] = m * U[pde_rows] + n * (ref.diagL() * U[pde_rows] + Lo @ a)
    out[len(pde_rows):] = ref.B[bc_rows] @ U
    return out


@pytest.fixture(scope="module")
def full(oracle_mod):
    torch = need_gpu()
    from paper_2305_04711_gb300.cpm import Band
    w = ci.config2(1 / 128, ci.BC_DIR1)
    band = Band(w.shape, w.h).set_boundary(w.curves)
    ref = oracle_mod.Oracle(w.shape, w.h).set_curves(w.curves)
    rng = np.random.default_rng(0)
    near = np.nonzero(ref.near_c >= 0)[0]
    rows = np.concatenate([rng.choice(ref.NS, 2000, replace=False),
                           rng.choice(near, min(2000, len(near)), replace=False),
                           ref.NS + rng.choice(ref.NC, min(500, ref.NC), replace=False)])
    rows = np.unique(rows)   # PDE rows first, then BC rows (sorted)
    yield torch, w, band, ref, rows
    band.close()


def test_full_band_and_boundary_bit_exact(full):
    torch, w, band, ref, rows = full
    assert band.NS == ref.NS and band.NC == ref.NC
    ijk, cp = band.export_band()
    assert np.array_equal(ijk.cpu().numpy(), ref.ijk)
    assert np.array_equal(cp.cpu().numpy(), ref.cp)
    b = band.export_boundary()
    assert np.array_equal(b["twin"].cpu().numpy(), ref.twin)
    assert np.array_equal(b["side"].cpu().numpy(), ref.bc_side)
    assert np.array_equal(b["cpc"].cpu().numpy(), ref.cpc)


def test_full_products_on_sampled_rows(full):
    torch, w, band, ref, rows = full
    U = ci.random_vector(ref.N, seed=31, nrhs=64)
    VR = sampled_product(ref, rows, 1.0, -0.01, U)
    scale = np.max(np.abs(VR))
    u = torch.tensor(U, device="cuda")
    idx = torch.tensor(rows, device="cuda")
    V64 = band.apply(1.0, -0.01, u)[idx].cpu().numpy()
    assert np.max(np.abs(V64 - VR)) <= 1e-14 * scale
    V32 = band.apply(1.0, -0.01, u.float())[idx].cpu().numpy()
    assert np.max(np.abs(V32 - VR)) <= 2e-6 * scale
    v1 = band.apply(1.0, -0.01, u[:, 0].contiguous())[idx].cpu().numpy()
    assert np.max(np.abs(v1 - VR[:, 0])) <= 1e-14 * np.max(np.abs(VR[:, 0]))
    del u, V64, V32


def test_full_solution_parity_against_oracle_bicgstab(full):
    """The solve at the full size (Laplace between the latitude circles, u = 0 and
    1 on them): the GPU's FP64 and FP32 + FP64-refinement solutions, both to the
    paper's test |f - A x|_2 <= 1e-12 |f|_2, against the oracle's own BiCGSTAB run
    to 1e-13 (minutes of host time at 1.76M DOFs).  The remaining difference is
    the two solutions' distance to the exact discrete one, at most about the
    condition number (~1e5 here) times the residuals."""
    torch, w, band, ref, rows = full
    g = np.where(ref.bc_curve == 0, 0.0, 1.0)
    f = ref.rhs(np.zeros(ref.NS), g)
    xr, it, rr = ref.bicgstab(0.0, 1.0, f, tol=1e-13, maxit=40000)
    assert rr <= 1e-13
    fg = band.rhs(g=torch.tensor(g, device="cuda"))
    assert np.array_equal(fg.cpu().numpy(), f)
    for mode, bar in (("fp64", 1e-10), ("fp32_ir", 1e-9)):
        x, st = band.solve(0.0, 1.0, fg, tol=1e-12, mode=mode, raise_on_error=False)
        assert st.status == "CPM_OK" and st.relres <= max(1e-12, 4 * st.relres_floor), (mode, st)
        assert rel_inf(x.cpu().numpy(), xr) < bar, (mode, st)
