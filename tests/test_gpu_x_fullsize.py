"""Parity at the benchmark's full size: config 2 (unit sphere, h = 1/128, the two
Dirichlet latitude circles, 1.76M DOFs) in the launch configuration bench.py
times (64 right-hand sides: batched FP32 and FP64 products; FP32 + FP64
refinement solve).  Band, DOF order, closest points and twins are compared bit
for bit; products and residuals on sampled rows, which the oracle evaluates one
by one from its assembled rows (random rows plus rows next to the curves)."""
import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import need_gpu

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


def test_full_bench_solve_residual_on_sampled_rows(full):
    """The bench's batch of 64 harmonic Poisson problems, solved as bench.py does
    (FP32 + FP64 refinement to a Jacobi-scaled relative residual of 1e-10): the
    oracle's rows give the residual on the sampled rows, each entry bounded by the
    residual's norm."""
    torch, w, band, ref, rows = full
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    wl = bench.Workload("sphere", 1 / 128)
    s, g = wl.host_inputs(band)
    f = np.concatenate([s, ref.bc_scale()[:, None] * g])   # f = [s ; c_alpha g_alpha]
    F = band.rhs(s=torch.tensor(s, device="cuda").contiguous(), g=torch.tensor(g, device="cuda").contiguous(),
                 nrhs=64)
    assert np.max(np.abs(F.cpu().numpy() - f)) <= 1e-15 * np.max(np.abs(f))
    x, st = band.solve(0.0, 1.0, F, tol=1e-10, mode="fp32_ir", raise_on_error=False)
    assert st.status == "CPM_OK", st
    X = x.cpu().numpy()
    R = f[rows] - sampled_product(ref, rows, 0.0, 1.0, X)
    wgt = np.where(rows < ref.NS, ref.precond(0.0, 1.0)[0], 1.0)[:, None]
    wf = np.concatenate([ref.precond(0.0, 1.0)[:ref.NS, None] * f[:ref.NS], f[ref.NS:]])
    fn = np.sqrt(np.sum(wf * wf, axis=0))
    assert np.all(np.max(np.abs(wgt * R), axis=0) <= 1.01e-10 * fn)
