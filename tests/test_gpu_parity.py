"""GPU parity: the sm_103a library (through the C ABI) against the CPU oracle,
element by element on the same seeded inputs.

Bars: band, DOF order, twins, sides and closest points bit-exact (analytic
shapes, no FMA contraction on either side); FP64 apply and extension within
1e-14 relative (they differ only in the order of rounding and in barycentric
vs product-form weights); FP32 apply within 2e-6 relative to max|A u| (FP32
rounding of weights and values); FP64 solves within 1e-10 relative L-inf of the
oracle's direct solve; FP32 + FP64-refinement solves within 1e-9."""
import math

import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import SMALL, need_gpu, pair, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    return need_gpu()


@pytest.mark.parametrize("name", list(SMALL))
def test_band_and_boundary_bit_exact(oracle_mod, torch_mod, name):
    w = SMALL[name]()
    band, ref = pair(oracle_mod, w)
    assert band.NS == ref.NS and band.NC == ref.NC
    ijk, cp = band.export_band()
    assert np.array_equal(ijk.cpu().numpy(), ref.ijk)
    assert np.array_equal(cp.cpu().numpy(), ref.cp)
    if ref.NC:
        b = band.export_boundary()
        assert np.array_equal(b["twin"].cpu().numpy(), ref.twin)
        assert np.array_equal(b["curve"].cpu().numpy(), ref.bc_curve)
        assert np.array_equal(b["side"].cpu().numpy(), ref.bc_side)
        assert np.array_equal(b["cpc"].cpu().numpy(), ref.cpc)
        assert np.max(np.abs(b["param"].cpu().numpy() - ref.curve_param())) < 1e-12
    assert band.diagnostics()["noflip_twin"] == ref.noflip_twin


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("m,n", [(0.0, 1.0), (1.0, -0.01)])
def test_apply_fp64_matches_oracle(oracle_mod, torch_mod, name, m, n):
    torch = torch_mod
    w = SMALL[name]()
    band, ref = pair(oracle_mod, w)
    u = ci.random_vector(ref.N, seed=5)
    v = band.apply(m, n, torch.tensor(u, device="cuda")).cpu().numpy()
    vr = ref.apply(m, n, u)
    assert rel_inf(v, vr) < 1e-14
    # the extension E u (surface values at cp_S) too
    a = band.extend(torch.tensor(u, device="cuda")).cpu().numpy()
    assert rel_inf(a, ref.extend(u)) < 1e-14


@pytest.mark.parametrize("name", ["circle_dir2", "sphere_lat_dir2", "torus_mer_dir2"])
def test_apply_fp32_and_batched(oracle_mod, torch_mod, name):
    torch = torch_mod
    w = SMALL[name]()
    band, ref = pair(oracle_mod, w)
    U = ci.random_vector(ref.N, seed=9, nrhs=5)
    V = band.apply(0.0, 1.0, torch.tensor(U, device="cuda")).cpu().numpy()
    A = ref.A(0.0, 1.0)
    VR = A @ U
    for r in range(5):
        assert rel_inf(V[:, r], VR[:, r]) < 1e-14
    V32 = band.apply(0.0, 1.0, torch.tensor(U, device="cuda", dtype=torch.float32)).cpu().numpy()
    assert np.max(np.abs(V32 - VR)) <= 2e-6 * np.max(np.abs(VR))


@pytest.mark.parametrize("name", ["circle_dir2", "sphere_lat_dir2", "torus_mer_dir2"])
@pytest.mark.parametrize("nrhs", [20, 33, 40, 64])
def test_apply_warp_per_row_batches(oracle_mod, torch_mod, name, nrhs):
    """Batched products (cell-bucketed gather with the flipped-entry correction,
    warp-per-row combine; 33 columns take the per-element path) in FP64 and
    FP32 against the oracle's assembled A, column by column."""
    torch = torch_mod
    w = SMALL[name]()
    band, ref = pair(oracle_mod, w)
    U = ci.random_vector(ref.N, seed=nrhs, nrhs=nrhs)
    VR = ref.A(1.0, -0.01) @ U
    V = band.apply(1.0, -0.01, torch.tensor(U, device="cuda")).cpu().numpy()
    V32 = band.apply(1.0, -0.01, torch.tensor(U, device="cuda", dtype=torch.float32)).cpu().numpy()
    for r in range(nrhs):
        assert rel_inf(V[:, r], VR[:, r]) < 1e-14
    assert np.max(np.abs(V32 - VR)) <= 2e-6 * np.max(np.abs(VR))


@pytest.mark.parametrize("name", ["circle_dir1", "circle_dir2", "sphere_lat_dir2", "torus_mer_dir2",
                                  "sphere_point_dir1"])
def test_fp64_solve_matches_oracle_direct(oracle_mod, torch_mod, name):
    torch = torch_mod
    w = SMALL[name]()
    band, ref = pair(oracle_mod, w)
    rng = np.random.default_rng(3)
    s = rng.uniform(-1, 1, ref.NS) if w.m != 0 else np.zeros(ref.NS)
    g = rng.uniform(0, 1, len(w.curves))[ref.bc_curve] if ref.NC else np.zeros(0)
    f = ref.rhs(s, g)
    fg = band.rhs(s=torch.tensor(s, device="cuda"), g=torch.tensor(g, device="cuda") if ref.NC else None)
    assert rel_inf(fg.cpu().numpy(), f) == 0.0
    # tol below the attainable level: the solver stops at its rounding floor
    x, st = band.solve(w.m, w.n, fg, tol=1e-14, raise_on_error=False)
    xr = ref.solve_direct(w.m, w.n, f)
    # converged to tol or to the FP64 rounding floor of the plain residual
    assert st.status == "CPM_OK" and st.relres <= max(1e-14, 4 * st.relres_floor), st
    assert rel_inf(x.cpu().numpy(), xr) < 1e-10, st


@pytest.mark.parametrize("name", ["circle_dir2", "sphere_lat_dir2"])
def test_fp32_refinement_solve_matches_oracle(oracle_mod, torch_mod, name):
    torch = torch_mod
    w = SMALL[name]()
    band, ref = pair(oracle_mod, w)
    g = np.where(ref.bc_curve == 0, 0.0, 1.0)
    f = ref.rhs(np.zeros(ref.NS), g)
    x, st = band.solve(w.m, w.n, torch.tensor(f, device="cuda"), tol=1e-13, mode="fp32_ir", raise_on_error=False)
    xr = ref.solve_direct(w.m, w.n, f)
    assert st.refinements >= 2 and st.status == "CPM_OK" and st.relres <= max(1e-13, 4 * st.relres_floor), st
    assert rel_inf(x.cpu().numpy(), xr) < 1e-9, st


def test_batched_solve_each_column_matches(oracle_mod, torch_mod):
    torch = torch_mod
    w = SMALL["sphere_lat_dir1"]()
    band, ref = pair(oracle_mod, w)
    rng = np.random.default_rng(4)
    G = rng.uniform(0, 1, (2, 6))[ref.bc_curve]          # [NC, 6]
    F = np.zeros((ref.N, 6))
    for r in range(6):
        F[:, r] = ref.rhs(np.zeros(ref.NS), G[:, r])
    x64, st64 = band.solve(0.0, 1.0, torch.tensor(F, device="cuda"), tol=1e-14, raise_on_error=False)
    x32, st32 = band.solve(0.0, 1.0, torch.tensor(F, device="cuda"), tol=1e-13, mode="fp32_ir",
                           raise_on_error=False)
    assert st64.status == "CPM_OK" and st32.status == "CPM_OK", (st64, st32)
    lu = __import__("scipy.sparse.linalg", fromlist=["splu"]).splu(ref.A(0.0, 1.0).tocsc())
    for r in range(6):
        xr = lu.solve(F[:, r])
        assert rel_inf(x64.cpu().numpy()[:, r], xr) < 1e-10
        assert rel_inf(x32.cpu().numpy()[:, r], xr) < 1e-9


def test_sampled_two_sided_rhs_matches(oracle_mod, torch_mod):
    """Two-sided point data (the Sec. 6.1 jump problem) and sampled circle data
    build the same right-hand side on both sides."""
    torch = torch_mod
    tC = 1.022 * math.pi
    w = ci.Workload("jump", ci.circle2d(), 0.01, [ci.circle_on_unit_circle(tC, ci.BC_DIR2, two_sided=True)], 0.0, 1.0)
    band, ref = pair(oracle_mod, w, n_samples=[1])
    samples = np.array([2.0, 22.0])
    gr = ref.sample_matrix([1]) @ samples
    fg = band.rhs(samples=torch.tensor(samples, device="cuda")).cpu().numpy()
    assert np.array_equal(fg[ref.NS:], ref.bc_scale() * gr)
    w2 = ci.Workload("lat", ci.sphere(), 1 / 16, [ci.latitude_circle(math.pi / 3, ci.BC_DIR1)], 0.0, 1.0)
    band2, ref2 = pair(oracle_mod, w2, n_samples=[64])
    s2 = ci.random_vector(64, seed=2)
    g2 = ref2.sample_matrix([64]) @ s2
    f2 = band2.rhs(samples=torch.tensor(s2, device="cuda")).cpu().numpy()
    assert np.max(np.abs(f2[ref2.NS:] - g2)) < 1e-12


def test_bad_arguments_return_status(oracle_mod, torch_mod):
    torch = torch_mod
    from paper_2305_04711_gb300 import _lib as L
    from paper_2305_04711_gb300.cpm import Band
    with pytest.raises(L.CpmError) as e:
        Band(ci.Shape(ci.SH_TORUS, 3, R=0.3, rt=0.4), 0.05)
    assert e.value.status == "CPM_ERR_ARG"
    band = Band(ci.sphere(), 1 / 16)
    with pytest.raises(L.CpmError) as e:
        band.apply(0.0, 1.0, torch.zeros(band.N, device="cuda", dtype=torch.float64))
    assert e.value.status == "CPM_ERR_STATE"   # apply before set_boundary
    # two circles whose 2r zones overlap
    with pytest.raises(L.CpmError) as e:
        band.set_boundary([ci.latitude_circle(1.0), ci.latitude_circle(1.1)])
    assert e.value.status == "CPM_ERR_OVERLAP"
    band.set_boundary([])
    assert band.NC == 0
    with pytest.raises(L.CpmError):
        band.apply(0.0, 1.0, torch.zeros((band.N, 300), device="cuda", dtype=torch.float64))
