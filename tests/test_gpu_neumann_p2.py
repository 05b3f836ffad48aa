"""GPU parity for the zero-Neumann and mixed IBC rows (Sec. 4.3) and for the
quadratic (p = 2) interpolation (Sec. 7): the sm_103a library through the C ABI
against the CPU oracle on the same inputs.

Bars as in test_gpu_parity: band, twins, sides and BC types bit-exact; FP64
products within 1e-14 relative; FP32 within 2e-6 of max |A u|; FP64 solves
within 1e-10 of the oracle's direct solve; FP32 + refinement within 1e-9."""
import math

import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import need_gpu, pair, rel_inf

pytestmark = pytest.mark.gpu

TC = 1.022 * math.pi


def _point(bc, bc_minus=0):
    cv = ci.circle_on_unit_circle(TC, bc, two_sided=True)
    cv.bc_minus = bc_minus
    return cv


def _great_circle(bc):
    n = np.array([0.31, 0.47, 0.83]); n /= np.linalg.norm(n)
    ref = np.cross(n, [1.0, 0.0, 0.0]); ref /= np.linalg.norm(ref)
    return ci.Curve(ci.CV_CIRCLE, bc, (0.0, 0.0, 0.0), nu=tuple(n), rad=1.0, ref=tuple(ref))


CASES = {
    # name: (workload factory, p)
    "circle_neu1": (lambda: ci.Workload("cn1", ci.circle2d(), 0.02, [_point(ci.BC_NEU1)], 1.0, -1.0), 3),
    "circle_neu2": (lambda: ci.Workload("cn2", ci.circle2d(), 0.01, [_point(ci.BC_NEU2)], 1.0, -1.0), 3),
    "circle_mixed2": (lambda: ci.Workload("cm2", ci.circle2d(), 0.01, [_point(ci.BC_DIR2, ci.BC_NEU2)], 1.0, -1.0), 3),
    "sphere_neu2": (lambda: ci.Workload("sn2", ci.sphere(), 1 / 12, [_great_circle(ci.BC_NEU2)], 1.0, -1.0), 3),
    "sphere_neu1_p2": (lambda: ci.Workload("sn1q", ci.sphere(), 1 / 12, [_great_circle(ci.BC_NEU1)], 1.0, -1.0), 2),
    "circle_dir2_p2": (lambda: ci.config1(0.01, ci.BC_DIR2), 2),
    "sphere_lat_dir2_p2": (lambda: ci.config2(1 / 20, ci.BC_DIR2), 2),
    "torus_mer_p2": (lambda: ci.Workload("tq", ci.torus(1.0, 0.4), 1 / 16,
                                         [ci.torus_meridian(0.3, 1.0, 0.4, ci.BC_DIR2),
                                          ci.torus_meridian(2.5, 1.0, 0.4, ci.BC_DIR1)], 0.0, 1.0), 2),
    "sphere_closed_p2": (lambda: ci.Workload("sq", ci.sphere(), 1 / 12, [], 1.0, -0.01), 2),
}


@pytest.fixture(scope="module")
def torch_mod():
    return need_gpu()


def _pair(oracle_mod, name):
    make, p = CASES[name]
    w = make()
    band, ref = pair(oracle_mod, w, p=p)
    return w, band, ref


@pytest.mark.parametrize("name", list(CASES))
def test_band_boundary_types_bit_exact(oracle_mod, torch_mod, name):
    w, band, ref = _pair(oracle_mod, name)
    assert band.NS == ref.NS and band.NC == ref.NC
    ijk, cp = band.export_band()
    assert np.array_equal(ijk.cpu().numpy(), ref.ijk)
    assert np.array_equal(cp.cpu().numpy(), ref.cp)
    if ref.NC:
        b = band.export_boundary()
        assert np.array_equal(b["twin"].cpu().numpy(), ref.twin)
        assert np.array_equal(b["side"].cpu().numpy(), ref.bc_side)
        assert np.array_equal(b["type"].cpu().numpy(), ref.bc_type)
    assert band.diagnostics()["noflip_twin"] == ref.noflip_twin


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nrhs", [1, 5, 40, 64])
def test_products_match_oracle(oracle_mod, torch_mod, name, nrhs):
    """A u and A^T u in FP64 (1e-14) and A u in FP32 (2e-6 of max), single and
    batched layouts (thread-per-row, cell-bucketed warp gathers)."""
    torch = torch_mod
    w, band, ref = _pair(oracle_mod, name)
    U = ci.random_vector(ref.N, seed=11 + nrhs, nrhs=nrhs)
    A = ref.A(w.m, w.n)
    VR = A @ U
    V = band.apply(w.m, w.n, torch.tensor(U, device="cuda")).cpu().numpy()
    VT = band.apply(w.m, w.n, torch.tensor(U, device="cuda"), transpose=True).cpu().numpy()
    VTR = A.T @ U
    V32 = band.apply(w.m, w.n, torch.tensor(U, device="cuda", dtype=torch.float32)).cpu().numpy()
    if nrhs == 1:
        V, VT, V32, VR, VTR = (x.reshape(-1, 1) for x in (V, VT, V32, VR, VTR))
    for r in range(V.shape[1]):
        assert rel_inf(V[:, r], VR[:, r]) < 1e-14
        assert rel_inf(VT[:, r], VTR[:, r]) < 1e-14
    assert np.max(np.abs(V32 - VR)) <= 2e-6 * np.max(np.abs(VR))


@pytest.mark.parametrize("name", ["circle_neu2", "circle_mixed2", "sphere_neu2", "sphere_neu1_p2", "circle_dir2_p2",
                                  "sphere_lat_dir2_p2", "torus_mer_p2"])
@pytest.mark.parametrize("mode", ["fp64", "fp32_ir"])
def test_solves_match_oracle_direct(oracle_mod, torch_mod, name, mode):
    torch = torch_mod
    w, band, ref = _pair(oracle_mod, name)
    rng = np.random.default_rng(21)
    s = rng.uniform(-1, 1, ref.NS)
    g = rng.uniform(0, 1, ref.NC)
    f = ref.rhs(s, g)
    xr = ref.solve_direct(w.m, w.n, f)
    fg = band.rhs(s=torch.tensor(s, device="cuda"), g=torch.tensor(g, device="cuda"))
    assert rel_inf(fg.cpu().numpy(), f) == 0.0
    x, st = band.solve(w.m, w.n, fg, tol=1e-13, mode=mode, raise_on_error=False)
    assert st.status == "CPM_OK" and st.relres <= max(1e-13, 4 * st.relres_floor), st
    assert rel_inf(x.cpu().numpy(), xr) < (1e-10 if mode == "fp64" else 1e-9), st


def test_neumann_circle_closed_form_on_gpu(oracle_mod, torch_mod):
    """The second-order Neumann point on the circle through the GPU solve:
    -u'' + u = 2 cos(psi), u = cos(psi); the error's order fitted over four
    grids is 2 (it is irregular from one grid to the next, as in the oracle's
    own pin), and each grid's error equals the oracle's."""
    torch = torch_mod
    from paper_2305_04711_gb300.cpm import Band
    errs, hs = [], (0.04, 0.02, 0.01, 0.005)
    for h in hs:
        band = Band(ci.circle2d(), h).set_boundary([_point(ci.BC_NEU2)])
        _, cp = band.export_band()
        cp = cp.cpu().numpy()
        psi = np.arctan2(cp[:, 1], cp[:, 0]) - TC
        f = band.rhs(s=torch.tensor(2.0 * np.cos(psi), device="cuda"),
                     g=torch.zeros(band.NC, dtype=torch.float64, device="cuda"))
        x, st = band.solve(1.0, -1.0, f, tol=1e-13)
        assert st.status == "CPM_OK", st
        errs.append(np.max(np.abs(band.extend(x).cpu().numpy() - np.cos(psi))))
        o = oracle_mod.Oracle(ci.circle2d(), h).set_curves([_point(ci.BC_NEU2)])
        ur = o.solve_direct(1.0, -1.0, o.rhs(2.0 * np.cos(psi), np.zeros(o.NC)))
        # at h = 0.005 the Neumann problem's condition number (~4/h^2) times
        # the FP64 residual floor bounds the agreement near 1e-9
        assert rel_inf(x.cpu().numpy(), ur) < 4e-9
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(order - 2.0) < 0.35, (errs, order)


def test_neumann_point_in_3d_is_rejected(torch_mod):
    from paper_2305_04711_gb300.cpm import Band
    from paper_2305_04711_gb300._lib import CpmError
    band = Band(ci.sphere(), 1 / 8)
    with pytest.raises(CpmError, match="CPM_ERR_ARG"):
        band.set_boundary([ci.point_curve((0.0, 0.0, 1.0), ci.BC_NEU1)])
