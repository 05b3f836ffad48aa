"""GPU parity for the projected crossing test (Sec. 4.7): the sm_103a library
through the C ABI against the CPU oracle with the same curves marked
`projected`.  Bars as in test_gpu_parity: BC DOFs, twins, sides and types
bit-exact; FP64 products within 1e-14 relative; FP64 solves within 1e-10 of the
oracle's direct solve."""
import math

import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import need_gpu, pair, rel_inf

pytestmark = pytest.mark.gpu


def _proj(curves):
    for cv in curves:
        cv.projected = True
    return curves


def _great_circle(bc):
    n = np.array([0.31, 0.47, 0.83]); n /= np.linalg.norm(n)
    ref = np.cross(n, [1.0, 0.0, 0.0]); ref /= np.linalg.norm(ref)
    return ci.Curve(ci.CV_CIRCLE, bc, (0.0, 0.0, 0.0), nu=tuple(n), rad=1.0, ref=tuple(ref))


CASES = {
    "sphere_lat_dir1": lambda: ci.config2(1 / 16, ci.BC_DIR1),
    "sphere_lat_dir2": lambda: ci.config2(1 / 20, ci.BC_DIR2),
    "circle_dir2": lambda: ci.config1(0.01, ci.BC_DIR2),
    "torus_mer_dir2": lambda: ci.Workload("tp", ci.torus(1.0, 0.4), 1 / 16,
                                          [ci.torus_meridian(0.3, 1.0, 0.4, ci.BC_DIR2),
                                           ci.torus_meridian(2.5, 1.0, 0.4, ci.BC_DIR2)], 0.0, 1.0),
    "sphere_point_dir1": lambda: ci.Workload("spp", ci.sphere(), 1 / 16,
                                             [ci.point_curve((0.0, 0.6, 0.8), ci.BC_DIR1)], 1.0, -1 / 16),
    "sphere_great_neu2": lambda: ci.Workload("sgn", ci.sphere(), 1 / 12, [_great_circle(ci.BC_NEU2)], 1.0, -1.0),
}


@pytest.fixture(scope="module")
def torch_mod():
    return need_gpu()


def _pair(oracle_mod, name):
    w = CASES[name]()
    w.curves = _proj(list(w.curves))
    band, ref = pair(oracle_mod, w)
    return w, band, ref


@pytest.mark.parametrize("name", list(CASES))
def test_projected_boundary_bit_exact_and_products(oracle_mod, torch_mod, name):
    torch = torch_mod
    w, band, ref = _pair(oracle_mod, name)
    assert band.NS == ref.NS and band.NC == ref.NC
    b = band.export_boundary()
    assert np.array_equal(b["twin"].cpu().numpy(), ref.twin)
    assert np.array_equal(b["side"].cpu().numpy(), ref.bc_side)
    assert np.array_equal(b["type"].cpu().numpy(), ref.bc_type)
    assert band.diagnostics()["noflip_twin"] == ref.noflip_twin
    U = ci.random_vector(ref.N, seed=5, nrhs=3)
    A = ref.A(w.m, w.n)
    V = band.apply(w.m, w.n, torch.tensor(U, device="cuda")).cpu().numpy()
    VT = band.apply(w.m, w.n, torch.tensor(U, device="cuda"), transpose=True).cpu().numpy()
    VR, VTR = A @ U, A.T @ U
    for r in range(3):
        assert rel_inf(V[:, r], VR[:, r]) < 1e-14
        assert rel_inf(VT[:, r], VTR[:, r]) < 1e-14


@pytest.mark.parametrize("name", ["sphere_lat_dir2", "circle_dir2", "torus_mer_dir2", "sphere_great_neu2"])
def test_projected_solves_match_oracle_direct(oracle_mod, torch_mod, name):
    torch = torch_mod
    w, band, ref = _pair(oracle_mod, name)
    rng = np.random.default_rng(8)
    s = rng.uniform(-1, 1, ref.NS) if w.m != 0 else np.zeros(ref.NS)
    g = rng.uniform(0, 1, ref.NC)
    f = ref.rhs(s, g)
    fg = band.rhs(s=torch.tensor(s, device="cuda"), g=torch.tensor(g, device="cuda"))
    x, st = band.solve(w.m, w.n, fg, tol=1e-13, raise_on_error=False)
    assert st.status == "CPM_OK" and st.relres <= max(1e-13, 4 * st.relres_floor), st
    assert rel_inf(x.cpu().numpy(), ref.solve_direct(w.m, w.n, f)) < 1e-10, st


def test_projected_equals_plain_on_the_sphere(oracle_mod, torch_mod):
    """On the smooth sphere both tests flip the same entries (the oracle pins
    this), so the two GPU operators give identical products."""
    torch = torch_mod
    from paper_2305_04711_gb300.cpm import Band
    h = 1 / 24
    plain = Band(ci.sphere(), h).set_boundary(ci.config2(h, ci.BC_DIR2).curves)
    proj = Band(ci.sphere(), h).set_boundary(_proj(ci.config2(h, ci.BC_DIR2).curves))
    u = torch.tensor(ci.random_vector(plain.N, seed=2), device="cuda")
    assert torch.equal(plain.apply(0.0, 1.0, u), proj.apply(0.0, 1.0, u))
