"""Heat-method pieces (Sec. 7.2) and the bumpy sphere on the GPU against the
oracle: the surface gradient and divergence of CP extensions, the full
heat-step / normalised-gradient / Poisson pipeline, and the band of the
level-set bumpy sphere (App. A closest points)."""
import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import SMALL, need_gpu, pair, rel_inf

pytestmark = pytest.mark.gpu


def _offaxis_point():
    p = np.array([0.3, 0.2, 0.93])
    return p / np.linalg.norm(p)


@pytest.mark.parametrize("name", ["sphere_lat_dir1", "circle_dir2", "sphere_point_dir1"])
def test_gradient_and_divergence_match_oracle(oracle_mod, name):
    torch = need_gpu()
    band, ref = pair(oracle_mod, SMALL[name]())
    u = ci.random_vector(ref.N, seed=17)
    for normalize in (False, True):
        Xg = band.surface_gradient(torch.tensor(u, device="cuda"), normalize=normalize).cpu().numpy()
        Xr = ref.surface_gradient(u, normalize=normalize)
        assert rel_inf(Xg, Xr) < 1e-12
    X = ci.random_vector(ref.N, seed=18, nrhs=3)
    if ref.dim == 2:
        X[:, 2] = 0.0
    bg = band.surface_divergence(torch.tensor(X, device="cuda")).cpu().numpy()
    br = ref.surface_divergence(X)
    assert rel_inf(bg, br) < 1e-12


def test_heat_geodesic_pipeline_matches_oracle_and_distance(oracle_mod):
    torch = need_gpu()
    from paper_2305_04711_gb300.heat import geodesic_distance
    p = _offaxis_point()
    h = 1 / 16
    w = ci.Workload("sph_pt", ci.sphere(), h, [ci.point_curve(tuple(p))], 0.0, 1.0)
    band, ref = pair(oracle_mod, w)
    phi, st1, st2 = geodesic_distance(band, h, tol=1e-12)
    pr = ref.heat_geodesic(h)
    assert rel_inf(phi.cpu().numpy(), pr) < 1e-7
    a = band.extend(phi).cpu().numpy()
    exact = np.arccos(np.clip(ref.cp @ p, -1.0, 1.0))
    keep = ref.cp @ p > -0.9
    assert np.abs(a - exact)[keep].max() < 2.5 * h


def test_bumpy_sphere_band_matches_oracle(oracle_mod):
    torch = need_gpu()
    from paper_2305_04711_gb300.cpm import Band
    sh = ci.bumpy_sphere(16, 0)
    h = 1 / 24
    ref = oracle_mod.Oracle(sh, h)
    band = Band(sh, h)
    ijk, cp = band.export_band()
    ijk, cp = ijk.cpu().numpy(), cp.cpu().numpy()
    # closest points come from a Newton iteration with exp(): the two sides may
    # differ in the last bits, so membership is compared as sets with nodes at
    # the band radius (|x - cp| within 1e-12 of r) allowed to differ
    A = {tuple(r) for r in ijk.tolist()}
    R = {tuple(r) for r in ref.ijk.tolist()}
    diff = A ^ R
    if diff:
        x = np.array(sorted(diff), dtype=np.float64) * h
        cps = np.array([oracle_mod.closest_point(sh, xi) for xi in x])
        dist = np.linalg.norm(x - cps, axis=1)
        assert np.all(np.abs(dist - ref.rband) < 1e-12)
    rindex = {k: i for i, k in enumerate(map(tuple, ref.ijk.tolist()))}
    pairs = [(i, rindex[k]) for i, k in enumerate(map(tuple, ijk.tolist())) if k in rindex]
    ga, gr = np.array(pairs).T
    assert np.max(np.abs(cp[ga] - ref.cp[gr])) < 1e-12
