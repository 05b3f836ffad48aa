"""Crank-Nicolson stepping on the GPU (apply + warm-started solve per step)
against the oracle's, on the closed sphere with u0 = x (exact exp(-2t) x) and on
the sphere with two Dirichlet latitude circles."""
import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import need_gpu, pair, rel_inf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("curves", ["none", "latitudes"])
def test_cn_steps_match_oracle(oracle_mod, curves):
    torch = need_gpu()
    from paper_2305_04711_gb300.timestep import heat_cn
    h = 1 / 16
    cv = [] if curves == "none" else ci.config2(h, ci.BC_DIR1).curves
    w = ci.Workload("sph_cn", ci.sphere(), h, cv, 1.0, -0.005)
    band, ref = pair(oracle_mod, w)
    u0 = np.concatenate([ref.cp[:, 0], ref.cpc[:, 0] if ref.NC else np.zeros(0)])
    u, stats = heat_cn(band, torch.tensor(u0, device="cuda"), 0.01, 10)
    ur = ref.heat_cn(u0, 0.01, 10)
    assert rel_inf(u.cpu().numpy(), ur) < 1e-9
    if curves == "none":
        a = band.extend(u).cpu().numpy()
        assert np.abs(a - np.exp(-0.2) * ref.cp[:, 0]).max() < 5e-4


def test_cn_dir2_with_time_dependent_data_matches_oracle(oracle_mod):
    """Second-order Dirichlet latitude circles carrying exp(-2t) z (the exact
    heat solution on the unit sphere): each step's BC rows take c_alpha g(t_{k+1})
    from cpm_rhs, as the oracle's rows do (Sec. 6.2)."""
    torch = need_gpu()
    from paper_2305_04711_gb300.timestep import heat_cn
    h = 1 / 16
    w = ci.Workload("sph_cn2", ci.sphere(), h, ci.config2(h, ci.BC_DIR2).curves, 1.0, -0.005)
    band, ref = pair(oracle_mod, w)
    u0 = np.concatenate([ref.cp[:, 2], ref.cp[ref.twin, 2]])
    gz = torch.tensor(ref.cpc[:, 2], device="cuda")
    u, stats = heat_cn(band, torch.tensor(u0, device="cuda"), 0.01, 10, g=lambda t: float(np.exp(-2 * t)) * gz)
    ur = ref.heat_cn(u0, 0.01, 10, g_bc=lambda t: np.exp(-2 * t) * ref.cpc[:, 2])
    assert rel_inf(u.cpu().numpy(), ur) < 1e-9
    a = band.extend(u).cpu().numpy()
    assert np.abs(a - np.exp(-0.2) * ref.cp[:, 2]).max() < 2e-3
