"""Pin of the oracle's Crank-Nicolson time stepping (the heat-equation study of
Sec. 6.2; rows with m = 1 and n = -+dt/2): on the closed unit sphere the heat
equation keeps u0 = x (a degree-1 harmonic, Delta_S x = -2x) as exp(-2t) x, and the
CPM error falls at second order in h (dt = 0.01, CN's O(dt^2) is below it)."""
import numpy as np

import cpm_inputs as ci


def test_cn_heat_on_sphere_second_order(oracle_mod):
    errs = []
    for h in (1 / 12, 1 / 16):
        ref = oracle_mod.Oracle(ci.sphere(), h).set_curves([])
        u = ref.heat_cn(ref.cp[:, 0].copy(), 0.01, 10)
        errs.append(np.abs(ref.extend(u) - np.exp(-0.2) * ref.cp[:, 0]).max())
    assert errs[1] < 5e-4, errs
    assert errs[1] < (12 / 16) ** 1.7 * errs[0], errs
