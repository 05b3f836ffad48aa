"""Pins of the oracle's heat-method pieces (Sec. 7.2) on the unit sphere with a
point source at +z:

* the central-difference gradient of the CP extension of z equals the gradient
  of z(x/|x|), (e_z - z n)/|x|, at every node with a complete stencil, and the
  error falls at least like h^1.5;
* the divergence of the CP extension of the tangential field grad_S z equals
  Delta_S z / |x| = -2 z / |x| in the same sense;
* the full heat method (one implicit Euler step with dt = h, normalised
  gradient, Poisson solve with phi = 0 at the source) gives the geodesic
  distance arccos(z), first-order accurate (the method's own order)."""
import numpy as np
import pytest

import cpm_inputs as ci


def _sphere_point(oracle_mod, h):
    w = ci.Workload("sph_pt", ci.sphere(), h, [ci.point_curve((0.0, 0.0, 1.0))], 0.0, 1.0)
    return oracle_mod.Oracle(w.shape, h).set_curves(w.curves)


def _grad_div_errors(ref):
    cp = ref.cp
    r = np.linalg.norm(ref.x(), axis=1)
    nb = ref.fd_neighbours()
    full = (nb >= 0).all(1) & (ref.near_c < 0)
    u = np.concatenate([cp[:, 2], ref.cpc[:, 2]])
    g = ref.surface_gradient(u)[:ref.NS]
    gs = np.stack([-cp[:, 0] * cp[:, 2], -cp[:, 1] * cp[:, 2], 1 - cp[:, 2] ** 2], 1)
    eg = np.abs(g - gs / r[:, None])[full].max()
    X = np.concatenate([gs, np.zeros((ref.NC, 3))])
    X[ref.NS:] = X[ref.twin]
    b = ref.surface_divergence(X)
    eb = np.abs(b + 2 * cp[:, 2] / r)[full].max()
    return eg, eb


def test_gradient_and_divergence_of_extensions():
    from oracle import oracle as oracle_mod
    e1 = _grad_div_errors(_sphere_point(oracle_mod, 1 / 12))
    e2 = _grad_div_errors(_sphere_point(oracle_mod, 1 / 16))
    assert e2[0] < 1e-2 and e2[1] < 3e-2, e2
    ratio = (12 / 16) ** 1.5
    assert e2[0] < ratio * e1[0] and e2[1] < ratio * e1[1], (e1, e2)


def test_heat_method_distance_on_sphere_is_first_order():
    from oracle import oracle as oracle_mod
    errs = []
    for h in (1 / 12, 1 / 16):
        ref = _sphere_point(oracle_mod, h)
        phi = ref.heat_geodesic(h)
        a = ref.extend(phi)
        exact = np.arccos(np.clip(ref.cp[:, 2], -1.0, 1.0))
        keep = ref.cp[:, 2] > -0.9     # away from the antipode, where grad v vanishes
        errs.append(np.abs(a - exact)[keep].max())
    assert errs[1] < 2.5 * (1 / 16), errs
    assert errs[1] < (12 / 16) ** 0.8 * errs[0], errs
