"""Closed-form pins of the oracle's interior boundary conditions: exact
solutions the paper gives or that follow from it, with the convergence orders
the paper reports (slope 1 for first-order and 2 for second-order IBCs)."""
import math

import numpy as np
import pytest

import cpm_inputs as ci


def fit_order(hs, errs):
    return float(np.polyfit(np.log(hs), np.log(errs), 1)[0])


def solve(o, m, n, f):
    if o.dim == 2:
        return o.solve_direct(m, n, f)
    u, it, rr = o.bicgstab(m, n, f, tol=1e-12)
    return u


# --- unit circle, Dirichlet points at grid nodes (the circle workload) -------

def exact_circle_points(cp):
    th = np.arctan2(cp[:, 1], cp[:, 0]) % (2 * math.pi)
    return np.where(th <= math.pi / 2, th / (math.pi / 2), (2 * math.pi - th) / (1.5 * math.pi))


@pytest.mark.parametrize("bc,order", [(ci.BC_DIR1, 1.0), (ci.BC_DIR2, 2.0)])
def test_circle_points_closed_form_and_order(oracle_mod, bc, order):
    hs, errs = [0.04, 0.02, 0.01, 0.005], []
    for h in hs:
        w = ci.config1(h, bc)
        o = oracle_mod.Oracle(w.shape, h).set_curves(w.curves)
        g = np.where(o.bc_curve == 0, 0.0, 1.0)
        u = solve(o, 0.0, 1.0, o.rhs(np.zeros(o.NS), g))
        errs.append(np.max(np.abs(o.extend(u) - exact_circle_points(o.cp))))
    assert abs(fit_order(hs, errs) - order) < 0.15, errs
    if bc == ci.BC_DIR2:
        assert errs[-1] < 1e-6


# --- Sec. 6.1: two-sided discontinuous Dirichlet point ------------------------

@pytest.mark.parametrize("bc,order", [(ci.BC_DIR1, 1.0), (ci.BC_DIR2, 2.0)])
def test_jump_problem_of_section_6_1(oracle_mod, bc, order):
    """-u_tt = 2cos(t - tC) on the unit circle with u jumping between 2 and 22 at
    tC = 1.022 pi; exact u = 2cos(psi) + (10/pi) psi with psi = t - tC in (0, 2pi)."""
    from test_oracle_pins import golden
    g0 = golden()
    tC = float(g0["jump_theta_C_over_pi"]) * math.pi
    lo, hi = float(g0["jump_value_low"]), float(g0["jump_value_high"])
    hs, errs = [0.04, 0.02, 0.01, 0.005, 0.0025], []
    for h in hs:
        o = oracle_mod.Oracle(ci.circle2d(), h).set_curves([ci.circle_on_unit_circle(tC, bc, two_sided=True)])
        psi = (np.arctan2(o.cp[:, 1], o.cp[:, 0]) - tC) % (2 * math.pi)
        # the counter-clockwise side (psi -> 0+) carries the value 2, the other 22
        g = o.sample_matrix([1]) @ np.array([lo, hi])
        u = solve(o, 0.0, 1.0, o.rhs(-2.0 * np.cos(psi), g))
        exact = 2 * np.cos(psi) + (10 / math.pi) * psi
        errs.append(np.max(np.abs(o.extend(u) - exact)))
    p = fit_order(hs, errs)
    assert abs(p - order) < 0.35, (errs, p)


# --- sphere between two Dirichlet latitude circles ---------------------------

A_LOG = 1.0 / (2.0 * math.log(1.0 + math.sqrt(2.0)))


def exact_latitudes(cp):
    th = np.arccos(np.clip(cp[:, 2], -1, 1))
    with np.errstate(divide='ignore'):
        u = A_LOG * np.log(np.tan(th / 2)) + 0.5
    return np.where(th <= math.pi / 4, 0.0, np.where(th >= 3 * math.pi / 4, 1.0, u))


@pytest.mark.parametrize("bc,order", [(ci.BC_DIR1, 1.0), (ci.BC_DIR2, 2.0)])
def test_sphere_latitude_circles_closed_form(oracle_mod, bc, order):
    """u = a ln tan(theta/2) + 1/2 between theta = pi/4 (u=0) and 3pi/4 (u=1),
    a = 1/(2 ln(1 + sqrt 2)); constant on the caps."""
    assert A_LOG == pytest.approx(0.567296, abs=1e-6)
    hs, errs = [1 / 16, 1 / 24, 1 / 32], []
    for h in hs:
        w = ci.config2(h, bc)
        o = oracle_mod.Oracle(w.shape, h).set_curves(w.curves)
        g = np.where(o.bc_curve == 0, 0.0, 1.0)
        u = solve(o, 0.0, 1.0, o.rhs(np.zeros(o.NS), g))
        errs.append(np.max(np.abs(o.extend(u) - exact_latitudes(o.cp))))
        if h == hs[0]:
            # the grid symmetry z -> -z maps the problem to 1 - u on the surface
            # values (band-edge rows with missing neighbours are not affine, so
            # compare E u, the values at cp_S, not the grid values).  Nodes whose
            # cp_S lies on C take a side by a stencil-order rule that is not
            # mirror symmetric, so the symmetry holds to the discretisation error.
            eu = o.extend(u)
            key = {tuple(r): i for i, r in enumerate(o.ijk.tolist())}
            mirror = np.array([key[(x, y, -z)] for x, y, z in o.ijk.tolist()])
            assert np.max(np.abs(eu[mirror] - (1.0 - eu))) <= errs[-1] * 1.05 + 1e-9
    p = fit_order(hs, errs)
    assert abs(p - order) < 0.45, (errs, p)


def test_sphere_circle_sampled_data_stereographic(oracle_mod):
    """Dirichlet data cos(phi) on the circle theta = pi/3, given as 2048 samples
    with periodic linear interpolation.  Harmonic functions are conformally
    invariant in 2D, so u = tan(theta/2)/tan(pi/6) cos(phi) on the north cap and
    cot(theta/2)/cot(pi/6) cos(phi) on the south part."""
    thc = math.pi / 3
    for bc, tol in ((ci.BC_DIR1, 0.03), (ci.BC_DIR2, 1.5e-3)):
        h = 1 / 20
        o = oracle_mod.Oracle(ci.sphere(), h).set_curves([ci.latitude_circle(thc, bc)])
        ns = 2048
        samp = np.cos(2 * math.pi * np.arange(ns) / ns)
        g = o.sample_matrix([ns]) @ samp
        u = solve(o, 0.0, 1.0, o.rhs(np.zeros(o.NS), g))
        th = np.arccos(np.clip(o.cp[:, 2], -1, 1))
        ph = np.arctan2(o.cp[:, 1], o.cp[:, 0])
        with np.errstate(divide="ignore"):
            rad = np.where(th <= thc, np.tan(th / 2) / math.tan(thc / 2), math.tan(thc / 2) / np.tan(th / 2))
        exact = rad * np.cos(ph)
        ok = th < math.pi - 1e-9
        assert np.max(np.abs(o.extend(u) - exact)[ok]) < tol


def test_torus_meridians_piecewise_linear(oracle_mod):
    """On the torus, Delta_S u(phi) = u_phiphi / (R + r cos psi)^2, so Laplace with
    Dirichlet meridians is piecewise linear in the toroidal angle phi."""
    R, rt, p0, p1 = 1.0, 0.4, 0.3, 2.5
    for bc, tol in ((ci.BC_DIR1, 0.03), (ci.BC_DIR2, 5e-4)):
        h = 1 / 16
        o = oracle_mod.Oracle(ci.torus(R, rt), h).set_curves(
            [ci.torus_meridian(p0, R, rt, bc), ci.torus_meridian(p1, R, rt, bc)])
        g = np.where(o.bc_curve == 0, 0.0, 1.0)
        u = solve(o, 0.0, 1.0, o.rhs(None, g))
        ph = np.arctan2(o.cp[:, 1], o.cp[:, 0]) % (2 * math.pi)
        a = (ph - p0) % (2 * math.pi)
        L1 = p1 - p0
        exact = np.where(a <= L1, a / L1, 1.0 - (a - L1) / (2 * math.pi - L1))
        assert np.max(np.abs(o.extend(u) - exact)) < tol


def test_point_source_heat_step_on_sphere_is_axisymmetric(oracle_mod):
    """(I - dt M) v = 0 off C with v = 1 at a point C = +z (the heat-method step 1,
    Sec. 7.2): the solution decreases away from C and stays in [0, 1]."""
    h = 1 / 16
    w = ci.Workload("pt", ci.sphere(), h, [ci.point_curve((0.0, 0.0, 1.0))], m=1.0, n=-h)
    o = oracle_mod.Oracle(w.shape, h).set_curves(w.curves)
    v = solve(o, 1.0, -h, o.rhs(np.zeros(o.NS), np.ones(o.NC)))
    ev = o.extend(v)
    th = np.arccos(np.clip(o.cp[:, 2], -1, 1))
    assert np.all(ev > -1e-3) and np.all(ev < 1.0 + 1e-3)
    # monotone decay in theta (binned)
    bins = np.linspace(0.2, 2.8, 14)
    means = [ev[(th >= bins[k]) & (th < bins[k + 1])].mean() for k in range(len(bins) - 1)]
    assert all(means[k] > means[k + 1] for k in range(len(means) - 1))
