"""Closed-form pins of the oracle's zero-Neumann and mixed interior boundary
conditions (Sec. 4.3) and of its quadratic (p = 2) interpolation (Sec. 7,
Eq. (3)), against exact solutions that follow from the paper's model problems
and the orders it reports (slope 1 for first-order and 2 for second-order IBCs;
second-order behaviour observed for p = 2, Sec. 7)."""
import math

import numpy as np
import pytest

import cpm_inputs as ci


def fit_order(hs, errs):
    return float(np.polyfit(np.log(hs), np.log(errs), 1)[0])


def point_on_circle(theta, bc, bc_minus=0):
    cv = ci.circle_on_unit_circle(theta, bc, two_sided=True)
    cv.bc_minus = bc_minus
    return cv


# --- Eq. (3) with p = 2 ------------------------------------------------------

def test_tube_radius_p2_matches_eq3(oracle_mod):
    from test_oracle_pins import golden
    g = golden()
    assert g["tube_radius_d2_p2_q1"] == "sqrt(8.5)" and g["tube_radius_d3_p2_q1"] == "sqrt(10.75)"
    h = 0.01
    assert oracle_mod.tube_radius(2, h, p=2) == pytest.approx(math.sqrt(8.5) * h, rel=1e-15)
    assert oracle_mod.tube_radius(3, h, p=2) == pytest.approx(math.sqrt(10.75) * h, rel=1e-15)


# --- quadratic barycentric weights --------------------------------------------

def test_quadratic_barycentric_weights(oracle_mod):
    rng = np.random.default_rng(7)
    for t in list(rng.uniform(0.5, 1.5, 200)) + [0.5, 1.0, 1.5 - 1e-12]:
        w = oracle_mod.bary_weights(t, p=2)
        assert w.shape == (3,)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        # Lagrange product form on nodes 0, 1, 2
        pf = np.array([(t - 1) * (t - 2) / 2, -t * (t - 2), t * (t - 1) / 2])
        assert np.max(np.abs(w - pf)) < 1e-14
        c = rng.normal(size=3)
        assert w @ np.polyval(c, np.arange(3.0)) == pytest.approx(np.polyval(c, t), abs=1e-12)
    assert np.array_equal(oracle_mod.bary_weights(1.0, p=2), np.array([0.0, 1.0, 0.0]))


@pytest.mark.parametrize("shape,h", [(ci.sphere(), 1 / 16), (ci.torus(), 1 / 16), (ci.circle2d(), 0.02)])
def test_E_p2_reproduces_tensor_quadratics_and_centres_the_stencil(oracle_mod, shape, h):
    """With p = 2, E u for a tensor-product quadratic P equals P(cp_S(x_i)); the
    stencil's nodes all lie within 1.5 h of the query point per axis."""
    o = oracle_mod.Oracle(shape, h, p=2).set_curves([])
    rng = np.random.default_rng(8)
    cx, cy, cz = rng.normal(size=(3, 3))

    def P(q):
        v = np.polyval(cx, q[:, 0]) * np.polyval(cy, q[:, 1])
        return v * np.polyval(cz, q[:, 2]) if shape.dim == 3 else v

    u = P(o.x())
    assert np.max(np.abs(o.extend(u) - P(o.cp))) < 1e-11 * max(1.0, np.max(np.abs(u)))
    npts = 27 if shape.dim == 3 else 9
    assert np.all(np.diff(o.E.indptr) == npts)
    E = o.E.tocoo()
    off = np.abs(o.ijk[E.col].astype(np.float64) * h - o.cp[E.row])[:, :shape.dim]
    assert off.max() <= 1.5 * h * (1 + 1e-12)


@pytest.mark.parametrize("shape,h,box", [(ci.circle2d(), 0.05, 26), (ci.sphere(), 1.0 / 10, 14)])
def test_bfs_band_p2_equals_bruteforce(oracle_mod, shape, h, box):
    o = oracle_mod.Oracle(shape, h, p=2)
    bf = oracle_mod.band_bruteforce(shape, h, [-box] * shape.dim, [box] * shape.dim, p=2)
    assert {tuple(r) for r in o.ijk.tolist()} == {tuple(r) for r in bf.tolist()}
    assert np.all(np.linalg.norm(o.x() - o.cp, axis=1) <= o.rband)


def test_M_p2_sphere_harmonic_eigen_relation(oracle_mod):
    """(M u)_i ~ -l(l+1) Y(cp_i) / |x_i|^2 for the extension of Y_4^2 with p = 2.
    The pointwise consistency error is O(h^(p+1) / h^2) = O(h) for quadratic
    interpolation (the first order that CPM theory predicts, Sec. 7); a wrong
    stencil would leave an O(1) error."""
    errs, hs = [], [1 / 10, 1 / 14, 1 / 20, 1 / 28]
    for h in hs:
        o = oracle_mod.Oracle(ci.sphere(), h, p=2).set_curves([])
        y = ci.real_ylm(4, 2, o.cp)
        Mu = o.M() @ y
        target = -20.0 * y / np.sum(o.x() ** 2, axis=1)
        interior = np.diff(o.Loff.indptr) == 6
        errs.append(np.max(np.abs(Mu - target)[interior]))
    assert 0.8 < fit_order(hs, errs) < 1.4, errs


@pytest.mark.parametrize("bc,order", [(ci.BC_DIR1, 1.0), (ci.BC_DIR2, 2.0)])
def test_circle_points_p2_closed_form(oracle_mod, bc, order):
    """Config 1's point Dirichlet problem with quadratic interpolation."""
    from test_oracle_ibc import exact_circle_points
    hs, errs = [0.04, 0.02, 0.01, 0.005], []
    for h in hs:
        w = ci.config1(h, bc)
        o = oracle_mod.Oracle(w.shape, h, p=2).set_curves(w.curves)
        u = o.solve_direct(0.0, 1.0, o.rhs(np.zeros(o.NS), np.where(o.bc_curve == 0, 0.0, 1.0)))
        errs.append(np.max(np.abs(o.extend(u) - exact_circle_points(o.cp))))
    assert abs(fit_order(hs, errs) - order) < 0.3, errs


# --- zero-Neumann on the unit circle (2D) --------------------------------------

@pytest.mark.parametrize("bc,order", [(ci.BC_NEU1, 1.0), (ci.BC_NEU2, 2.0)])
def test_circle_neumann_point_screened_poisson(oracle_mod, bc, order):
    """-u'' + u = 2 cos(psi) on the unit circle cut at tC = 1.022 pi (Sec. 6.1's
    point) with u' = 0 on both sides: exact u = cos(psi), psi = theta - tC.
    A = I - M (m = 1, n = -1)."""
    tC = 1.022 * math.pi
    hs, errs = [0.04, 0.02, 0.01, 0.005], []
    for h in hs:
        o = oracle_mod.Oracle(ci.circle2d(), h).set_curves([point_on_circle(tC, bc)])
        assert set(o.bc_type.tolist()) == {bc}
        psi = np.arctan2(o.cp[:, 1], o.cp[:, 0]) - tC
        u = o.solve_direct(1.0, -1.0, o.rhs(2.0 * np.cos(psi), np.zeros(o.NC)))
        errs.append(np.max(np.abs(o.extend(u) - np.cos(psi))))
    p = fit_order(hs, errs)
    assert abs(p - order) < 0.35, (errs, p)


def test_circle_neumann_rows_are_interpolation_equations(oracle_mod):
    """A first-order zero-Neumann BC row is u_alpha - sum_beta w_beta u_beta = 0
    with the weights of the stencil at cp_C(x_alpha): its entries sum to zero,
    and for a point C the query point is C itself."""
    tC = 1.022 * math.pi
    o = oracle_mod.Oracle(ci.circle2d(), 0.02).set_curves([point_on_circle(tC, ci.BC_NEU1)])
    B = o.B.tocsr()
    for a in range(o.NC):
        row = B[a]
        assert row.sum() == pytest.approx(0.0, abs=1e-13)
        assert B[a, o.NS + a] != 0.0
    assert np.allclose(o.bc_scale(), 0.0)


@pytest.mark.parametrize("bc,order", [((ci.BC_DIR1, ci.BC_NEU1), 1.0), ((ci.BC_DIR2, ci.BC_NEU2), 2.0)])
def test_circle_mixed_dirichlet_neumann(oracle_mod, bc, order):
    """Mixed two-sided IBC (Sec. 4.2): u = 0 on the plus side of tC (psi -> 0+)
    and u' = 0 on the minus side (psi -> 2 pi-).  -u'' + u = f with
    u = cos((psi - 2 pi) / 4), f = (1 + 1/16) u, psi in (0, 2 pi)."""
    tC = 1.022 * math.pi
    hs, errs = [0.04, 0.02, 0.01, 0.005], []
    for h in hs:
        o = oracle_mod.Oracle(ci.circle2d(), h).set_curves([point_on_circle(tC, bc[0], bc[1])])
        # plus-side BC DOFs (cp on the plus side) stand in for the minus side: Neumann rows
        assert np.all(o.bc_type[o.bc_side > 0] == bc[1]) and np.all(o.bc_type[o.bc_side < 0] == bc[0])
        psi = (np.arctan2(o.cp[:, 1], o.cp[:, 0]) - tC) % (2 * math.pi)
        ex = np.cos((psi - 2 * math.pi) / 4)
        u = o.solve_direct(1.0, -1.0, o.rhs((1 + 1 / 16) * ex, np.zeros(o.NC)))
        errs.append(np.max(np.abs(o.extend(u) - ex)))
    p = fit_order(hs, errs)
    assert abs(p - order) < 0.35, (errs, p)


# --- zero-Neumann great circle on the sphere -----------------------------------

def neumann_great_circle(bc):
    """A great circle whose plane normal n is generic, so that no grid node lies
    on it (a closest point on C at a grid node would make that Neumann row
    u_alpha - u_alpha = 0), and a unit p in its plane."""
    n = np.array([0.31, 0.47, 0.83]); n /= np.linalg.norm(n)
    ref = np.cross(n, [1.0, 0.0, 0.0]); ref /= np.linalg.norm(ref)
    return ci.Curve(ci.CV_CIRCLE, bc, (0.0, 0.0, 0.0), nu=tuple(n), rad=1.0, ref=tuple(ref)), ref


def test_sphere_neumann_great_circle_second_order(oracle_mod):
    """-Delta_S u + u = 3u on the unit sphere for u = p.x (Delta_S u = -2u) with a
    second-order zero-Neumann IBC on a great circle through p: its conormal is
    the plane normal n, and grad_S u . n = p . n = 0 there (the zero-Neumann
    setting of Sec. 6.2-6.3)."""
    cv, pdir = neumann_great_circle(ci.BC_NEU2)
    hs, errs = [1 / 8, 1 / 12, 1 / 16], []
    for h in hs:
        o = oracle_mod.Oracle(ci.sphere(), h).set_curves([cv])
        ue = o.cp @ pdir
        u = o.solve_direct(1.0, -1.0, o.rhs(3.0 * ue, np.zeros(o.NC)))
        errs.append(np.max(np.abs(o.extend(u) - ue)))
    assert fit_order(hs, errs) > 1.6, errs
    assert errs[-1] < 5e-3, errs


# --- time stepping with second-order Dirichlet data ----------------------------

def test_cn_heat_dir2_latitudes_with_time_dependent_data(oracle_mod):
    """The heat study of Sec. 6.2: exact exp(-2t) z on the unit sphere, with that
    value prescribed on the latitude circles (second-order Dirichlet rows carry
    2 g(t_{k+1})); second-order decay of the error at t = 0.1."""
    errs, hs = [], (1 / 16, 1 / 32)
    for h in hs:
        o = oracle_mod.Oracle(ci.sphere(), h).set_curves(ci.config2(h, ci.BC_DIR2).curves)
        # BC DOFs start at the smooth continuation of u0 across C (the value at
        # their own closest point), which the second-order rows reproduce to
        # O(h^2); the first step then imposes the rows exactly
        u0 = np.concatenate([o.cp[:, 2], o.cp[o.twin, 2]])
        dt = 0.01
        u = o.heat_cn(u0, dt, 10, g_bc=lambda t: np.exp(-2 * t) * o.cpc[:, 2])
        errs.append(np.abs(o.extend(u) - np.exp(-0.2) * o.cp[:, 2]).max())
    # the second-order IBC error is irregular on coarse grids (Sec. 7); over a
    # factor 2 in h from 1/16 it falls at better than order 1.5
    assert errs[1] < 0.5 ** 1.5 * errs[0], errs
    assert errs[1] < 2e-4, errs
