"""Pins of the oracle's projected crossing test (Sec. 4.7): the crossing vector
cp_{S-C}(x) with its components along the surface normal n_S and the curve
tangent t_C (both at cp_C(x)) removed.

What fixes it independently of the oracle's own formula:
  * geometry: on the unit sphere the projected vector of a node near a circle C
    lies along C's conormal (the direction in S normal to C) -- e_theta for a
    latitude circle, the plane normal for a great circle -- and its sign along
    the conormal is the side of cp_S(x) (the sign of theta - theta_C);
  * on a point C of the unit circle (2D) it is the tangential part of
    cp_S(x) - C, whose sign is that of the angle from C;
  * the method: with the projected test the latitude-circle Laplace problem
    keeps its closed form and its convergence orders (first / second order
    Dirichlet rows), as with the plain test (Sec. 6)."""
import math

import numpy as np
import pytest

import cpm_inputs as ci
from test_oracle_ibc import exact_latitudes, fit_order, solve


def _projected(curves):
    out = []
    for cv in curves:
        cv.projected = True
        out.append(cv)
    return out


def test_latitude_circle_vectors_lie_along_e_theta(oracle_mod):
    h = 1 / 24
    w = ci.config2(h, ci.BC_DIR1)
    o = oracle_mod.Oracle(w.shape, h).set_curves(_projected(w.curves))
    th_c = (math.pi / 4, 3 * math.pi / 4)
    checked = 0
    for i in np.nonzero(o.near_c >= 0)[0][::7]:
        k = int(o.near_c[i])
        z = o.crossing_vector(k, i)
        x = h * o.ijk[i].astype(float)
        # cp_C of a latitude circle: the point of C at the node's longitude
        phi = math.atan2(x[1], x[0])
        cc = np.array([math.sin(th_c[k]) * math.cos(phi), math.sin(th_c[k]) * math.sin(phi), math.cos(th_c[k])])
        e_th = np.array([math.cos(th_c[k]) * math.cos(phi), math.cos(th_c[k]) * math.sin(phi), -math.sin(th_c[k])])
        if np.linalg.norm(o.cp[i] - cc) < 0.2 * h * h:
            continue  # cp_S on C: the node takes a stencil neighbour's vector (Sec. 4.2 tie)
        assert abs(np.dot(z, cc)) < 1e-12 and np.linalg.norm(np.cross(z, e_th)) < 1e-12 * max(1.0, np.linalg.norm(z))
        th_s = math.acos(max(-1.0, min(1.0, o.cp[i, 2])))
        assert np.sign(np.dot(z, e_th)) == np.sign(th_s - th_c[k])
        checked += 1
    assert checked > 50


def test_great_circle_vectors_lie_along_the_plane_normal(oracle_mod):
    n = np.array([0.31, 0.47, 0.83]); n /= np.linalg.norm(n)
    ref = np.cross(n, [1.0, 0.0, 0.0]); ref /= np.linalg.norm(ref)
    cv = ci.Curve(ci.CV_CIRCLE, ci.BC_DIR1, (0.0, 0.0, 0.0), nu=tuple(n), rad=1.0, ref=tuple(ref), projected=True)
    h = 1 / 16
    o = oracle_mod.Oracle(ci.sphere(), h).set_curves([cv])
    checked = 0
    for i in np.nonzero(o.near_c >= 0)[0][::5]:
        z = o.crossing_vector(0, int(i))
        if abs(np.dot(o.cp[i], n)) < 0.2 * h * h:
            continue  # cp_S on C (Sec. 4.2 tie)
        assert np.linalg.norm(np.cross(z, n)) < 1e-12 * max(1.0, np.linalg.norm(z))
        assert np.sign(np.dot(z, n)) == np.sign(np.dot(o.cp[i], n))
        checked += 1
    assert checked > 50


def test_circle_point_vectors_are_tangential(oracle_mod):
    tc = 1.022 * math.pi
    c = np.array([math.cos(tc), math.sin(tc), 0.0])
    tang = np.array([-math.sin(tc), math.cos(tc), 0.0])
    cv = ci.Curve(ci.CV_POINT, ci.BC_DIR1, tuple(c), nu=tuple(tang), projected=True)
    h = 0.01
    o = oracle_mod.Oracle(ci.circle2d(), h).set_curves([cv])
    checked = 0
    for i in np.nonzero(o.near_c >= 0)[0]:
        z = o.crossing_vector(0, int(i))
        if np.linalg.norm(o.cp[i] - c) < 0.2 * h * h:
            continue  # cp_S on C (Sec. 4.2 tie)
        assert abs(np.dot(z, c)) < 1e-15 and abs(z[2]) == 0.0
        ang = math.atan2(o.cp[i, 1], o.cp[i, 0]) - tc
        ang = (ang + math.pi) % (2 * math.pi) - math.pi
        assert np.sign(np.dot(z, tang)) == np.sign(ang)
        checked += 1
    assert checked > 10


@pytest.mark.parametrize("bc,order", [(ci.BC_DIR1, 1.0), (ci.BC_DIR2, 2.0)])
def test_projected_latitude_circles_keep_the_closed_form_and_order(oracle_mod, bc, order):
    hs, errs, same = [1 / 16, 1 / 24, 1 / 32], [], []
    for h in hs:
        w = ci.config2(h, bc)
        o = oracle_mod.Oracle(w.shape, h).set_curves(_projected(w.curves))
        g = np.where(o.bc_curve == 0, 0.0, 1.0)
        u = solve(o, 0.0, 1.0, o.rhs(np.zeros(o.NS), g))
        errs.append(np.max(np.abs(o.extend(u) - exact_latitudes(o.cp))))
        # on the smooth sphere the plain test already decides by the conormal
        # side, so both tests assemble the same operator here
        o2 = oracle_mod.Oracle(w.shape, h).set_curves(ci.config2(h, bc).curves)
        same.append(abs(o.A(0.0, 1.0) - o2.A(0.0, 1.0)).max())
    assert abs(fit_order(hs, errs) - order) < 0.45, errs
    assert max(same) == 0.0, same


def test_torus_meridian_vectors_lie_along_the_toroidal_direction(oracle_mod):
    """A meridian phi = phi0 of the torus: its conormal in S is the toroidal
    direction e_phi = (-sin phi0, cos phi0, 0) all along it."""
    R, rt, p0 = 1.0, 0.4, 0.3
    cv = ci.torus_meridian(p0, R, rt, ci.BC_DIR1)
    cv.projected = True
    h = 1 / 16
    o = oracle_mod.Oracle(ci.torus(R, rt), h).set_curves([cv])
    e_phi = np.array([-math.sin(p0), math.cos(p0), 0.0])
    checked = 0
    for i in np.nonzero(o.near_c >= 0)[0][::3]:
        z = o.crossing_vector(0, int(i))
        dphi = (math.atan2(o.cp[i, 1], o.cp[i, 0]) - p0 + math.pi) % (2 * math.pi) - math.pi
        if abs(dphi) * R < 0.5 * h * h:
            continue  # cp_S on C (Sec. 4.2 tie)
        assert np.linalg.norm(np.cross(z, e_phi)) < 1e-12 * max(1.0, np.linalg.norm(z))
        assert np.sign(np.dot(z, e_phi)) == np.sign(dphi)
        checked += 1
    assert checked > 50


def test_bumpy_point_vectors_are_tangent_to_the_surface(oracle_mod):
    """A point C on the bumpy sphere: only n_S is projected out, so every vector
    is orthogonal to the level-set gradient at C (App. A)."""
    sh = ci.bumpy_sphere(16, seed=0)
    d = np.array([0.0, 0.6, 0.8])
    c = d * float(ci.bumpy_radius(sh, d))
    cv = ci.point_curve(tuple(c), ci.BC_DIR1)
    cv.projected = True
    h = 1 / 24
    o = oracle_mod.Oracle(sh, h).set_curves([cv])
    # the gradient of phi(x) = |x| - rho(x/|x|) at C by central differences
    def phi(x):
        return np.linalg.norm(x) - float(ci.bumpy_radius(sh, x / np.linalg.norm(x)))
    eps = 1e-6
    g = np.array([(phi(c + eps * e) - phi(c - eps * e)) / (2 * eps) for e in np.eye(3)])
    n = g / np.linalg.norm(g)
    checked = 0
    for i in np.nonzero(o.near_c >= 0)[0]:
        z = o.crossing_vector(0, int(i))
        if np.linalg.norm(o.cp[i] - c) < 0.2 * h * h:
            continue
        assert abs(np.dot(z, n)) < 1e-8 * max(1.0, np.linalg.norm(z))
        checked += 1
    assert checked > 20
