"""Pins of the CPU oracle's geometry, band, interpolation and operator against
facts fixed by the paper and by mathematics (not against the oracle itself)."""
import math
import os

import numpy as np
import pytest

import cpm_inputs as ci

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if "=" in line:
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


# --- Eq. (3): tube radius --------------------------------------------------

def test_tube_radius_matches_eq3(oracle_mod):
    g = golden()
    assert g["tube_radius_d2_p3_q1"] == "sqrt(13)" and g["tube_radius_d3_p3_q1"] == "sqrt(17)"
    h = 0.01
    assert oracle_mod.tube_radius(2, h) == pytest.approx(math.sqrt(13.0) * h, rel=1e-15)
    assert oracle_mod.tube_radius(3, h) == pytest.approx(math.sqrt(17.0) * h, rel=1e-15)


# --- closest points (Sec. 3.1, App. A) ---------------------------------------

def test_cp_sphere_circle_torus_geometry(oracle_mod):
    rng = np.random.default_rng(1)
    sph, cir, tor = ci.sphere(1.3), ci.circle2d(), ci.torus(1.0, 0.4)
    for _ in range(200):
        x = rng.uniform(-1.6, 1.6, size=3)
        cp = oracle_mod.closest_point(sph, x)
        # on the surface, and x - cp is radial (normal)
        assert np.linalg.norm(cp) == pytest.approx(1.3, abs=1e-14)
        assert np.linalg.norm(np.cross(x - cp, cp)) < 1e-13
        # and no sampled surface point is closer
        w = rng.normal(size=(64, 3)); w = 1.3 * w / np.linalg.norm(w, axis=1, keepdims=True)
        assert np.linalg.norm(x - cp) <= np.min(np.linalg.norm(w - x, axis=1)) + 1e-14
        x2 = x.copy(); x2[2] = 0
        cp2 = oracle_mod.closest_point(cir, x2[:2])
        assert math.hypot(cp2[0], cp2[1]) == pytest.approx(1.0, abs=1e-15)
        assert abs(cp2[0] * x2[1] - cp2[1] * x2[0]) < 1e-14
        cpt = oracle_mod.closest_point(tor, x)
        # on the torus: (sqrt(x^2+y^2) - R)^2 + z^2 = r^2
        assert (math.hypot(cpt[0], cpt[1]) - 1.0) ** 2 + cpt[2] ** 2 == pytest.approx(0.16, abs=1e-14)
        # distance equals | dist to tube centre circle - r |
        rho = math.hypot(x[0], x[1])
        dc = math.hypot(rho - 1.0, x[2])
        assert np.linalg.norm(x - cpt) == pytest.approx(abs(dc - 0.4), abs=1e-13)


def test_bumpy_phi_derivatives_match_finite_differences(oracle_mod):
    sh = ci.bumpy_sphere(16, seed=0)
    rng = np.random.default_rng(2)
    for _ in range(10):
        x = rng.normal(size=3); x *= rng.uniform(0.8, 1.2) / np.linalg.norm(x)
        phi, g, H = oracle_mod.bumpy_phi(sh, x)
        eps = 1e-5
        gfd = np.zeros(3); Hfd = np.zeros((3, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = eps
            pp, gp, _ = oracle_mod.bumpy_phi(sh, x + e)
            pm, gm, _ = oracle_mod.bumpy_phi(sh, x - e)
            gfd[k] = (pp - pm) / (2 * eps)
            Hfd[:, k] = (gp - gm) / (2 * eps)
        assert np.max(np.abs(g - gfd)) < 1e-8
        assert np.max(np.abs(H - Hfd)) < 1e-6
        # level set really is |x| - rho(x/|x|)
        w = x / np.linalg.norm(x)
        assert phi == pytest.approx(np.linalg.norm(x) - ci.bumpy_radius(sh, w), abs=1e-14)


def test_bumpy_newton_cp_is_a_closest_point(oracle_mod):
    """App. A Newton result: on the level set, x - cp parallel to grad phi, and
    no nearby surface sample is closer."""
    sh = ci.bumpy_sphere(16, seed=0)
    rng = np.random.default_rng(3)
    for _ in range(40):
        w = rng.normal(size=3); w /= np.linalg.norm(w)
        r0 = float(ci.bumpy_radius(sh, w))
        x = w * (r0 + rng.uniform(-0.02, 0.02))
        cp = oracle_mod.closest_point(sh, x)
        phi, g, _ = oracle_mod.bumpy_phi(sh, cp)
        assert abs(phi) < 1e-12
        d = x - cp
        assert np.linalg.norm(np.cross(d, g)) < 1e-10 * max(1.0, np.linalg.norm(g))
        # brute force over a local patch of surface points
        t1 = np.cross(w, [0.3, 0.5, 0.8]); t1 /= np.linalg.norm(t1); t2 = np.cross(w, t1)
        a, b = np.meshgrid(np.linspace(-0.08, 0.08, 41), np.linspace(-0.08, 0.08, 41))
        dirs = w[None, :] + a.reshape(-1, 1) * t1 + b.reshape(-1, 1) * t2
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        pts = dirs * ci.bumpy_radius(sh, dirs)[:, None]
        assert np.linalg.norm(d) <= np.min(np.linalg.norm(pts - x, axis=1)) + 1e-9


def test_circle_curve_closest_point(oracle_mod):
    cv = ci.latitude_circle(math.pi / 3)
    rng = np.random.default_rng(4)
    for _ in range(50):
        x = rng.uniform(-1.2, 1.2, size=3)
        c = oracle_mod.curve_cp(cv, x)
        assert c[2] == pytest.approx(0.5, abs=1e-15)
        assert math.hypot(c[0], c[1]) == pytest.approx(math.sin(math.pi / 3), abs=1e-14)
        ang = np.linspace(0, 2 * math.pi, 2001)
        pts = np.stack([math.sin(math.pi / 3) * np.cos(ang), math.sin(math.pi / 3) * np.sin(ang),
                        0.5 * np.ones_like(ang)], 1)
        assert np.linalg.norm(x - c) <= np.min(np.linalg.norm(pts - x, axis=1)) + 1e-12


# --- Alg. 1 band == brute force over a bounding box --------------------------

@pytest.mark.parametrize("shape,h,box", [
    (ci.circle2d(), 0.05, 26),
    (ci.sphere(), 1.0 / 10, 14),
    (ci.torus(1.0, 0.4), 1.0 / 12, 22),
])
def test_bfs_band_equals_bruteforce(oracle_mod, shape, h, box):
    o = oracle_mod.Oracle(shape, h)
    lo = [-box] * shape.dim
    hi = [box] * shape.dim
    bf = oracle_mod.band_bruteforce(shape, h, lo, hi)
    a = {tuple(r) for r in o.ijk.tolist()}
    b = {tuple(r) for r in bf.tolist()}
    assert a == b
    # every member really is within r of S, and the ordering is canonical
    d = np.linalg.norm(o.x() - o.cp, axis=1)
    assert np.all(d <= o.rband)
    keys = [((z >> 3), (y >> 3), (x >> 3), z & 7, y & 7, x & 7) for x, y, z in o.ijk.tolist()]
    assert keys == sorted(keys)


def test_band_contains_all_interpolation_and_fd_nodes(oracle_mod):
    """Eq. (3) is an upper bound on the nodes needed: every FD neighbour of every
    interpolation node is in the band (sphere, torus, circle)."""
    for shape, h in ((ci.sphere(), 1 / 16), (ci.torus(), 1 / 16), (ci.circle2d(), 0.02)):
        o = oracle_mod.Oracle(shape, h).set_curves([])
        members = {tuple(r) for r in o.ijk.tolist()}
        interp = {tuple(o.ijk[j]) for j in np.unique(o.E.indices)}
        d = shape.dim
        for node in interp:
            for a in range(d):
                for s in (-1, 1):
                    nb = list(node); nb[a] += s
                    assert tuple(nb) in members


# --- barycentric Lagrange weights (Sec. 3.2) ---------------------------------

def product_form(t):
    return np.array([np.prod([(t - k) / (j - k) for k in range(4) if k != j]) for j in range(4)])


def test_barycentric_weights(oracle_mod):
    rng = np.random.default_rng(5)
    for t in list(rng.uniform(1.0, 2.0, 200)) + [1.0, 1.5, 2.0 - 1e-12]:
        w = oracle_mod.bary_weights(t)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.max(np.abs(w - product_form(t))) < 1e-14
        # reproduces every cubic exactly
        c = rng.normal(size=4)
        vals = np.polyval(c, np.arange(4.0))
        assert w @ vals == pytest.approx(np.polyval(c, t), abs=1e-12)
    assert np.array_equal(oracle_mod.bary_weights(1.0), np.array([0.0, 1.0, 0.0, 0.0]))


@pytest.mark.parametrize("shape,h", [(ci.sphere(), 1 / 16), (ci.torus(), 1 / 16), (ci.circle2d(), 0.02)])
def test_E_reproduces_tensor_cubics_at_closest_points(oracle_mod, shape, h):
    """E u for u = P(x) with P a tensor-product cubic equals P(cp_S(x_i)) exactly:
    pins the stencil base, the weights and the node indexing of E."""
    o = oracle_mod.Oracle(shape, h).set_curves([])
    rng = np.random.default_rng(6)
    cx, cy, cz = rng.normal(size=(3, 4))

    def P(p):
        v = np.polyval(cx, p[:, 0]) * np.polyval(cy, p[:, 1])
        return v * np.polyval(cz, p[:, 2]) if shape.dim == 3 else v

    u = P(o.x())
    eu = o.extend(u)
    assert np.max(np.abs(eu - P(o.cp))) < 1e-11 * max(1.0, np.max(np.abs(u)))


# --- operator M (Sec. 5.3) ---------------------------------------------------

def test_M_annihilates_constants_on_complete_rows(oracle_mod):
    for shape, h in ((ci.sphere(), 1 / 16), (ci.circle2d(), 0.02), (ci.torus(), 1 / 16)):
        o = oracle_mod.Oracle(shape, h).set_curves([])
        M = o.M()
        r = M @ np.ones(o.N)
        complete = np.diff(o.Loff.indptr) == 2 * shape.dim
        assert np.max(np.abs(r[complete])) < 1e-9 / h ** 2 * 1e-3
        # incomplete (band edge) rows are exactly short of the missing 1/h^2 terms
        miss = 2 * shape.dim - np.diff(o.Loff.indptr)
        assert np.allclose(r, -miss / h ** 2, atol=1e-8)


def test_M_on_sphere_harmonic_is_eigen_relation_second_order(oracle_mod):
    """For u = Y_l^m(cp_S(x)) (the CP extension), (M u)_i ~ -l(l+1) Y(cp_i)/|x_i|^2
    (Laplacian of a degree-0 homogeneous extension) with an O(h^2) error."""
    errs, hs = [], [1 / 10, 1 / 14, 1 / 20, 1 / 28]
    l, m = 4, 2
    for h in hs:
        o = oracle_mod.Oracle(ci.sphere(), h).set_curves([])
        y = ci.real_ylm(l, m, o.cp)
        Mu = o.M() @ y
        x2 = np.sum(o.x() ** 2, axis=1)
        target = -l * (l + 1) * y / x2
        interior = np.diff(o.Loff.indptr) == 6
        errs.append(np.max(np.abs(Mu - target)[interior]))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert slope > 1.7, (errs, slope)
    assert errs[-1] < 0.5
