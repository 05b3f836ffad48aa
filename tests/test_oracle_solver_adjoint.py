"""Pins of the oracle's solver paths and adjoint: the four-step matrix-free
product (Sec. 5.4) against the assembled A, BiCGSTAB against a direct LU
solve, and the adjoint gradient against central finite differences."""
import math

import numpy as np
import pytest

import cpm_inputs as ci


@pytest.mark.parametrize("m,n", [(0.0, 1.0), (1.0, -0.05), (1.0, 1.0)])
def test_four_step_product_equals_assembled_A(oracle_mod, m, n):
    for w in (ci.config1(0.02, ci.BC_DIR2), ci.config2(1 / 16, ci.BC_DIR2)):
        o = oracle_mod.Oracle(w.shape, w.h).set_curves(w.curves)
        u = ci.random_vector(o.N, seed=7)
        v = o.apply(m, n, u)
        ref = o.A(m, n) @ u
        assert np.max(np.abs(v - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_bicgstab_matches_direct_solve(oracle_mod):
    w = ci.config2(1 / 12, ci.BC_DIR2)
    o = oracle_mod.Oracle(w.shape, w.h).set_curves(w.curves)
    f = o.rhs(ci.random_vector(o.NS, seed=3), np.where(o.bc_curve == 0, 0.0, 1.0))
    xd = o.solve_direct(0.0, 1.0, f)
    xi, it, rr = o.bicgstab(0.0, 1.0, f, tol=1e-13)
    assert rr <= 1e-13
    assert np.max(np.abs(xi - xd)) <= 1e-9 * np.max(np.abs(xd))


def test_adjoint_gradient_matches_central_differences(oracle_mod):
    """loss = 1/2 sum_{i in J_S} (u_i - target_i)^2 with Dirichlet samples s on a
    circle as parameters: dL/ds = B^T diag(c) lambda_C with A^T lambda = [u_S - t; 0].
    The loss is quadratic in s, so central differences are exact up to rounding."""
    h = 1 / 10
    w, samples, coef = ci.config4(h, nsamples=64, seed=0)
    o = oracle_mod.Oracle(w.shape, h).set_curves(w.curves)
    B = o.sample_matrix([len(samples)])
    c = o.bc_scale()
    target = ci.target_field(coef, o.cp)
    A = o.A(0.0, 1.0)
    import scipy.sparse.linalg as spla
    lu, luT = spla.splu(A.tocsc()), spla.splu(A.T.tocsc())

    def loss(s):
        u = lu.solve(o.rhs(None, B @ s))
        return 0.5 * np.sum((u[:o.NS] - target) ** 2), u

    L0, u0 = loss(samples)
    rhs = np.zeros(o.N)
    rhs[:o.NS] = u0[:o.NS] - target
    lam = luT.solve(rhs)
    grad = B.T @ (c * lam[o.NS:])
    rng = np.random.default_rng(11)
    idx = rng.choice(len(samples), size=8, replace=False)
    eps = 1e-6
    for k in idx:
        e = np.zeros(len(samples)); e[k] = eps
        fd = (loss(samples + e)[0] - loss(samples - e)[0]) / (2 * eps)
        denom = max(abs(grad[k]), 1e-3 * np.max(np.abs(grad)))
        assert abs(fd - grad[k]) / denom < 1e-6
