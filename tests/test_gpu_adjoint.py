"""Adjoint path on the GPU against the oracle: the transposed product A^T u
(FP64 and FP32, single and batched), the duality <A x, y> = <x, A^T y>, the
adjoint solve, the boundary gradient B^T (c lambda_C), and the autograd
wrapper's gradient against central differences of the (quadratic) loss."""
import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import SMALL, need_gpu, pair, rel_inf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["circle_dir2", "sphere_lat_dir2", "torus_mer_dir2", "sphere_point_dir1"])
@pytest.mark.parametrize("nrhs", [1, 5, 40])
def test_transpose_product_matches_oracle(oracle_mod, name, nrhs):
    torch = need_gpu()
    band, ref = pair(oracle_mod, SMALL[name]())
    U = ci.random_vector(ref.N, seed=21 + nrhs, nrhs=nrhs)
    VR = ref.A(1.0, -0.02).T.tocsr() @ U
    u = torch.tensor(U, device="cuda")
    V = band.apply(1.0, -0.02, u, transpose=True).cpu().numpy()
    V32 = band.apply(1.0, -0.02, u.float(), transpose=True).cpu().numpy()
    VR2, V2 = VR.reshape(ref.N, -1), V.reshape(ref.N, -1)
    for r in range(VR2.shape[1]):
        assert rel_inf(V2[:, r], VR2[:, r]) < 1e-14
    assert np.max(np.abs(V32 - VR)) <= 2e-6 * np.max(np.abs(VR))


def test_duality_on_a_larger_band():
    torch = need_gpu()
    from paper_2305_04711_gb300.cpm import Band
    w = ci.config2(1 / 64, ci.BC_DIR2)
    band = Band(w.shape, w.h).set_boundary(w.curves)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand((band.N, 3), generator=g, device="cuda", dtype=torch.float64)
    y = torch.rand((band.N, 3), generator=g, device="cuda", dtype=torch.float64)
    Ax = band.apply(0.3, 1.0, x)
    ATy = band.apply(0.3, 1.0, y, transpose=True)
    lhs, rhs = (Ax * y).sum(0), (x * ATy).sum(0)
    scale = (Ax.abs() * y.abs()).sum(0)
    assert float(((lhs - rhs).abs() / scale).max()) < 1e-13


@pytest.mark.parametrize("name", ["circle_dir2", "sphere_lat_dir1", "torus_mer_dir2"])
def test_adjoint_solve_matches_oracle_direct(oracle_mod, name):
    torch = need_gpu()
    w = SMALL[name]()
    band, ref = pair(oracle_mod, w)
    y = np.zeros(ref.N)
    y[:ref.NS] = ci.random_vector(ref.NS, seed=4)
    lam, st = band.solve(w.m, w.n, torch.tensor(y, device="cuda"), tol=1e-14, adjoint=True, raise_on_error=False)
    # the right-preconditioned adjoint iteration stops at its attainable accuracy
    assert st.relres < 1e-10, st
    lr = ref.solve_adjoint_direct(w.m, w.n, y)
    assert rel_inf(lam.cpu().numpy(), lr) < 1e-10


def test_boundary_gradient_and_autograd_against_oracle_and_differences(oracle_mod):
    torch = need_gpu()
    from paper_2305_04711_gb300.autograd import cpm_solve
    h = 1 / 12
    w, samples, coef = ci.config4(h, nsamples=64, seed=0)
    band, ref = pair(oracle_mod, w, n_samples=[len(samples)])
    target = torch.tensor(ci.target_field(coef, ref.cp), device="cuda")
    s_dev = torch.tensor(samples, device="cuda", requires_grad=True)

    def loss_of(sv):
        u = cpm_solve(band, 0.0, 1.0, None, sv, tol=1e-11)
        return 0.5 * ((u[:band.NS] - target) ** 2).sum()

    L = loss_of(s_dev)
    L.backward()
    grad = s_dev.grad.cpu().numpy()
    # oracle gradient: B^T (c lambda_C) with A^T lambda = [u_S - t ; 0]
    B = ref.sample_matrix([len(samples)])
    c = ref.bc_scale()
    u0 = ref.solve_direct(0.0, 1.0, ref.rhs(None, B @ samples))
    rhs = np.zeros(ref.N)
    rhs[:ref.NS] = u0[:ref.NS] - ci.target_field(coef, ref.cp)
    lam = ref.solve_adjoint_direct(0.0, 1.0, rhs)
    g_ref = B.T @ (c * lam[ref.NS:])
    assert rel_inf(grad, g_ref) < 1e-8
    # the loss is quadratic in the samples: central differences are exact up to
    # rounding for any step, so a large step keeps solver round-off out
    rng = np.random.default_rng(2)
    eps = 1.0
    with torch.no_grad():
        for k in rng.choice(len(samples), size=6, replace=False):
            e = torch.zeros_like(s_dev)
            e[k] = eps
            fd = (float(loss_of(s_dev + e)) - float(loss_of(s_dev - e))) / (2 * eps)
            denom = max(abs(grad[k]), 1e-3 * np.max(np.abs(grad)))
            assert abs(fd - grad[k]) / denom < 1e-6
