"""cpm_apply_noalloc against cpm_apply.

cpm_apply_noalloc is the operator product for callers that cannot allocate
device memory while they call it -- a host framework that has already handed
the whole device to its own memory pool (a cudaMalloc would fail), or a
latency-bound caller that cannot afford the device synchronisation that
cudaMalloc/cudaFree imply.  It keeps its intermediate in one fixed array inside
the library.  These tests check its result against cpm_apply on two calls in a
row (the array keeps the previous call's contents) and that an oversized call is
refused.  The file is collected last so that it also runs after every other test
has used the library on the same device."""
import numpy as np
import pytest

import cpm_inputs as ci
from gpu_common import need_gpu


def _band(torch):
    from paper_2305_04711_gb300.cpm import Band
    w = ci.config2(1 / 20, ci.BC_DIR2)
    return Band(w.shape, w.h).set_boundary(w.curves)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nrhs", [1, 20, 40])
def test_noalloc_apply_matches_apply_twice(prec, nrhs):
    torch = need_gpu()
    band = _band(torch)
    dt = torch.float64 if prec == "fp64" else torch.float32
    U = torch.tensor(ci.random_vector(band.N, seed=3, nrhs=nrhs), device="cuda").to(dt)
    if nrhs == 1:
        U = U.reshape(-1).contiguous()
    ref = band.apply(1.0, -0.01, U)
    tol = 1e-14 if prec == "fp64" else 2e-6
    scale = float(ref.abs().max())
    for _ in range(2):   # two calls in a row reuse the same array
        out = torch.full_like(U, float("nan"))
        band.apply_noalloc(1.0, -0.01, U, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert float((out - ref).abs().max()) <= tol * scale
    band.close()


@pytest.mark.gpu
def test_noalloc_apply_rejects_oversize():
    torch = need_gpu()
    from paper_2305_04711_gb300 import _lib as L
    band = _band(torch)
    cap = L.load().cpm_apply_noalloc_max_bytes()
    nrhs = 256
    assert 8 * band.NS * nrhs > cap, "workload too small to exceed the fixed array"
    U = torch.zeros((band.N, nrhs), dtype=torch.float64, device="cuda")
    out = torch.empty_like(U)
    with pytest.raises(L.CpmError) as e:
        band.apply_noalloc(1.0, 1.0, U, out)
    assert e.value.status == "CPM_ERR_CAPACITY"
    band.close()
