"""Shared helpers of the GPU parity tests (CUDA library vs CPU oracle)."""
import numpy as np
import pytest

import cpm_inputs as ci


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def pair(oracle_mod, workload, n_samples=None, p=3):
    """(GPU band, oracle) for the same workload, boundary set on both."""
    from paper_2305_04711_gb300.cpm import Band
    band = Band(workload.shape, workload.h, p=p).set_boundary(workload.curves, n_samples)
    ref = oracle_mod.Oracle(workload.shape, workload.h, p=p).set_curves(workload.curves)
    return band, ref


def rel_inf(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


SMALL = {
    "circle_dir1": lambda: ci.config1(0.02, ci.BC_DIR1),
    "circle_dir2": lambda: ci.config1(0.01, ci.BC_DIR2),
    "sphere_lat_dir1": lambda: ci.config2(1 / 16, ci.BC_DIR1),
    "sphere_lat_dir2": lambda: ci.config2(1 / 20, ci.BC_DIR2),
    "torus_mer_dir2": lambda: ci.Workload("torus2", ci.torus(1.0, 0.4), 1 / 16,
                                          [ci.torus_meridian(0.3, 1.0, 0.4, ci.BC_DIR2),
                                           ci.torus_meridian(2.5, 1.0, 0.4, ci.BC_DIR1)], 0.0, 1.0),
    "sphere_point_dir1": lambda: ci.Workload("spt", ci.sphere(), 1 / 16, [ci.point_curve((0.0, 0.0, 1.0))], 1.0,
                                             -1 / 16),
    "sphere_closed": lambda: ci.Workload("sph0", ci.sphere(), 1 / 12, [], 1.0, 1.0),
}
