"""Timing of the operator product A u (cpm_apply) alone, for kernel work.

    python -m paper_2305_04711_gb300.microbench [--workload sphere|torus|circle|bumpy]
        [--h H] [--nrhs R] [--prec fp32|fp64] [--iters K] [--warmup W] [--transpose]
        [--autotune] [--single-mode M]

Builds the band and boundary of a workload (the sphere at h = 1/128 with two
Dirichlet latitude circles by default), fills u with seeded uniform values and
times K products with CUDA events on the launching stream, after W untimed
ones.  Prints one JSON line: per-product milliseconds (median, min) and the
per-kernel split reported by the library's profiler.  Every product runs in the
library's kernels; this module only sets up inputs and reads clocks.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def workload(kind: str, h: float):
    import cpm_inputs as ci
    if kind == "sphere":
        return ci.config2(h or 1.0 / 128, ci.BC_DIR1)
    if kind == "torus":
        w, _, _ = ci.config3(h=h or 1.0 / 256, ncurves=8, nrhs=1, seed=0, min_gap=0.2)
        return w
    if kind == "bumpy":
        # the bumpy sphere of the heat-method workload (16 seeded Gaussian bumps),
        # no interior boundary
        return ci.Workload("bumpy", ci.bumpy_sphere(16, seed=0), h or 1.0 / 640, [], 0.0, 1.0)
    return ci.config1(h or 0.01, ci.BC_DIR2)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sphere", choices=["sphere", "torus", "circle", "bumpy"])
    ap.add_argument("--h", type=float, default=0.0)
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--transpose", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="run cpm_autotune for this width first")
    ap.add_argument("--single-mode", type=int, default=-1, help="fix the single right-hand side form (0, 1, 2)")
    a = ap.parse_args(argv)

    import torch
    from paper_2305_04711_gb300 import Band

    w = workload(a.workload, a.h)
    band = Band(w.shape, w.h).set_boundary(w.curves)
    dt = torch.float32 if a.prec == "fp32" else torch.float64
    tune = band.autotune(a.nrhs, dt) if a.autotune else None
    if a.single_mode >= 0:
        band.set_tune(a.nrhs, dt, single_mode=a.single_mode)
    g = torch.Generator(device="cuda").manual_seed(0)
    shape = (band.N,) if a.nrhs == 1 else (band.N, a.nrhs)
    u = torch.rand(shape, generator=g, device="cuda", dtype=torch.float64).to(dt)
    v = torch.empty_like(u)
    st = torch.cuda.current_stream()
    for _ in range(a.warmup):
        band.apply(0.0, 1.0, u, out=v, transpose=a.transpose)
    torch.cuda.synchronize()
    times = []
    band.profile(True)
    for _ in range(a.iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        band.apply(0.0, 1.0, u, out=v, transpose=a.transpose)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    prof = band.profile(False)
    times.sort()
    print(json.dumps({"workload": a.workload, "h": w.h, "N": band.N, "NS": band.NS, "NC": band.NC,
                      "nrhs": a.nrhs, "prec": a.prec, "transpose": a.transpose,
                      "ms_median": times[len(times) // 2], "ms_min": times[0],
                      "special_rows": band.diagnostics()["special_rows"], "profile": prof, "tune": tune}))
    band.close()


if __name__ == "__main__":
    main()
