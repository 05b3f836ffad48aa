#!/usr/bin/env python
"""Benchmark of the CPM hot path on GB300: batched FP32 + FP64-refinement solves
against plain FP64 solves.

Default workload (one step), the unit-sphere configuration at h = 1/128
(about 1.76M DOFs): the Dirichlet latitude circles theta = pi/4 and 3 pi/4
with a batch of 64 Poisson problems -Delta_S u = l(l+1) Y_l^m, the circles
carrying Y_l^m, for the first 64 real spherical harmonics with 1 <= l <= 8
(the exact solution of column k is Y_l^m itself).  One step solves the 64
together by mixed-precision iterative refinement (FP32 BiCGSTAB inner solves, FP64
residuals and solution) to a Jacobi-scaled
relative residual of 1e-10.  The metric is seconds per right-hand side.
Alongside: the plain FP64 solve of one right-hand side of the same workload,
the single-RHS operator product's algorithmic bandwidth against the measured
HBM peak, the dominant kernel's roofline (timed live during the timed region by
the library's event pairs), an end-to-end number through host buffers, and the
CPU oracle as baseline.  --workload torus runs the torus batch instead
(R = 1, r = 0.4, h = 1/256, 8 meridians, 64 right-hand sides U[0,1]).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one process per GPU): every rank solves its own batch, with no
communication (the path does not shard); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve s/RHS to 1e-10 (FP64 vs FP32+refine, batched); cpm_apply GB/s vs HBM"
NRHS = 64
TOL = 1e-10
# algorithmic work of one operator product per PDE row (and right-hand side):
# bytes: FP32 u, v (4 + 4) + FP32 fractions t (12) + packed stencil base (4);
#        FP64 u, v (8 + 8) + FP64 t (24) + base (4)
BYTES_ROW_FP32 = 24.0
BYTES_ROW_FP64 = 44.0
# flops per row and right-hand side of the FP32 product: 84 FMA of the separable
# 4x4x4 gather (168), 64 difference subtractions, 14 for the 7-point combine
FLOPS_ROW_RHS_FP32 = 246.0
SMS, FP32_LANES = 152, 128


def max_over_ranks(ms: float) -> float:
    """The slowest rank's time (all ranks get it); the value itself without a
    process group.  Replicas share nothing else: no collective on the data path."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(ms)
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_rhs(ms: float, steps: int, nrhs: int, world: int) -> float:
    """Whole-job metric: wall time of the timed steps over every right-hand side
    that all ranks solved in them (weak scaling: each rank solves its own batch)."""
    return (ms / 1000.0) / (steps * nrhs * world)


def profiled_traffic():
    """DRAM bytes per batched product from the committed ncu summary (None if absent)."""
    import re
    p = os.path.join(ROOT, "profiles", "batched_product_sphere128_64rhs.md")
    try:
        m = re.search(r"traffic_bytes_per_product:\s*(\d+)", open(p).read())
        return int(m.group(1)) if m else None
    except OSError:
        return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere", choices=["sphere", "torus"])
    ap.add_argument("--h", type=float, default=0.0, help="grid spacing (0: the workload's own)")
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def ylm_pairs(n):
    out = []
    for l in range(1, 9):
        for m in range(-l, l + 1):
            out.append((l, m))
    return out[:n]


class Workload:
    """The benchmark problem: geometry, boundary, and a batch of right-hand
    sides built through the library (cpm_rhs) from per-BC-DOF values."""

    def __init__(self, kind, h):
        import cpm_inputs as ci
        self.kind = kind
        if kind == "sphere":
            self.h = h or 1.0 / 128
            self.w = ci.config2(self.h, ci.BC_DIR1)
            self.n_samples = None
        else:
            self.h = h or 1.0 / 256
            self.w, self.ang, self.g = ci.config3(h=self.h, ncurves=8, nrhs=NRHS, seed=0, min_gap=0.2)
            self.n_samples = [1] * len(self.w.curves)

    def describe(self, N=None):
        if self.kind == "sphere":
            wl = (f"unit sphere, h=1/{round(1 / self.h)}, Dirichlet circles theta=pi/4, 3pi/4; {NRHS} Poisson "
                  f"problems -Delta u = l(l+1) Y_l^m with the circles carrying Y_l^m (first {NRHS} real harmonics, "
                  f"1<=l<=8); batched mixed-precision refinement (FP32 BiCGSTAB inner solves, FP64 residuals) to a Jacobi-scaled relative residual "
                  f"of {TOL:g}")
        else:
            wl = (f"torus R=1 r=0.4, h=1/{round(1 / self.h)}, 8 Dirichlet meridians (seeded angles, min gap 0.2 "
                  f"rad), {NRHS} right-hand sides U[0,1]; batched mixed-precision refinement (FP32 BiCGSTAB inner solves) to a "
                  f"Jacobi-scaled relative residual of {TOL:g}")
        d = {"workload": wl, "nrhs": NRHS, "tol": TOL, "norm": "Jacobi-scaled residual",
             "l2": "inputs larger than L2 (each [N][64] Krylov vector is several hundred MB vs 129 MB L2)"}
        if N is not None:
            d["N"] = int(N)
        return d

    def host_inputs(self, band):
        """(s [NS][64] or None, g [NC][64]) as host arrays; for the sphere from
        the exported closest points (input data only)."""
        import numpy as np
        import torch
        import cpm_inputs as ci
        if self.kind == "torus":
            return None, None
        _, cp = band.export_band()
        cpc = band.export_boundary()["cpc"].cpu().numpy()
        cp = cp.cpu().numpy()
        s = np.zeros((band.NS, NRHS))
        g = np.zeros((band.NC, NRHS))
        for k, (l, m) in enumerate(ylm_pairs(NRHS)):
            # M u = -f with f = l(l+1) Y: source of the row equations (m=0, n=1)
            s[:, k] = -l * (l + 1) * ci.real_ylm(l, m, cp)
            g[:, k] = ci.real_ylm(l, m, cpc)
        return s, g

    def exact(self, band, col):
        import cpm_inputs as ci
        _, cp = band.export_band()
        l, m = ylm_pairs(NRHS)[col]
        return ci.real_ylm(l, m, cp.cpu().numpy())


# --------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1])); mx.append(float(f[2]))
                except ValueError:
                    continue
                for k, nm in enumerate(names):
                    if f[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
def cpu_baseline_sample(kind):
    """The oracle as it stands (plain C, OpenMP) on the same workload at a
    coarser grid sized for tens of seconds of CPU work: band, assembly and one
    BiCGSTAB solve of one right-hand side to 1e-10.  Returns its time per DOF
    per iteration, used to project s/RHS to the full workload."""
    import numpy as np
    import cpm_inputs as ci
    from oracle import oracle as O
    O.build()
    h = 1.0 / 48 if kind == "sphere" else 1.0 / 64
    wl = Workload(kind, h)
    t0 = time.perf_counter()
    o = O.Oracle(wl.w.shape, h).set_curves(wl.w.curves)
    t_setup = time.perf_counter() - t0
    if kind == "sphere":
        f = o.rhs(-2 * 3 * ci.real_ylm(2, 1, o.cp), ci.real_ylm(2, 1, o.cpc))
    else:
        f = o.rhs(np.zeros(o.NS), wl.g[:, 0][o.bc_curve])
    t0 = time.perf_counter()
    x, it, rr = o.bicgstab(0.0, 1.0, f, tol=TOL, maxit=20000)
    t_solve = time.perf_counter() - t0
    return {"N": o.N, "h": h, "iters": it, "relres": rr, "t_solve": t_solve, "t_setup": t_setup,
            "s_per_dof_iter": t_solve / (o.N * max(it, 1)), "cores": O.n_threads()}


def run_reference(args):
    """--impl reference: the CPU oracle, each step a bounded sample of the
    workload (see cpu_baseline_sample), projected to s/RHS of the full one:
    the band grows like h^-2 and BiCGSTAB's iteration count like 1/h."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = Workload(args.workload, args.h)
    samples = []
    for k in range(args.warmup + args.steps):
        s = cpu_baseline_sample(args.workload)
        if k >= args.warmup:
            samples.append(s)
    s = samples[-1]
    n_full = s["N"] * (s["h"] / wl.h) ** 2
    it_full = s["iters"] * s["h"] / wl.h
    per = sum(x["s_per_dof_iter"] for x in samples) / len(samples)
    value = per * n_full * it_full
    sample = (f"oracle BiCGSTAB solve of 1 RHS on the same geometry at h=1/{round(1 / s['h'])} ({s['N']} DOF, "
              f"{s['iters']} iterations, {s['t_solve']:.1f} s); time per DOF-iteration scaled to {n_full:.3g} DOF x "
              f"{it_full:.0f} iterations (band ~ h^-2, iterations ~ 1/h)")
    line = {"metric": METRIC, "value": value, "unit": "s/RHS", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(x["t_solve"] for x in samples) / len(samples), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": wl.describe(),
            "cpu_baseline": {"value": value, "unit": "s/RHS", "cores": s["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s/RHS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2305_04711_gb300.cpm import Band

    def log(msg):
        if rank == 0:
            sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg}\n")
            sys.stderr.flush()

    wl = Workload(args.workload, args.h)
    band = Band(wl.w.shape, wl.h).set_boundary(wl.w.curves, n_samples=wl.n_samples)
    log(f"band N={band.N} (NS={band.NS}, NC={band.NC})")
    s_host, g_host = wl.host_inputs(band)
    if args.workload == "torus":
        h_in = torch.tensor(wl.g, dtype=torch.float64).contiguous()   # [8][64] samples

        def make_rhs(dev_in):
            return band.rhs(samples=dev_in, nrhs=NRHS)
    else:
        h_in = torch.tensor(np.concatenate([s_host, g_host], axis=0), dtype=torch.float64).contiguous()

        def make_rhs(dev_in):
            return band.rhs(s=dev_in[:band.NS].contiguous(), g=dev_in[band.NS:].contiguous(), nrhs=NRHS)
    d_in = h_in.to("cuda")
    F = make_rhs(d_in)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            torch.distributed.barrier()

    def step(fb):
        return band.solve(0.0, 1.0, fb, tol=TOL, mode="fp32_ir", maxit=args.maxit, raise_on_error=False)

    stats = []
    for k in range(args.warmup):
        t0 = time.perf_counter()
        x, st = step(F)
        torch.cuda.synchronize()
        stats.append(st)
        log(f"warmup {k}: {time.perf_counter() - t0:.2f} s {st}")
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    band.profile(True)
    with Clocks(local) as clk:
        barrier()
        ev0.record()
        for _ in range(args.steps):
            x, st = step(F)
            stats.append(st)
        ev1.record()
        barrier()
    prof = band.profile(False)
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    log(f"timed: {ms / args.steps:.1f} ms/step {stats[-1]}")
    ms_per_step = ms / args.steps
    value = seconds_per_rhs(ms, args.steps, NRHS, world)
    clocks = clk.summary()
    hbm, sm_max, peak_src = peaks()

    # e2e through host buffers: per step the inputs come from pinned host memory,
    # the right-hand sides are built and solved on the device, and the solution
    # goes back to pinned host memory
    h_pin = h_in.pin_memory()
    h_x = torch.empty((band.N, NRHS), dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        d_in = h_pin.to("cuda", non_blocking=True)
        fb = make_rhs(d_in)
        x, st = step(fb)
        h_x.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    log(f"e2e: {e2e_s / args.steps:.2f} s/step")
    e2e = {"value": e2e_s / (args.steps * NRHS * world), "unit": "s/RHS",
           "h2d_bytes_per_step": int(h_pin.numel() * 8), "d2h_bytes_per_step": int(h_x.numel() * 8)}

    line = {"metric": METRIC, "value": value, "unit": "s/RHS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 solution, residual and refinement)", "data": "synthetic",
            "config": wl.describe(band.N), "clocks": clocks, "e2e": e2e, "gpu_launches": int(prof["launches"])}
    if rank == 0:
        last = stats[-1]
        line["solve"] = {"iterations": last.iterations, "fp64_iterations": last.fp64_iterations,
                         "refinements": last.refinements, "relres_max": last.relres, "status": last.status}
        # roofline of the dominant kernel, the batched FP32 product: the products
        # of the timed region mix it with the FP64 residual / finish products, so
        # it is timed by its own event series right after the timed region, on the
        # same band and batch width
        step_mean_ms = prof["apply_ms"] / max(prof["applies"], 1)
        peak_tf = SMS * FP32_LANES * 2 * sm_max * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": None, "peak": peak_tf, "unit": "TFLOP/s", "frac": None,
                "traffic": profiled_traffic(),
                "kernel": f"batched FP32 operator product (gather_cells + correct + combine_batched), {NRHS} RHS",
                "peak_source": f"FP32 lanes x SMs x 2 x max SM clock ({sm_max:.0f} MHz), derived",
                "products_share_of_step": prof["apply_ms"] / ms if ms > 0 else None,
                "step_products": prof["applies"] // max(args.steps, 1), "step_mean_product_ms": step_mean_ms}
        try:
            u32 = torch.rand((band.N, NRHS), dtype=torch.float32, device="cuda")
            v32 = torch.empty_like(u32)
            for _ in range(3):
                band.apply(0.0, 1.0, u32, out=v32)
            band.profile(True)
            for _ in range(20):
                band.apply(0.0, 1.0, u32, out=v32)
            p2 = band.profile(False)
            per_ms = p2["apply_ms"] / p2["applies"]
            achieved_tf = FLOPS_ROW_RHS_FP32 * band.NS * NRHS / (per_ms * 1e-3) / 1e12
            roof.update({"achieved": achieved_tf, "frac": achieved_tf / peak_tf, "launch_ms": per_ms,
                         "launches": p2["applies"]})
            del u32, v32
        except Exception as e:  # reported, not required
            roof["error"] = str(e)
        line["roofline"] = roof
        # accuracy of the batched result against the exact solutions (sphere)
        if args.workload == "sphere":
            a = band.extend(x)
            errs = []
            for k in (0, NRHS // 2, NRHS - 1):
                ex = torch.tensor(wl.exact(band, k), device="cuda")
                errs.append((a[:, k] - ex).abs().max().item())
            line["surface_error_linf_vs_exact"] = max(errs)
        # single right-hand side: FP64 solve (the comparison) and product bandwidth
        f0 = F[:, 0].contiguous()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x64, st64 = band.solve(0.0, 1.0, f0, tol=TOL, mode="fp64", maxit=args.maxit, raise_on_error=False)
        e1.record()
        torch.cuda.synchronize()
        line["fp64_single"] = {"s_per_rhs": e0.elapsed_time(e1) / 1000.0, "iterations": st64.iterations,
                               "relres": st64.relres, "status": st64.status}
        log(f"fp64 single: {line['fp64_single']}")
        diff = (x[:, 0] - x64).abs().max().item() / max(x64.abs().max().item(), 1e-300)
        line["fp32ir_vs_fp64_rel_linf"] = diff
        for dt, bytes_row, key in ((torch.float32, BYTES_ROW_FP32, "apply_fp32"),
                                   (torch.float64, BYTES_ROW_FP64, "apply_fp64")):
            u = torch.rand(band.N, dtype=dt, device="cuda")
            v = torch.empty_like(u)
            for _ in range(3):
                band.apply(0.0, 1.0, u, out=v)
            band.profile(True)
            for _ in range(20):
                band.apply(0.0, 1.0, u, out=v)
            p1 = band.profile(False)
            tms = p1["apply_ms"] / p1["applies"]
            gbs = bytes_row * band.NS / (tms * 1e-3) / 1e9
            line[key] = {"ms": tms, "GB/s_algorithmic": gbs, "hbm_peak_GB/s": hbm, "frac": gbs / hbm,
                         "peak_source": peak_src, "rows": band.NS}
        if not args.no_cpu_baseline and world == 1:
            try:
                s = cpu_baseline_sample(args.workload)
                value_cpu = s["s_per_dof_iter"] * band.N * st64.iterations
                line["cpu_baseline"] = {
                    "value": value_cpu, "unit": "s/RHS", "cores": s["cores"], "kind": "oracle",
                    "sample": f"oracle BiCGSTAB solve of 1 RHS on the same geometry at h=1/{round(1 / s['h'])} "
                              f"({s['N']} DOF, {s['iters']} iterations, {s['t_solve']:.1f} s); time per "
                              f"DOF-iteration x {band.N} DOF x {st64.iterations} iterations (the GPU FP64 count)"}
            except Exception as e:  # the baseline is reported, not required
                line["cpu_baseline"] = {"value": None, "unit": "s/RHS", "cores": None, "kind": "oracle",
                                        "sample": f"failed: {e}"}
        print(json.dumps(line), flush=True)
    band.close()
    if dist:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
