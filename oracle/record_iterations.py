"""Records the oracle's own BiCGSTAB iteration count on a benchmark workload,
solved to the paper's stopping test |r|_2 <= 1e-10 |f|_2 (Sec. 5.4):

  torus   R = 1, r = 0.4, h = 1/256, 8 seeded meridians, right-hand side column
          0 of the 64 U[0,1] sets -> tests/golden/oracle_torus256_iterations.json
  sphere  unit sphere, h = 1/128, Dirichlet latitude circles theta = pi/4,
          3 pi/4, column 0 of the spherical-harmonic batch (l = 1, m = -1:
          -Delta u = 2 Y, Y on the circles)
          -> tests/golden/oracle_sphere128_iterations.json

The benchmark's CPU baseline times oracle BiCGSTAB iterations on the same band
on the host it runs on and multiplies by this count.  The script calls only the
oracle (and the seeded input generators); the torus takes tens of minutes on a
few CPU cores, the sphere a few.

    python oracle/record_iterations.py [torus|sphere]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
# run as a script, this folder is first on the path and its oracle.py would
# shadow the oracle package
sys.path = [q for q in sys.path if os.path.abspath(q or ".") != HERE]
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import cpm_inputs as ci  # noqa: E402
from oracle import oracle as O  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(HERE), "tests", "golden")


def main():
    kind = sys.argv[1] if len(sys.argv) > 1 else "torus"
    if kind == "torus":
        h = 1.0 / 256
        w, ang, g = ci.config3(h=h, ncurves=8, nrhs=64, seed=0, min_gap=0.2)
        desc = "torus R=1 r=0.4 h=1/256, 8 meridians (seed 0, min gap 0.2), column 0 of 64 U[0,1]"
        out = os.path.join(GOLDEN, "oracle_torus256_iterations.json")
    else:
        h = 1.0 / 128
        w = ci.config2(h, ci.BC_DIR1)
        desc = ("unit sphere h=1/128, Dirichlet circles theta=pi/4, 3pi/4, column 0 of the Y_l^m batch "
                "(l=1, m=-1: s = -2 Y at cp_S, g = Y at cp_C)")
        out = os.path.join(GOLDEN, "oracle_sphere128_iterations.json")
    t0 = time.perf_counter()
    o = O.Oracle(w.shape, h).set_curves(w.curves)
    t_setup = time.perf_counter() - t0
    if kind == "torus":
        f = o.rhs(np.zeros(o.NS), g[:, 0][o.bc_curve])
    else:
        f = o.rhs(-2.0 * ci.real_ylm(1, -1, o.cp), ci.real_ylm(1, -1, o.cpc))
    t0 = time.perf_counter()
    x, it, rr = o.bicgstab(0.0, 1.0, f, tol=1e-10, maxit=40000)
    t_solve = time.perf_counter() - t0
    rec = {"workload": desc,
           "N": int(o.N), "NS": int(o.NS), "NC": int(o.NC), "iterations": int(it), "relres": float(rr),
           "tol": 1e-10, "norm": "|f - A x|_2 / |f|_2", "threads": O.n_threads(),
           "setup_s": t_setup, "solve_s": t_solve, "command": f"python oracle/record_iterations.py {kind}"}
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
