"""Records the oracle's own BiCGSTAB iteration count on the torus diffusion-curve
workload (R = 1, r = 0.4, h = 1/256, 8 seeded meridians, right-hand side column
0 of the 64 U[0,1] sets), solved to the paper's stopping test |r|_2 <= 1e-10
|f|_2 (Sec. 5.4), into tests/golden/oracle_torus256_iterations.json.

The benchmark's reference arm times oracle BiCGSTAB iterations on the same band
on the host it runs on and multiplies by this count.  The script calls only the
oracle (and the seeded input generators); it runs for tens of minutes on a few
CPU cores.

    python oracle/record_iterations.py
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

OUT = os.path.join(os.path.dirname(HERE), "tests", "golden", "oracle_torus256_iterations.json")


def main():
    h = 1.0 / 256
    w, ang, g = ci.config3(h=h, ncurves=8, nrhs=64, seed=0, min_gap=0.2)
    t0 = time.perf_counter()
    o = O.Oracle(w.shape, h).set_curves(w.curves)
    t_setup = time.perf_counter() - t0
    f = o.rhs(np.zeros(o.NS), g[:, 0][o.bc_curve])
    t0 = time.perf_counter()
    x, it, rr = o.bicgstab(0.0, 1.0, f, tol=1e-10, maxit=40000)
    t_solve = time.perf_counter() - t0
    rec = {"workload": "torus R=1 r=0.4 h=1/256, 8 meridians (seed 0, min gap 0.2), column 0 of 64 U[0,1]",
           "N": int(o.N), "NS": int(o.NS), "NC": int(o.NC), "iterations": int(it), "relres": float(rr),
           "tol": 1e-10, "norm": "|f - A x|_2 / |f|_2", "threads": O.n_threads(),
           "setup_s": t_setup, "solve_s": t_solve, "command": "python oracle/record_iterations.py"}
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
