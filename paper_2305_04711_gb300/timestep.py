"""Crank-Nicolson time stepping of u_t = Delta_S u on a fixed band (the
heat-equation setting of Sec. 6.2): (I - dt/2 M) u^{k+1} = (I + dt/2 M) u^k, the
BC rows carrying the current boundary values.  Each step is one cpm_apply and
one cpm_solve warm-started from u^k; this module only sequences the calls."""
from __future__ import annotations


def heat_cn(band, u0, dt: float, nsteps: int, tol: float = 1e-12, mode: str = "fp64"):
    """nsteps CN steps from u0 ([N] or [N, nrhs], FP64 device tensor).  Returns
    (u, list of per-step solve stats)."""
    u = u0.clone()
    stats = []
    for _ in range(nsteps):
        rhs = band.apply(1.0, 0.5 * dt, u)
        rhs[band.NS:] = u[band.NS:]
        u, st = band.solve(1.0, -0.5 * dt, rhs, x0=u, tol=tol, mode=mode)
        stats.append(st)
    return u, stats
