"""Crank-Nicolson time stepping of u_t = Delta_S u on a fixed band (the
heat-equation setting of Sec. 6.2): (I - dt/2 M) u^{k+1} = (I + dt/2 M) u^k on the
PDE rows, the BC rows carrying the BC equations with the boundary data of the
new time level (cpm_rhs forms c_alpha g_alpha: c = 1 or 2 for first- or
second-order Dirichlet rows, 0 for zero-Neumann rows).  Each step is one
cpm_apply, one cpm_rhs and one cpm_solve warm-started from u^k; this module only
sequences the calls."""
from __future__ import annotations


def heat_cn(band, u0, dt: float, nsteps: int, g=None, tol: float = 1e-12, mode: str = "fp64"):
    """nsteps CN steps from u0 ([N] FP64 device tensor).  g: Dirichlet data per
    BC DOF ([N_C] device tensor held fixed, or a function of t returning one;
    None: zero data).  Returns (u, list of per-step solve stats)."""
    import torch
    u = u0.clone()
    stats = []
    zero = torch.zeros(max(band.NC, 1), dtype=torch.float64, device=u0.device)[:band.NC]
    for k in range(nsteps):
        rhs = band.apply(1.0, 0.5 * dt, u)
        gk = g((k + 1) * dt) if callable(g) else (zero if g is None else g)
        if band.NC:
            rhs[band.NS:] = band.rhs(g=gk.contiguous())[band.NS:]
        u, st = band.solve(1.0, -0.5 * dt, rhs, x0=u, tol=tol, mode=mode)
        stats.append(st)
    return u, stats
