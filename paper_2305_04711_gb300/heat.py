"""The heat method for geodesic distance on the CPM (Sec. 7.2), driven through
the C ABI: (1) one implicit Euler heat step (I - dt M) v = 0 off C with v = 1 on
the curves C, (2) X = -grad v / |grad v|, (3) M phi = div X with phi = 0 on C;
`extra` repeats (2)-(3) from phi.  Every step runs in the CUDA library; this
module only sequences the calls."""
from __future__ import annotations

import torch


def geodesic_distance(band, dt: float, extra: int = 0, mode: str = "fp64", tol: float = 1e-10,
                      maxit: int = 20000):
    """Distance to the curves set on `band` (Dirichlet, first order).  Returns
    (phi [N], stats of the heat solve, stats of the last Poisson solve)."""
    ones = torch.ones(band.NC, dtype=torch.float64, device="cuda")
    zeros = torch.zeros(band.NC, dtype=torch.float64, device="cuda")
    v, st_heat = band.solve(1.0, -dt, band.rhs(g=ones), tol=tol, mode=mode, maxit=maxit)
    X = band.surface_gradient(v, normalize=True)
    st_poisson = None
    for _ in range(extra + 1):
        b = band.surface_divergence(X)
        phi, st_poisson = band.solve(0.0, 1.0, band.rhs(s=b, g=zeros), tol=tol, mode=mode, maxit=maxit)
        X = band.surface_gradient(-phi, normalize=True)
    return phi, st_heat, st_poisson
