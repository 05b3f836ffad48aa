"""torch.autograd.Function over cpm_solve: u = A^{-1} f(s, samples) with
f = [s ; c_alpha g_alpha(samples)] (the right-hand side of Sec. 5.2).  The
backward pass solves the adjoint system A^T lambda = dL/du (cpm_solve_adjoint)
and maps lambda to the inputs: dL/ds = lambda on the PDE rows and
dL/dsamples = B^T (c lambda_C) (cpm_boundary_grad).  All arithmetic runs in the
CUDA library."""
from __future__ import annotations

import torch


class CPMSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, band, m, n, s, samples, tol=1e-12, mode="fp64"):
        s_in = s.detach().contiguous() if s is not None else None
        f = band.rhs(s=s_in, samples=samples.detach().contiguous())
        u, _ = band.solve(m, n, f, tol=tol, mode=mode)
        ctx.band, ctx.m, ctx.n, ctx.tol, ctx.mode = band, m, n, tol, mode
        ctx.has_s = s is not None
        return u

    @staticmethod
    def backward(ctx, grad_u):
        band = ctx.band
        lam, _ = band.solve(ctx.m, ctx.n, grad_u.contiguous(), tol=ctx.tol, mode=ctx.mode, adjoint=True)
        grad_s = lam[:band.NS].clone() if ctx.has_s else None
        grad_samples = band.boundary_grad(lam)
        return None, None, None, grad_s, grad_samples, None, None


def cpm_solve(band, m: float, n: float, s, samples, tol: float = 1e-12, mode: str = "fp64"):
    """Differentiable solve of A u = [s ; c g(samples)] on `band` (boundary set)."""
    return CPMSolve.apply(band, m, n, s, samples, tol, mode)
