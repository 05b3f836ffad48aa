// krylov.cuh -- solver entry points (see krylov.cu).
#pragma once

#include "cpm_internal.cuh"

cpm_status cpm_internal_solve(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                              int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t st);
void cpm_free_solve(cpm_ctx *c);
