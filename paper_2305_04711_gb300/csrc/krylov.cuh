// krylov.cuh -- solver entry points (see krylov.cu).
#pragma once

#include "cpm_internal.cuh"

cpm_status cpm_internal_solve(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                              int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t st);
void cpm_free_solve(cpm_ctx *c);
// reserve the solve workspace for leading dimension ld (FP32 refinement
// buffers too with fp32); the solve path's only allocation
cpm_status cpm_reserve_solve(cpm_ctx *c, int64_t ld, bool fp32);
// milliseconds per launch of the vector reductions with G blocks (autotuner)
cpm_status cpm_time_vector_kernels(cpm_ctx *c, int prec, int nrhs, int64_t ld, int G, int reps, cudaStream_t st,
                                   double *ms);
// two reserved [N][ld] vectors of precision prec (the autotuner's scratch)
struct cpm_solve_buffers { void *u, *v; };
cpm_status cpm_solve_buffers_of(cpm_ctx *c, int prec, cpm_solve_buffers *b);

