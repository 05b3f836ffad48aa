// apply.cuh -- launch interface of the operator kernels (see apply.cu).
#pragma once

#include <algorithm>
#include <vector>

#include "cpm_internal.cuh"

template <typename T>
struct ApplyArgs {
  BandView v;
  const uint32_t *rbase;
  const uint32_t *rself;
  const T *t;
  const int32_t *spec_of;
  const int32_t *ecol;
  const T *ew;
  const int32_t *fcol;
  const int32_t *nbr8;  // [NS][8] FD neighbour columns (NULL: computed per row)
  const int32_t *bc_cnt;
  const int32_t *bc_col;
  const T *bc_val;
};

template <typename T>
ApplyArgs<T> cpm_apply_args(const cpm_ctx *c);
template <typename T>
void cpm_launch_gather(const ApplyArgs<T> &A, T cs, const T *u, T *a, int nrhs, int64_t ld, cudaStream_t st,
                       bool diff);
template <typename T>
void cpm_launch_combine(const ApplyArgs<T> &A, T m, T n, T rowscale, T cs, const T *u, const T *a, T *v, int nrhs,
                        int64_t ld, cudaStream_t st, bool diff);
// v = R A C u: R scales the PDE rows of the result, C the PDE entries of the
// input (diagonal row scaling and right preconditioning without extra vectors)
template <typename T>
cpm_status cpm_apply_rc_T(cpm_ctx *c, double m, double n, double rowscale, double colscale, const T *u, T *v,
                          int nrhs, int64_t ld, cudaStream_t st);
template <typename T>
cpm_status cpm_apply_transpose_rc_T(cpm_ctx *c, double m, double n, double rowscale, double colscale, const T *u,
                                    T *v, int nrhs, int64_t ld, cudaStream_t st);
// the product with the intermediate in a fixed module array (no allocation)
template <typename T>
cpm_status cpm_apply_noalloc_T(cpm_ctx *c, double m, double n, const T *u, T *v, int nrhs, int64_t ld,
                               cudaStream_t st);
size_t cpm_noalloc_scratch_bytes();
template <typename T>
cpm_status cpm_apply_T(cpm_ctx *c, double m, double n, const T *u, T *v, int nrhs, int64_t ld, cudaStream_t st);
template <typename T>
cpm_status cpm_apply_transpose_T(cpm_ctx *c, double m, double n, const T *u, T *v, int nrhs, int64_t ld,
                                 cudaStream_t st);

// cell-bucketed E u for all PDE rows plus the flipped-entry correction of the
// rows near curves (batched layouts); returns the number of kernels launched
template <typename T>
int cpm_launch_gather_cells(const cpm_ctx *c, const ApplyArgs<T> &A, T cs, const T *u, T *a, int nrhs, int64_t ld,
                            cudaStream_t st, bool diff, int rpl);

cpm_status cpm_internal_surface_gradient(cpm_ctx *c, const double *u, double *X, int normalize, cudaStream_t st);
cpm_status cpm_internal_surface_divergence(cpm_ctx *c, const double *X, double *b, cudaStream_t st);
// single right-hand side: E u for all PDE rows in cell order plus the
// flipped-entry correction; returns the number of kernels launched
template <typename T>
int cpm_launch_gather1(const cpm_ctx *c, const ApplyArgs<T> &A, T cs, const T *u, T *a, cudaStream_t st, bool diff);

// the cell gather's default x passes for a stencil of np1 nodes per axis, the
// precision and the columns per lane (1 or 2); the autotuner starts from it
int cpm_cells_default_xh(int np1, bool fp64, int rpl);

// the single right-hand side product in one persistent kernel (fused1.cu);
// returns the launches (0: not built for this band)
template <typename T>
int cpm_launch_fused1(const cpm_ctx *c, const ApplyArgs<T> &A, T m, T n, T rowscale, T cs, const T *u, T *a, T *v,
                      cudaStream_t st);
cpm_status cpm_build_fused1(cpm_ctx *c);
void cpm_free_fused1(cpm_ctx *c);

cpm_status cpm_internal_extend(cpm_ctx *c, const double *u, double *a, int nrhs, int64_t ld, cudaStream_t st);
cpm_status cpm_internal_rhs(cpm_ctx *c, const double *s, const double *g, const double *samples, double *f, int nrhs,
                            int64_t ld, cudaStream_t st);
cpm_status cpm_internal_boundary_grad(cpm_ctx *c, const double *lam, double *out, int nrhs, int64_t ld,
                                      cudaStream_t st);
cpm_status cpm_internal_band_build(cpm_ctx *c, const cpm_shape_desc *s, double h, int p, double r_band);
void cpm_internal_free_band(cpm_ctx *c);
cpm_status cpm_internal_set_boundary(cpm_ctx *c, const cpm_curve_desc *curves, int n);
cpm_status cpm_internal_autotune(cpm_ctx *c, int nrhs, int64_t ld, int prec, cpm_tune_info *info, cudaStream_t st);
cpm_status cpm_internal_set_tune(cpm_ctx *c, int nrhs, int prec, const cpm_tune_info *info);

