// transpose.cu -- v = A^T u (placeholder until the transposed gather lands).
#include "apply.cuh"
#include "cpm_internal.cuh"

cpm_status cpm_build_transpose(cpm_ctx *c) {
  (void)c;
  return CPM_ERR_STATE;
}

template <typename T>
cpm_status cpm_apply_transpose_T(cpm_ctx *c, double m, double n, const T *u, T *v, int nrhs, int64_t ld,
                                 cudaStream_t st) {
  (void)c; (void)m; (void)n; (void)u; (void)v; (void)nrhs; (void)ld; (void)st;
  return CPM_ERR_STATE;
}
template cpm_status cpm_apply_transpose_T<double>(cpm_ctx *, double, double, const double *, double *, int, int64_t,
                                                  cudaStream_t);
template cpm_status cpm_apply_transpose_T<float>(cpm_ctx *, double, double, const float *, float *, int, int64_t,
                                                 cudaStream_t);

template <typename T>
cpm_status cpm_apply_transpose_scaled_T(cpm_ctx *c, double m, double n, double rowscale, const T *u, T *v, int nrhs,
                                        int64_t ld, cudaStream_t st) {
  (void)rowscale;
  return cpm_apply_transpose_T<T>(c, m, n, u, v, nrhs, ld, st);
}
template cpm_status cpm_apply_transpose_scaled_T<double>(cpm_ctx *, double, double, double, const double *, double *,
                                                         int, int64_t, cudaStream_t);
template cpm_status cpm_apply_transpose_scaled_T<float>(cpm_ctx *, double, double, double, const float *, float *, int,
                                                        int64_t, cudaStream_t);
