// heat.cu -- the vector-field steps of the heat method for geodesic distance
// (Sec. 7.2): the surface gradient of a field and the surface divergence of a
// vector field, each by central differences of its closest-point extension over
// the FD neighbours that the Laplacian rows use (flipped across interior
// boundaries as in Eq. 11).
//
//   gradient  : a = E u on PDE DOFs (u itself on BC DOFs, whose E rows are the
//               identity); g_d(x_i) = (a(n_i^{+d}) - a(n_i^{-d})) / 2h, or
//               X = -g / |g| when normalised (0 where g = 0).  A BC DOF takes
//               the value of its twin node.
//   divergence: b_i = sum_d (X~_d(n_i^{+d}) - X~_d(n_i^{-d})) / 2h with
//               X~ = E X on PDE DOFs and X on BC DOFs.
// A missing neighbour (band-edge rows, which no interpolation stencil reads)
// takes the row's own extended value.
#include <cmath>

#include "apply.cuh"
#include "cpm_internal.cuh"

namespace {

__device__ __forceinline__ double ext_val(int32_t c, int64_t i, int64_t NS, const double *a, const double *u,
                                          int comp, int ncomp) {
  if (c < 0) return a[i * ncomp + comp];
  if (c < NS) return a[(int64_t)c * ncomp + comp];
  return u[(int64_t)c * ncomp + comp];
}

__global__ void grad_kernel(int64_t NS, int64_t NC, int dim, double inv2h, const int32_t *nbr8, const int32_t *twin,
                            const double *a, const double *u, int normalize, double *X) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < NS + NC;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (j < NS) ? j : (int64_t)twin[j - NS];
    double g[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < dim; ++d) {
      const int32_t cp = nbr8[i * 8 + 2 * d + 1], cm = nbr8[i * 8 + 2 * d];
      g[d] = (ext_val(cp, i, NS, a, u, 0, 1) - ext_val(cm, i, NS, a, u, 0, 1)) * inv2h;
    }
    if (normalize) {
      const double nrm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      for (int d = 0; d < 3; ++d) g[d] = (nrm > 0.0) ? -g[d] / nrm : 0.0;
    }
    for (int d = 0; d < 3; ++d) X[j * 3 + d] = g[d];
  }
}

__global__ void div_kernel(int64_t NS, int dim, double inv2h, const int32_t *nbr8, const double *xe,
                           const double *X, double *b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NS; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int d = 0; d < dim; ++d) {
      const int32_t cp = nbr8[i * 8 + 2 * d + 1], cm = nbr8[i * 8 + 2 * d];
      acc += (ext_val(cp, i, NS, xe, X, d, 3) - ext_val(cm, i, NS, xe, X, d, 3)) * inv2h;
    }
    b[i] = acc;
  }
}

}  // namespace

cpm_status cpm_internal_surface_gradient(cpm_ctx *c, const double *u, double *X, int normalize, cudaStream_t st) {
  // the extension goes to the context's product scratch (reserved at set-up
  // for at least 3 FP64 columns)
  if (sizeof(double) * (size_t)c->NS > c->a_scratch.bytes) return CPM_ERR_CAPACITY;
  double *a = reinterpret_cast<double *>(c->a_scratch.p);
  cpm_status rc = cpm_internal_extend(c, u, a, 1, 1, st);
  if (rc) return rc;
  grad_kernel<<<cpm_grid(c->NS + c->NC, 256), 256, 0, st>>>(c->NS, c->NC, c->dim, 0.5 / c->h, c->d_nbr8, c->d_twin, a,
                                                            u, normalize, X);
  cpm_count_launches(c, 2);
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}

cpm_status cpm_internal_surface_divergence(cpm_ctx *c, const double *X, double *b, cudaStream_t st) {
  if (sizeof(double) * 3 * (size_t)c->NS > c->a_scratch.bytes) return CPM_ERR_CAPACITY;
  double *xe = reinterpret_cast<double *>(c->a_scratch.p);
  cpm_status rc = cpm_internal_extend(c, X, xe, 3, 3, st);
  if (rc) return rc;
  div_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(c->NS, c->dim, 0.5 / c->h, c->d_nbr8, xe, X, b);
  cpm_count_launches(c, 2);
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}
