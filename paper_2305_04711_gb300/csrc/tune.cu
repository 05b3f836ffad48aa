// tune.cu -- the launch-shape autotuner.
//
// The batched product's cell gather keeps a cell's node values in registers
// for x passes of the stencil (more passes: fewer registers and more warps per
// SM, but more weight loads and partial sums through shared memory); its grid,
// the warp-per-row combine's grid and the Krylov vector kernels' blocks per SM
// trade occupancy against tail effects.  Which is fastest depends on the band
// (cells per brick, rows per cell), the batch width and the precision, so the
// tuner times each candidate on the context's own band with the caller's batch
// layout, by coordinate descent (passes, then the gather grid, then the
// combine grid, then the vector kernels), and keeps the fastest in the
// context.  Every candidate computes the same product; only the vector
// kernels' reduction grouping changes with their block count (each choice is
// deterministic).
#include <algorithm>
#include <vector>

#include "apply.cuh"
#include "cpm_internal.cuh"
#include "krylov.cuh"

namespace {

// the columns per lane of the cell gather for a batch (0: the batch does not
// use it): two above 32 columns, one from 16 to 32
int cells_rpl(int nrhs, int64_t ld) {
  return (nrhs > 32 && nrhs <= 64 && nrhs % 2 == 0 && ld % 2 == 0) ? 2 : (nrhs >= 16 && nrhs <= 32) ? 1 : 0;
}

template <typename T>
__global__ void fill_pattern_kernel(T *u, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(i * 2654435761u);
    u[i] = T(0.25) + T(0.5) * T(k >> 8) * T(1.0 / 16777216.0);
  }
}

template <typename T>
cpm_status time_products(cpm_ctx *c, const T *u, T *v, int nrhs, int64_t ld, cudaStream_t st, double *ms) {
  cudaEvent_t e0, e1;
  CPM_CUDA_TRY(cudaEventCreate(&e0));
  CPM_CUDA_TRY(cudaEventCreate(&e1));
  cpm_status rc = cpm_apply_rc_T<T>(c, 0.0, 1.0, 1.0, 1.0, u, v, nrhs, ld, st);
  const int reps = 3;
  cudaEventRecord(e0, st);
  for (int k = 0; k < reps && rc == CPM_OK; ++k) rc = cpm_apply_rc_T<T>(c, 0.0, 1.0, 1.0, 1.0, u, v, nrhs, ld, st);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (e != cudaSuccess) return cpm_internal_cuda_err(e);
  *ms = (double)t / reps;
  return CPM_OK;
}

template <typename T>
cpm_status tune_products(cpm_ctx *c, int nrhs, int64_t ld, T *u, T *v, cudaStream_t st, cpm_tune_info *info) {
  const int64_t N = c->NS + c->NC;
  fill_pattern_kernel<T><<<cpm_grid(N * ld, 256), 256, 0, st>>>(u, N * ld);
  CPM_CUDA_TRY(cudaGetLastError());
  Tune &t = c->tune;
  const int pi = (sizeof(T) == 8) ? 1 : 0;
  // the cell gather serves batches of 16 to 64 columns (2 per lane above 32)
  const int rpl = cells_rpl(nrhs, ld);
  double best = 0.0;
  cpm_status rc = time_products<T>(c, u, v, nrhs, ld, st, &best);
  if (rc) return rc;
  info->product_ms_default = best;
  if (rpl > 0) {
    const int np1 = c->p + 1;
    std::vector<int> xhs;
    for (int xh : {1, 2, 3, 4}) {
      if (np1 % xh) continue;
      if (sizeof(T) == 8 && np1 / xh > 2) continue;  // FP64 node values held at most two x wide
      xhs.push_back(xh);
    }
    // the defaults made explicit, so that the report names the kept choice
    if (t.cells_xh[pi][rpl - 1] <= 0) t.cells_xh[pi][rpl - 1] = cpm_cells_default_xh(np1, sizeof(T) == 8, rpl);
    if (t.cells_blocks_per_sm <= 0) t.cells_blocks_per_sm = 16;
    if (t.combine_warps_per_sm <= 0) t.combine_warps_per_sm = 64;
    int best_xh = t.cells_xh[pi][rpl - 1];
    for (int xh : xhs) {
      t.cells_xh[pi][rpl - 1] = xh;
      double ms = 0.0;
      rc = time_products<T>(c, u, v, nrhs, ld, st, &ms);
      if (rc) return rc;
      if (ms < best) { best = ms; best_xh = xh; }
    }
    t.cells_xh[pi][rpl - 1] = best_xh;
    int best_g = t.cells_blocks_per_sm;
    for (int g : {4, 8, 16, 32}) {
      t.cells_blocks_per_sm = g;
      double ms = 0.0;
      rc = time_products<T>(c, u, v, nrhs, ld, st, &ms);
      if (rc) return rc;
      if (ms < best) { best = ms; best_g = g; }
    }
    t.cells_blocks_per_sm = best_g;
    int best_w = t.combine_warps_per_sm;
    for (int wps : {16, 32, 64, 128}) {
      t.combine_warps_per_sm = wps;
      double ms = 0.0;
      rc = time_products<T>(c, u, v, nrhs, ld, st, &ms);
      if (rc) return rc;
      if (ms < best) { best = ms; best_w = wps; }
    }
    t.combine_warps_per_sm = best_w;
    info->cells_xh = t.cells_xh[pi][rpl - 1];
  }
  if (nrhs == 1 && c->ncells > 0) {
    // the single right-hand side product: a gather per cell or per row then the combine, or fused
    int best_m = t.single_mode;
    for (int mode : {0, 1, 2}) {
      t.single_mode = mode;
      double ms = 0.0;
      rc = time_products<T>(c, u, v, nrhs, ld, st, &ms);
      if (rc) return rc;
      if (ms < best) { best = ms; best_m = mode; }
    }
    t.single_mode = best_m;
    info->single_mode = best_m;
  }
  info->cells_blocks_per_sm = t.cells_blocks_per_sm;
  info->combine_warps_per_sm = t.combine_warps_per_sm;
  info->product_ms = best;
  return CPM_OK;
}

}  // namespace

cpm_status cpm_internal_set_tune(cpm_ctx *c, int nrhs, int prec, const cpm_tune_info *info) {
  const bool fp64 = (prec == CPM_PREC_FP64);
  const int np1 = c->p + 1;
  const int xh = info->cells_xh;
  if (xh < 0 || xh > 4 || (xh > 0 && (np1 % xh != 0 || (fp64 && np1 / xh > 2)))) return CPM_ERR_ARG;
  if (info->cells_blocks_per_sm < 0 || info->cells_blocks_per_sm > 256) return CPM_ERR_ARG;
  if (info->combine_warps_per_sm < 0 || info->combine_warps_per_sm > 256) return CPM_ERR_ARG;
  if (info->vec_blocks_per_sm < 0 || info->vec_blocks_per_sm > 4 || info->vec_blocks_per_sm == 3) return CPM_ERR_ARG;
  if (info->single_mode < 0 || info->single_mode > 2) return CPM_ERR_ARG;
  const int rpl = cells_rpl(nrhs, nrhs);
  if (rpl > 0) c->tune.cells_xh[fp64 ? 1 : 0][rpl - 1] = xh;
  c->tune.cells_blocks_per_sm = info->cells_blocks_per_sm;
  c->tune.combine_warps_per_sm = info->combine_warps_per_sm;
  c->tune.vec_blocks_per_sm = info->vec_blocks_per_sm;
  c->tune.single_mode = info->single_mode;
  return CPM_OK;
}

cpm_status cpm_internal_autotune(cpm_ctx *c, int nrhs, int64_t ld, int prec, cpm_tune_info *info, cudaStream_t st) {
  if (!c->solve || ld > c->res_ld) return CPM_ERR_CAPACITY;
  cpm_tune_info out{};
  cpm_status rc;
  // the workspace's Krylov vectors serve as input and output
  cpm_solve_buffers b;
  rc = cpm_solve_buffers_of(c, prec, &b);
  if (rc) return rc;
  if (prec == CPM_PREC_FP32) rc = tune_products<float>(c, nrhs, ld, (float *)b.u, (float *)b.v, st, &out);
  else rc = tune_products<double>(c, nrhs, ld, (double *)b.u, (double *)b.v, st, &out);
  if (rc) return rc;
  double best = 0.0;
  int best_b = c->tune.vec_blocks_per_sm > 0 ? c->tune.vec_blocks_per_sm : 2;
  rc = cpm_time_vector_kernels(c, prec, nrhs, ld, c->nsm * best_b, 5, st, &best);
  if (rc) return rc;
  for (int bps : {1, 2, 4}) {
    double ms = 0.0;
    rc = cpm_time_vector_kernels(c, prec, nrhs, ld, c->nsm * bps, 5, st, &ms);
    if (rc) return rc;
    if (ms < best) { best = ms; best_b = bps; }
  }
  c->tune.vec_blocks_per_sm = best_b;
  c->tune.tuned = true;
  out.vec_blocks_per_sm = best_b;
  out.vector_ms = best;
  if (info) *info = out;
  return CPM_OK;
}
