// api.cu -- the extern "C" entry points declared in include/cpm.h.
// Argument checking and status mapping live here; the work is in band.cu,
// boundary.cu, apply.cu, transpose.cu and krylov.cu.
#include <algorithm>
#include <cstring>
#include <new>

#include "apply.cuh"
#include "cpm_internal.cuh"
#include "krylov.cuh"

static cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

const char *cpm_status_str(cpm_status s) {
  switch (s) {
    case CPM_OK: return "CPM_OK";
    case CPM_ERR_ARG: return "CPM_ERR_ARG";
    case CPM_ERR_OOM: return "CPM_ERR_OOM";
    case CPM_ERR_CUDA: return "CPM_ERR_CUDA";
    case CPM_ERR_CAPACITY: return "CPM_ERR_CAPACITY";
    case CPM_ERR_CP_FAILED: return "CPM_ERR_CP_FAILED";
    case CPM_ERR_OVERLAP: return "CPM_ERR_OVERLAP";
    case CPM_ERR_BREAKDOWN: return "CPM_ERR_BREAKDOWN";
    case CPM_ERR_NOT_CONVERGED: return "CPM_ERR_NOT_CONVERGED";
    case CPM_ERR_TIMEOUT: return "CPM_ERR_TIMEOUT";
    case CPM_ERR_STATE: return "CPM_ERR_STATE";
  }
  return "CPM_ERR_UNKNOWN";
}

void cpm_destroy(cpm_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->istream) cudaStreamSynchronize(c->istream);
  cpm_free_solve(c);
  cpm_free_boundary(c);
  cpm_internal_free_band(c);
  cudaFree(c->d_shape_a);
  cudaFree(c->d_shape_c);
  cudaFree(c->a_scratch.p);
  cudaFree(c->b_scratch.p);
  for (auto e : c->ev_join)
    if (e) cudaEventDestroy(e);
  if (c->istream) cudaStreamDestroy(c->istream);
  cudaFree(c->d_err);
  cudaFree(c->d_counter);
  for (auto e : c->prof.ev) cudaEventDestroy(e);
  delete c;
}

cpm_status cpm_band_build(const cpm_shape_desc *shape, double h, int p, double r_band, void *stream,
                          cpm_ctx **out) {
  if (!out) return CPM_ERR_ARG;
  *out = nullptr;
  if (!shape || !(h > 0.0) || (p != 2 && p != 3)) return CPM_ERR_ARG;
  if (shape->kind < CPM_SHAPE_CIRCLE || shape->kind > CPM_SHAPE_BUMPY) return CPM_ERR_ARG;
  if ((shape->kind == CPM_SHAPE_CIRCLE) != (shape->dim == 2)) return CPM_ERR_ARG;
  if (shape->dim != 2 && shape->dim != 3) return CPM_ERR_ARG;
  if (shape->kind == CPM_SHAPE_BUMPY && (shape->K < 0 || (shape->K > 0 && (!shape->a || !shape->c)))) return CPM_ERR_ARG;
  if (shape->kind == CPM_SHAPE_TORUS && !(shape->rt > 0.0 && shape->R > shape->rt)) return CPM_ERR_ARG;
  cpm_ctx *c = new (std::nothrow) cpm_ctx;
  if (!c) return CPM_ERR_OOM;
  c->stream = as_stream(stream);
  c->nsm = cpm_device_sms();
  if (cudaMalloc(&c->d_err, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->d_counter, sizeof(unsigned long long) * 4) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->istream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join[1], cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    cpm_destroy(c);
    return CPM_ERR_OOM;
  }
  cpm_status rc = cpm_internal_band_build(c, shape, h, p, r_band);
  if (rc != CPM_OK) {
    cpm_destroy(c);
    return rc;
  }
  *out = c;
  return CPM_OK;
}

cpm_status cpm_band_info(const cpm_ctx *c, int64_t *n_s, int64_t *n_c, double *r_band, int64_t *n_bricks) {
  if (!c) return CPM_ERR_ARG;
  if (n_s) *n_s = c->NS;
  if (n_c) *n_c = c->NC;
  if (r_band) *r_band = c->rband;
  if (n_bricks) *n_bricks = c->nb;
  return CPM_OK;
}

cpm_status cpm_export_band(const cpm_ctx *c, int32_t *ijk, double *cp, void *stream) {
  if (!c) return CPM_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  if (ijk) CPM_CUDA_TRY(cudaMemcpyAsync(ijk, c->d_ijk, sizeof(int32_t) * 3 * c->NS, cudaMemcpyDeviceToDevice, st));
  if (cp) CPM_CUDA_TRY(cudaMemcpyAsync(cp, c->d_cp, sizeof(double) * 3 * c->NS, cudaMemcpyDeviceToDevice, st));
  return CPM_OK;
}

cpm_status cpm_set_boundary(cpm_ctx *c, const cpm_curve_desc *curves, int n) {
  if (!c || n < 0 || (n > 0 && !curves) || n > 127) return CPM_ERR_ARG;
  for (int k = 0; k < n; ++k) {
    const cpm_curve_desc &d = curves[k];
    if (d.kind != CPM_CURVE_POINT && d.kind != CPM_CURVE_CIRCLE) return CPM_ERR_ARG;
    if (d.bc < CPM_BC_DIR1 || d.bc > CPM_BC_NEU2) return CPM_ERR_ARG;
    if (d.bc_minus < 0 || d.bc_minus > CPM_BC_NEU2) return CPM_ERR_ARG;
    // a point in 3D has no sides, hence no conormal for a Neumann condition (Sec. 4.5)
    const bool neu = d.bc >= CPM_BC_NEU1 || d.bc_minus >= CPM_BC_NEU1;
    if (neu && d.kind == CPM_CURVE_POINT && c->dim == 3) return CPM_ERR_ARG;
    if (d.n_samples < 1) return CPM_ERR_ARG;
    if (d.kind == CPM_CURVE_POINT && d.n_samples != 1) return CPM_ERR_ARG;
    if (d.kind == CPM_CURVE_CIRCLE && !(d.rad > 0.0)) return CPM_ERR_ARG;
  }
  cpm_free_solve(c);
  c->res_ld = 0;
  c->res_flags = 0;
  cpm_status rc = cpm_internal_set_boundary(c, curves, n);
  if (rc) return rc;
  // single right-hand side workspaces of every product and solve form
  return cpm_reserve(c, 1, CPM_RESERVE_FP64 | CPM_RESERVE_FP32_IR);
}

cpm_status cpm_reserve(cpm_ctx *c, int64_t ld, int flags) {
  if (!c || ld < 1 || ld > 256 || (flags & ~(CPM_RESERVE_FP64 | CPM_RESERVE_FP32_IR))) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  // product intermediates: [N_S][ld] of the widest element (FP64), at least 3
  // FP64 columns for the heat steps' vector extensions
  const size_t scratch = sizeof(double) * (size_t)std::max<int64_t>(c->NS, 1) * (size_t)std::max<int64_t>(ld, 3);
  const size_t bscr = sizeof(double) * (size_t)std::max<int64_t>(c->NS, 1) * (size_t)ld;
  cpm_status rc = cpm_ensure(c->a_scratch, scratch);
  if (rc) return rc;
  rc = cpm_ensure(c->b_scratch, bscr);
  if (rc) return rc;
  if (flags) {
    rc = cpm_reserve_solve(c, ld, (flags & CPM_RESERVE_FP32_IR) != 0);
    if (rc) return rc;
  }
  c->res_ld = std::max(c->res_ld, ld);
  c->res_flags |= flags;
  return CPM_OK;
}

cpm_status cpm_export_boundary(const cpm_ctx *c, int64_t *twin, int32_t *curve, double *cpc, int32_t *side,
                               double *param, int32_t *type, void *stream) {
  if (!c || !c->boundary_set) return c ? CPM_ERR_STATE : CPM_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  if (c->NC == 0) return CPM_OK;
  if (twin) {
    // int32 on the device, int64 in the ABI: widen through a small kernel-free path
    int64_t *tmp = new (std::nothrow) int64_t[c->NC];
    int32_t *t32 = new (std::nothrow) int32_t[c->NC];
    if (!tmp || !t32) { delete[] tmp; delete[] t32; return CPM_ERR_OOM; }
    CPM_CUDA_TRY(cudaMemcpyAsync(t32, c->d_twin, sizeof(int32_t) * c->NC, cudaMemcpyDeviceToHost, st));
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t a = 0; a < c->NC; ++a) tmp[a] = t32[a];
    cudaError_t e = cudaMemcpyAsync(twin, tmp, sizeof(int64_t) * c->NC, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    delete[] tmp;
    delete[] t32;
    if (e) return cpm_internal_cuda_err(e);
  }
  if (curve) CPM_CUDA_TRY(cudaMemcpyAsync(curve, c->d_bc_curve, sizeof(int32_t) * c->NC, cudaMemcpyDeviceToDevice, st));
  if (cpc) CPM_CUDA_TRY(cudaMemcpyAsync(cpc, c->d_cpc, sizeof(double) * 3 * c->NC, cudaMemcpyDeviceToDevice, st));
  if (side) CPM_CUDA_TRY(cudaMemcpyAsync(side, c->d_side, sizeof(int32_t) * c->NC, cudaMemcpyDeviceToDevice, st));
  if (param) CPM_CUDA_TRY(cudaMemcpyAsync(param, c->d_param, sizeof(double) * c->NC, cudaMemcpyDeviceToDevice, st));
  if (type) CPM_CUDA_TRY(cudaMemcpyAsync(type, c->d_bc_type, sizeof(int32_t) * c->NC, cudaMemcpyDeviceToDevice, st));
  return CPM_OK;
}

static bool bad_batch(int nrhs, int64_t ld) { return nrhs < 1 || nrhs > 256 || ld < nrhs; }

cpm_status cpm_rhs(cpm_ctx *c, const double *s, const double *g, const double *samples, double *f, int nrhs,
                   int64_t ld, void *stream) {
  if (!c || !f || bad_batch(nrhs, ld)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  if (c->NC > 0 && !g && !samples) return CPM_ERR_ARG;
  return cpm_internal_rhs(c, s, g, samples, f, nrhs, ld, as_stream(stream));
}

cpm_status cpm_apply(cpm_ctx *c, double m, double n, int prec, const void *u, void *v, int nrhs, int64_t ld,
                     void *stream) {
  if (!c || !u || !v || bad_batch(nrhs, ld)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  if (prec == CPM_PREC_FP64)
    return cpm_apply_T<double>(c, m, n, (const double *)u, (double *)v, nrhs, ld, as_stream(stream));
  if (prec == CPM_PREC_FP32)
    return cpm_apply_T<float>(c, m, n, (const float *)u, (float *)v, nrhs, ld, as_stream(stream));
  return CPM_ERR_ARG;
}

cpm_status cpm_apply_noalloc(cpm_ctx *c, double m, double n, int prec, const void *u, void *v, int nrhs,
                             int64_t ld, void *stream) {
  if (!c || !u || !v || bad_batch(nrhs, ld)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  if (prec == CPM_PREC_FP64)
    return cpm_apply_noalloc_T<double>(c, m, n, (const double *)u, (double *)v, nrhs, ld, as_stream(stream));
  if (prec == CPM_PREC_FP32)
    return cpm_apply_noalloc_T<float>(c, m, n, (const float *)u, (float *)v, nrhs, ld, as_stream(stream));
  return CPM_ERR_ARG;
}

size_t cpm_apply_noalloc_max_bytes(void) { return cpm_noalloc_scratch_bytes(); }

cpm_status cpm_apply_transpose(cpm_ctx *c, double m, double n, int prec, const void *u, void *v, int nrhs, int64_t ld,
                               void *stream) {
  if (!c || !u || !v || bad_batch(nrhs, ld)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  if (prec == CPM_PREC_FP64)
    return cpm_apply_transpose_T<double>(c, m, n, (const double *)u, (double *)v, nrhs, ld, as_stream(stream));
  if (prec == CPM_PREC_FP32)
    return cpm_apply_transpose_T<float>(c, m, n, (const float *)u, (float *)v, nrhs, ld, as_stream(stream));
  return CPM_ERR_ARG;
}

cpm_status cpm_surface_gradient(cpm_ctx *c, const double *u, double *X, int normalize, void *stream) {
  if (!c || !u || !X) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  return cpm_internal_surface_gradient(c, u, X, normalize, as_stream(stream));
}

cpm_status cpm_surface_divergence(cpm_ctx *c, const double *X, double *b, void *stream) {
  if (!c || !X || !b) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  return cpm_internal_surface_divergence(c, X, b, as_stream(stream));
}

cpm_status cpm_extend(cpm_ctx *c, const double *u, double *a, int nrhs, int64_t ld, void *stream) {
  if (!c || !u || !a || bad_batch(nrhs, ld)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  return cpm_internal_extend(c, u, a, nrhs, ld, as_stream(stream));
}

static cpm_status check_solve(cpm_ctx *c, const double *f, double *x, int nrhs, int64_t ld,
                              const cpm_solve_opts *o) {
  if (!c || !f || !x || bad_batch(nrhs, ld)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  if (o && o->mode != CPM_SOLVE_FP64 && o->mode != CPM_SOLVE_FP32_IR) return CPM_ERR_ARG;
  return CPM_OK;
}

cpm_status cpm_solve(cpm_ctx *c, double m, double n, const double *f, double *x, int nrhs, int64_t ld,
                     const cpm_solve_opts *o, cpm_solve_stats *stats, void *stream) {
  cpm_status rc = check_solve(c, f, x, nrhs, ld, o);
  if (rc) return rc;
  return cpm_internal_solve(c, false, m, n, f, x, nrhs, ld, o, stats, as_stream(stream));
}

cpm_status cpm_solve_adjoint(cpm_ctx *c, double m, double n, const double *g, double *lam, int nrhs, int64_t ld,
                             const cpm_solve_opts *o, cpm_solve_stats *stats, void *stream) {
  cpm_status rc = check_solve(c, g, lam, nrhs, ld, o);
  if (rc) return rc;
  rc = cpm_build_transpose(c);
  if (rc) return rc;
  return cpm_internal_solve(c, true, m, n, g, lam, nrhs, ld, o, stats, as_stream(stream));
}

cpm_status cpm_boundary_grad(cpm_ctx *c, const double *lam, double *out, int nrhs, int64_t ld, void *stream) {
  if (!c || !lam || !out || bad_batch(nrhs, ld)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  return cpm_internal_boundary_grad(c, lam, out, nrhs, ld, as_stream(stream));
}

cpm_status cpm_profile(cpm_ctx *c, int enable, double *apply_ms, int64_t *apply_calls, int64_t *kernel_launches,
                       int64_t *row_rhs_processed) {
  if (!c) return CPM_ERR_ARG;
  Profiler &p = c->prof;
  if (enable) {
    p.on = true;
    p.used = 0;
    p.applies = 0;
    p.launches = 0;
    p.row_rhs = 0;
    return CPM_OK;
  }
  p.on = false;
  double total = 0.0;
  if (p.used) {
    CPM_CUDA_TRY(cudaEventSynchronize(p.ev[p.used - 1]));
    for (size_t k = 0; k + 1 < p.used; k += 2) {
      float ms = 0.0f;
      CPM_CUDA_TRY(cudaEventElapsedTime(&ms, p.ev[k], p.ev[k + 1]));
      total += ms;
    }
  }
  if (apply_ms) *apply_ms = total;
  if (apply_calls) *apply_calls = p.applies;
  if (kernel_launches) *kernel_launches = p.launches;
  if (row_rhs_processed) *row_rhs_processed = p.row_rhs;
  p.used = 0;
  return CPM_OK;
}

cpm_status cpm_autotune(cpm_ctx *c, int nrhs, int64_t ld, int prec, cpm_tune_info *info, void *stream) {
  if (!c || bad_batch(nrhs, ld) || (prec != CPM_PREC_FP32 && prec != CPM_PREC_FP64)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  return cpm_internal_autotune(c, nrhs, ld, prec, info, as_stream(stream));
}

cpm_status cpm_set_tune(cpm_ctx *c, int nrhs, int prec, const cpm_tune_info *t) {
  if (!c || !t || nrhs < 1 || (prec != CPM_PREC_FP32 && prec != CPM_PREC_FP64)) return CPM_ERR_ARG;
  if (!c->boundary_set) return CPM_ERR_STATE;
  return cpm_internal_set_tune(c, nrhs, prec, t);
}

cpm_status cpm_diagnostics(const cpm_ctx *c, int64_t *noflip, int64_t *nspec) {
  if (!c) return CPM_ERR_ARG;
  if (noflip) *noflip = c->noflip_twin;
  if (nspec) *nspec = c->nspec;
  return CPM_OK;
}

}  // extern "C"
