// krylov.cu -- preconditioned BiCGSTAB on the device (Sec. 5.4), in FP64 or as
// FP32 inner solves of a mixed-precision iterative refinement.
//
// The solver is van der Vorst's BiCGSTAB with the diagonal of m I + n diag(L)
// on PDE rows and 1 on BC rows as preconditioner (Sec. 5.4).  Two forms:
//  * scaled (default): BiCGSTAB on the row-scaled system (W A) x = W f with W
//    that diagonal's inverse, so the recursive residual is the Jacobi-scaled
//    one, in which PDE rows (scale 1/h^2) and BC rows (scale 1) are comparable;
//  * plain: the paper's right-preconditioned form with the unscaled residual.
// All right-hand sides of a batch ([N][ld] layout) iterate together, each with
// its own scalars (rho, alpha, omega) in device memory, so iterations run
// without a host round trip; the host reads the per-column flags every
// `check_every` iterations.  Dot products are deterministic: fixed-size block
// partials reduced in a fixed order.  A right-hand side that reaches the
// tolerance is frozen.  A near-zero rho restarts that right-hand side's shadow
// residual (r_hat = r); too many restarts is a breakdown.
//
// The FP32 form is mixed-precision iterative refinement: the solution x and
// the residual f - A x are FP64; each outer step solves for a correction with
// FP32 BiCGSTAB (FP32 operator in its difference form and FP32 Krylov vectors,
// the correction itself accumulated in FP64) and adds it to x.  Storing a
// smooth field in FP32 limits the FP32 operator's relative accuracy to about
// eps_32 / h^2 times the field-to-Laplacian ratio, so each outer step targets
// a modest reduction (1e-2 by default) and starts a fresh Krylov space.
// Convergence is decided on the FP64 residual only; a column that the FP32
// steps stop improving finishes in FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "apply.cuh"
#include "cpm_internal.cuh"
#include "krylov.cuh"

namespace {

constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs: fixed, so reductions are deterministic
constexpr int RED_THREADS = 256;

// partial sums of up to 3 dot products per column: part[blk][q][r];
// products on PDE rows (i < NS) are weighted by wpde (1 for plain dot products)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) dots_kernel(const T *__restrict__ a0, const T *__restrict__ b0,
                                                           const T *__restrict__ a1, const T *__restrict__ b1,
                                                           const T *__restrict__ a2, const T *__restrict__ b2, int nq,
                                                           int64_t N, int64_t NS, double wpde, int nrhs, int64_t ld,
                                                           double *part) {
  __shared__ double sh[3][RED_THREADS];
  const int rows_per = RED_THREADS / nrhs;
  const int t = threadIdx.x;
  const int r = t % nrhs, sub = t / nrhs;
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  if (sub < rows_per) {
    int64_t chunk = (N + gridDim.x - 1) / gridDim.x;
    int64_t lo = blockIdx.x * chunk, hi = lo + chunk < N ? lo + chunk : N;
    // runs of 16 products are summed in T, the runs in FP64 (for FP32 vectors
    // this keeps the FP64 pipe, 1/64 of the FP32 rate here, off the hot loop)
    for (int64_t i = lo + sub; i < hi;) {
      T c0 = T(0), c1 = T(0), c2 = T(0);
      for (int k = 0; k < 16 && i < hi; ++k, i += rows_per) {
        const int64_t o = i * ld + r;
        const T wi = (i < NS) ? T(wpde) : T(1);
        c0 += wi * (a0[o] * b0[o]);
        if (nq > 1) c1 += wi * (a1[o] * b1[o]);
        if (nq > 2) c2 += wi * (a2[o] * b2[o]);
      }
      acc0 += (double)c0;
      acc1 += (double)c1;
      acc2 += (double)c2;
    }
  }
  sh[0][t] = acc0; sh[1][t] = acc1; sh[2][t] = acc2;
  __syncthreads();
  if (t < nrhs) {
    for (int q = 0; q < nq; ++q) {
      double s = 0.0;
      for (int k = 0; k < rows_per; ++k) s += sh[q][k * nrhs + t];
      part[((int64_t)blockIdx.x * 3 + q) * nrhs + t] = s;
    }
  }
}

__global__ void reduce_parts_kernel(const double *part, int nblocks, int nq, int nrhs, double *out) {
  int t = threadIdx.x;
  for (int qr = t; qr < nq * nrhs; qr += blockDim.x) {
    int q = qr / nrhs, r = qr % nrhs;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[((int64_t)b * 3 + q) * nrhs + r];
    out[q * nrhs + r] = s;
  }
}

// ---- per-RHS scalar state ---------------------------------------------------
// sc layout per rhs r: [0] rho_old [1] alpha [2] omega [3] rho [4] beta
//                      [5] active (1/0) [6] restart flag [7] restarts
//                      [8] |W f|^2 [9] |r|^2 (recursive) [10] breakdown
//                      [11] best |r|^2 [12] iterations since |r| last halved
//                      [13] stopped without reaching tol (stall or divergence)
//                      [14] |r|^2 at the start
constexpr int NSC = 15;

__global__ void scal_init_kernel(double *sc, const double *dots /* (r,r),(f,f) */, int nrhs, double tol) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  double *s = sc + r * NSC;
  s[0] = 1.0; s[1] = 1.0; s[2] = 1.0; s[3] = 0.0; s[4] = 0.0;
  s[6] = 0.0; s[7] = 0.0; s[10] = 0.0; s[12] = 0.0; s[13] = 0.0;
  double fn2 = dots[nrhs + r];
  s[8] = fn2 > 0.0 ? fn2 : 1.0;
  s[9] = dots[r];
  s[11] = s[9];
  s[14] = s[9];
  s[5] = (sqrt(s[9]) <= tol * sqrt(s[8]) || !isfinite(s[9])) ? 0.0 : 1.0;
}

// after dots (rhat, r), (rhat, rhat): rho, beta, restart decision
__global__ void scal_rho_kernel(double *sc, const double *dots, int nrhs) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  double *s = sc + r * NSC;
  if (s[5] == 0.0) return;
  double rho = dots[r], rhn2 = dots[nrhs + r];
  s[6] = 0.0;
  if (fabs(rho) <= 1e-28 * sqrt(rhn2) * sqrt(s[9]) || rho == 0.0) {
    // restart the shadow residual: rhat = r, rho = (r, r), p = r
    s[6] = 1.0;
    s[7] += 1.0;
    if (s[7] > 20.0) { s[10] = 1.0; s[5] = 0.0; return; }
    rho = s[9];
    s[0] = 1.0; s[1] = 1.0; s[2] = 1.0;
  }
  s[4] = (rho / s[0]) * (s[1] / s[2]);
  s[3] = rho;
}

__global__ void scal_alpha_kernel(double *sc, const double *dots, int nrhs) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  double *s = sc + r * NSC;
  if (s[5] == 0.0) return;
  double d = dots[r];
  if (d == 0.0 || !isfinite(d)) { s[10] = 1.0; s[5] = 0.0; return; }
  s[1] = s[3] / d;
}

__global__ void scal_omega_kernel(double *sc, const double *dots, int nrhs) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  double *s = sc + r * NSC;
  if (s[5] == 0.0) return;
  double ts = dots[r], tt = dots[nrhs + r];
  s[2] = (tt > 0.0) ? ts / tt : 0.0;
  if (s[2] == 0.0) { s[10] = 1.0; s[5] = 0.0; }
}

// after (r, r): convergence on the recursive residual (decide == 1) or only
// bookkeeping (decide == 0: the FP64 residual decides, FP32 form)
__global__ void scal_conv_kernel(double *sc, const double *dots, int nrhs, double tol, double stall, int decide) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  double *s = sc + r * NSC;
  if (s[5] == 0.0) return;
  s[9] = dots[r];
  s[0] = s[3];
  if (!isfinite(s[9]) || s[9] > 1e16 * s[11]) { s[13] = 1.0; s[5] = 0.0; return; }
  if (decide && sqrt(s[9]) <= tol * sqrt(s[8])) { s[5] = 0.0; return; }
  if (s[9] < 0.25 * s[11]) { s[11] = s[9]; s[12] = 0.0; }
  else { s[12] += 1.0; if (decide && s[12] > stall) { s[13] = 1.0; s[5] = 0.0; } }
}

// ---- fused vector updates ---------------------------------------------------
template <typename T>
__device__ __forceinline__ T dinv_of(int64_t i, int64_t NS, T dS) { return (i < NS) ? dS : T(1); }

// shadow-residual weight 1 + mix * u(i, c), u a fixed hash in [-1, 1]: with mix
// in [0, 1) it keeps (rhat, r) > 0 while breaking the structure that drives
// BiCGSTAB to near breakdown in FP32 (mix = 0: the classical rhat = r)
__device__ __forceinline__ float shadow_weight(int64_t i, int c, float mix) {
  if (mix == 0.0f) return 1.0f;
  uint64_t k = (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)c * 0xD1B54A32D192ED03ull;
  k ^= k >> 31; k *= 0xBF58476D1CE4E5B9ull; k ^= k >> 29;
  float u = (float)((k >> 40) & 0xFFFFFF) * (2.0f / 16777215.0f) - 1.0f;
  return 1.0f + mix * u;
}

// p = restart ? r : r + beta (p - omega v);  ph = D p;  (restart: rhat = r)
template <typename T>
__global__ void upd_p_kernel(const double *sc, int64_t N, int64_t NS, int nrhs, int64_t ld, T dS, float mix,
                             const T *r, T *rh, T *p, const T *v, T *ph) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    const double *s = sc + c * NSC;
    if (s[5] == 0.0) continue;
    int64_t o = i * ld + c;
    T pv;
    if (s[6] != 0.0) {
      rh[o] = r[o] * T(shadow_weight(i, c, mix));
      pv = r[o];
    } else {
      pv = r[o] + T(s[4]) * (p[o] - T(s[2]) * v[o]);
    }
    p[o] = pv;
    if (ph != p) ph[o] = dinv_of<T>(i, NS, dS) * pv;
  }
}

// s = r - alpha v;  sh = D s
template <typename T>
__global__ void upd_s_kernel(const double *sc, int64_t N, int64_t NS, int nrhs, int64_t ld, T dS, const T *r,
                             const T *v, T *s_, T *sh) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    const double *s = sc + c * NSC;
    if (s[5] == 0.0) continue;
    int64_t o = i * ld + c;
    T sv = r[o] - T(s[1]) * v[o];
    s_[o] = sv;
    if (sh != s_) sh[o] = dinv_of<T>(i, NS, dS) * sv;
  }
}

// x += alpha ph + omega sh;  r = s - omega t
// (x may be kept in a wider type TX than the Krylov vectors: the increment is
// formed in T and accumulated in TX)
template <typename T, typename TX>
__global__ void upd_xr_kernel(const double *sc, int64_t N, int nrhs, int64_t ld, TX *x, T *r, const T *ph,
                              const T *sh, const T *s_, const T *t) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    const double *s = sc + c * NSC;
    if (s[5] == 0.0) continue;
    int64_t o = i * ld + c;
    T al = T(s[1]), om = T(s[2]);
    x[o] = x[o] + TX(al * ph[o] + om * sh[o]);
    r[o] = s_[o] - om * t[o];
  }
}

// r = f - r (r holds A x);  rhat = r;  p = v = 0
template <typename T>
__global__ void init_r_kernel(int64_t N, int nrhs, int64_t ld, const T *f, T *r, T *rh, T *p, T *v) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    T rv = f[o] - r[o];
    r[o] = rv;
    rh[o] = rv;
    p[o] = T(0);
    v[o] = T(0);
  }
}

// ---- FP64 pieces ------------------------------------------------------------
// r = f - r (r holds A x)
__global__ void residual64_kernel(int64_t N, int nrhs, int64_t ld, const double *f, double *r) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    r[o] = f[o] - r[o];
  }
}

// out = W f (PDE rows scaled by dS)
__global__ void scale_rows64_kernel(int64_t N, int64_t NS, int nrhs, int64_t ld, double dS, const double *f,
                                    double *out) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    out[o] = (i < NS) ? dS * f[o] : f[o];
  }
}

// columns with acc != 0 take the candidate
__global__ void accept_kernel(int64_t N, int nrhs, int64_t ld, const double *acc, const double *xc, double *x) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    if (acc[c] != 0.0) x[o] = xc[o];
  }
}

// restarted refinement: FP32 right-hand side W r / |W r| per active column
// (scale 0: inactive column, zero right-hand side)
__global__ void ir_rhs_kernel(int64_t N, int64_t NS, double wrow, int nrhs, int64_t ld, const double *scale,
                              const double *r64, float *f32) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    double sc = scale[c];
    f32[o] = (sc > 0.0) ? (float)(((i < NS) ? wrow : 1.0) * r64[o] / sc) : 0.0f;
  }
}

// candidate xc = x + scale * d (FP64 accumulation of the FP32 correction)
__global__ void ir_candidate_kernel(int64_t N, int nrhs, int64_t ld, const double *scale, const double *d,
                                    const double *x, double *xc) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    double sc = scale[c];
    xc[o] = (sc > 0.0) ? x[o] + sc * d[o] : x[o];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
struct SolveWork {
  cpm_ctx *owner = nullptr;  // for launch counting
  int nrhs = 0;
  int64_t ld = 0;
  int elem = 0;  // bytes per element of the Krylov vectors
  void *vec[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double *r64 = nullptr;    // FP64 true residual
  double *fs = nullptr;     // W f (scaled FP64 form)
  float *f32 = nullptr;     // FP32 right-hand side of the inner solves
  double *xd = nullptr;     // FP64 solution of the inner solves
  double *part = nullptr, *dots = nullptr, *sc = nullptr;
  double *h_pinned = nullptr;  // host mirror of sc
  double *d_cols = nullptr;    // per-column host-set arrays: [4][nrhs]
};

static void free_work(SolveWork *w) {
  if (!w) return;
  for (auto &p : w->vec) cudaFree(p);
  cudaFree(w->r64); cudaFree(w->fs); cudaFree(w->f32); cudaFree(w->xd);
  cudaFree(w->part); cudaFree(w->dots); cudaFree(w->sc); cudaFree(w->d_cols);
  if (w->h_pinned) cudaFreeHost(w->h_pinned);
  delete w;
}

void cpm_free_solve(cpm_ctx *c) {
  free_work(c->solve);
  free_work(c->solve_adj);
  free_work(c->solve64);
  free_work(c->solve_adj64);
  c->solve = nullptr;
  c->solve_adj = nullptr;
  c->solve64 = nullptr;
  c->solve_adj64 = nullptr;
}

static cpm_status get_work(cpm_ctx *c, SolveWork *&w, int64_t N, int nrhs, int64_t ld, int elem) {
  if (w && w->nrhs == nrhs && w->ld == ld && w->elem == elem) return CPM_OK;
  free_work(w);
  w = new SolveWork;
  w->owner = c;
  w->nrhs = nrhs; w->ld = ld; w->elem = elem;
  size_t vb = (size_t)N * (size_t)ld * (size_t)elem;
  for (auto &p : w->vec) CPM_CUDA_TRY(cudaMalloc(&p, vb));
  CPM_CUDA_TRY(cudaMalloc(&w->r64, (size_t)N * ld * sizeof(double)));
  CPM_CUDA_TRY(cudaMalloc(&w->fs, (size_t)N * ld * sizeof(double)));
  if (elem == (int)sizeof(float)) {
    CPM_CUDA_TRY(cudaMalloc(&w->f32, (size_t)N * ld * sizeof(float)));
    CPM_CUDA_TRY(cudaMalloc(&w->xd, (size_t)N * ld * sizeof(double)));
  }
  CPM_CUDA_TRY(cudaMalloc(&w->part, sizeof(double) * RED_BLOCKS * 3 * nrhs));
  CPM_CUDA_TRY(cudaMalloc(&w->dots, sizeof(double) * 3 * nrhs));
  CPM_CUDA_TRY(cudaMalloc(&w->sc, sizeof(double) * NSC * nrhs));
  CPM_CUDA_TRY(cudaMalloc(&w->d_cols, sizeof(double) * 4 * nrhs));
  CPM_CUDA_TRY(cudaMallocHost(&w->h_pinned, sizeof(double) * (NSC + 3) * nrhs));
  return CPM_OK;
}

template <typename T>
static void dots(SolveWork *w, int nq, const T *a0, const T *b0, const T *a1, const T *b1, const T *a2, const T *b2,
                 int64_t N, cudaStream_t st, int64_t NS = 0, double wpde = 1.0) {
  dots_kernel<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a0, b0, a1, b1, a2, b2, nq, N, NS, wpde, w->nrhs, w->ld,
                                                     w->part);
  reduce_parts_kernel<<<1, 256, 0, st>>>(w->part, RED_BLOCKS, nq, w->nrhs, w->dots);
  if (w->owner) cpm_count_launches(w->owner, 2);
}

// operator with a PDE-row scale: v = R A u (or R A^T u)
template <typename T>
using ApplyFn = cpm_status (*)(cpm_ctx *, double, double, double, const T *, T *, int, int64_t, cudaStream_t);

// Krylov variant: right diagonal preconditioning (the paper's form, Sec. 5.4)
// or left row scaling (scaled residual)
struct KrylovForm {
  double right;     // PDE-row value of the right preconditioner (1: none)
  double rowscale;  // PDE-row scale applied to the operator and rhs (1: none)
  double stall;     // iterations without halving the residual before giving up
  float shadow_mix;  // perturbation of the shadow residual (0: rhat = r)
};

// one BiCGSTAB iteration for all active columns (device only)
template <typename T, typename TX = T>
static cpm_status iteration(cpm_ctx *c, ApplyFn<T> apply, const KrylovForm &form, double m, double n, TX *x,
                            SolveWork *w, double tol, int decide, cudaStream_t st) {
  const int64_t N = c->NS + c->NC, NS = c->NS;
  const int nrhs = w->nrhs;
  const int64_t ld = w->ld;
  T *r = (T *)w->vec[0], *rh = (T *)w->vec[1], *p = (T *)w->vec[2], *v = (T *)w->vec[3], *s = (T *)w->vec[4],
    *t = (T *)w->vec[5], *ph = (T *)w->vec[6], *sh = (T *)w->vec[7];
  const T dS = T(form.right);
  // without a right preconditioner D p = p and D s = s: no copies
  if (form.right == 1.0) {
    ph = p;
    sh = s;
  }
  const unsigned g = cpm_grid(N * nrhs, 256);
  dots<T>(w, 2, rh, r, rh, rh, nullptr, nullptr, N, st);
  scal_rho_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs);
  upd_p_kernel<T><<<g, 256, 0, st>>>(w->sc, N, NS, nrhs, ld, dS, form.shadow_mix, r, rh, p, v, ph);
  cpm_status rc = apply(c, m, n, form.rowscale, ph, v, nrhs, ld, st);
  if (rc) return rc;
  dots<T>(w, 1, rh, v, nullptr, nullptr, nullptr, nullptr, N, st);
  scal_alpha_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs);
  upd_s_kernel<T><<<g, 256, 0, st>>>(w->sc, N, NS, nrhs, ld, dS, r, v, s, sh);
  rc = apply(c, m, n, form.rowscale, sh, t, nrhs, ld, st);
  if (rc) return rc;
  dots<T>(w, 2, t, s, t, t, nullptr, nullptr, N, st);
  scal_omega_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs);
  upd_xr_kernel<T, TX><<<g, 256, 0, st>>>(w->sc, N, nrhs, ld, x, r, ph, sh, s, t);
  dots<T>(w, 1, r, r, nullptr, nullptr, nullptr, nullptr, N, st);
  scal_conv_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs, tol, form.stall, decide);
  cpm_count_launches(c, 7);  // 4 scalar + 3 vector kernels (products and dots count themselves)
  return CPM_OK;
}

static cpm_status read_scalars(SolveWork *w, cudaStream_t st) {
  CPM_CUDA_TRY(cudaMemcpyAsync(w->h_pinned, w->sc, sizeof(double) * NSC * w->nrhs, cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  return CPM_OK;
}

// BiCGSTAB on A x = f in one precision T; x holds the initial guess.
// (x of a wider type TX than T requires x = 0 on entry: the initial product
// is skipped)
template <typename T, typename TX = T>
static cpm_status bicgstab(cpm_ctx *c, ApplyFn<T> apply, const KrylovForm &form, double m, double n, const T *f,
                           TX *x, SolveWork *w, double tol, int maxit, int check_every, int *iters, int *restarts,
                           bool *broke, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  const int nrhs = w->nrhs;
  const int64_t ld = w->ld;
  T *r = (T *)w->vec[0], *rh = (T *)w->vec[1], *p = (T *)w->vec[2], *v = (T *)w->vec[3];
  const unsigned g = cpm_grid(N * nrhs, 256);
  cpm_status rc = CPM_OK;
  if constexpr (std::is_same<T, TX>::value) {
    rc = apply(c, m, n, form.rowscale, x, r, nrhs, ld, st);
    if (rc) return rc;
  } else {
    CPM_CUDA_TRY(cudaMemsetAsync(r, 0, sizeof(T) * (size_t)N * ld, st));
  }
  init_r_kernel<T><<<g, 256, 0, st>>>(N, nrhs, ld, f, r, rh, p, v);
  cpm_count_launches(c, 1);
  dots<T>(w, 2, r, r, f, f, nullptr, nullptr, N, st);
  scal_init_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs, tol);
  cpm_count_launches(c, 1);
  int it = 0;
  *broke = false;
  while (true) {
    rc = read_scalars(w, st);
    if (rc) return rc;
    bool any = false;
    int nrestart = 0;
    for (int q = 0; q < nrhs; ++q) {
      const double *sq = w->h_pinned + q * NSC;
      if (sq[5] != 0.0) any = true;
      if (sq[10] != 0.0) *broke = true;
      nrestart += (int)sq[7];
    }
    *restarts = nrestart;
    if (!any || it >= maxit) break;
    int steps = std::min(check_every, maxit - it);
    for (int k = 0; k < steps; ++k) {
      rc = iteration<T, TX>(c, apply, form, m, n, x, w, tol, 1, st);
      if (rc) return rc;
    }
    CPM_CUDA_TRY(cudaGetLastError());
    it += steps;
  }
  *iters = it;
  return CPM_OK;
}

// FP64 residual r64 = f - A x and its squared weighted norms per column:
// |W r|^2 and |W f|^2 with W = diag(wrow on PDE rows, 1 on BC rows)
static cpm_status residual64(cpm_ctx *c, ApplyFn<double> apply, double m, double n, const double *f, const double *x,
                             SolveWork *w, double wrow, std::vector<double> &rn2, std::vector<double> &fn2,
                             cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  cpm_status rc = apply(c, m, n, 1.0, x, w->r64, w->nrhs, w->ld, st);
  if (rc) return rc;
  residual64_kernel<<<cpm_grid(N * w->nrhs, 256), 256, 0, st>>>(N, w->nrhs, w->ld, f, w->r64);
  cpm_count_launches(c, 1);
  dots<double>(w, 2, w->r64, w->r64, f, f, nullptr, nullptr, N, st, c->NS, wrow * wrow);
  CPM_CUDA_TRY(cudaMemcpyAsync(w->h_pinned, w->dots, sizeof(double) * 2 * w->nrhs, cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  rn2.assign(w->h_pinned, w->h_pinned + w->nrhs);
  fn2.assign(w->h_pinned + w->nrhs, w->h_pinned + 2 * w->nrhs);
  return CPM_OK;
}

static double relres_of(double rn2, double fn2) {
  double fnq = fn2 > 0 ? std::sqrt(fn2) : 1.0;
  double rr = std::sqrt(rn2) / fnq;
  return std::isfinite(rr) ? rr : INFINITY;
}

static double worst_relres(const std::vector<double> &rn2, const std::vector<double> &fn2) {
  double worst = 0.0;
  for (size_t q = 0; q < rn2.size(); ++q) worst = std::max(worst, relres_of(rn2[q], fn2[q]));
  return worst;
}

// Mixed-precision iterative refinement with restarted inner solves: each
// outer step takes the FP64 residual r = f - A x, solves (W A) d = W r / |W r|
// by FP32 BiCGSTAB from d = 0 to the relative inner tolerance, and adds
// |W r| d to x in FP64.  Every inner solve starts a fresh Krylov space, so a
// loss of accuracy in one FP32 solve does not carry into the next.  A column
// whose FP64 residual fails to halve over two outer steps is left for the
// FP64 finish.  rhs_w weights the PDE rows of the inner right-hand side: the
// scaling of the left-scaled form, or 1 for a right-preconditioned inner form.
static cpm_status ir_restarted(cpm_ctx *c, ApplyFn<double> ap64, ApplyFn<float> ap32, const KrylovForm &form32,
                               double m, double n, const double *f, double *x, SolveWork *w, double wrow,
                               double rhs_w, double tol, double inner_tol, int inner_maxit, int maxit, int max_outer,
                               int check_every, bool trace, int *iters, int *outers, int *restarts,
                               std::vector<double> &rn2, std::vector<double> &fn2, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  const int nrhs = w->nrhs;
  const int64_t ld = w->ld;
  const unsigned g = cpm_grid(N * nrhs, 256);
  double *d_scale = w->d_cols;
  std::vector<double> scale(nrhs, 0.0), best(nrhs, INFINITY);
  std::vector<int> stall(nrhs, 0);
  std::vector<char> act(nrhs, 1);
  cpm_status rc = residual64(c, ap64, m, n, f, x, w, wrow, rn2, fn2, st);
  if (rc) return rc;
  int it_total = 0, nout = 0, nrs = 0;
  while (nout < max_outer && it_total < maxit) {
    bool any = false;
    for (int q = 0; q < nrhs; ++q) {
      if (!act[q]) { scale[q] = 0.0; continue; }
      if (relres_of(rn2[q], fn2[q]) <= tol) { act[q] = 0; scale[q] = 0.0; continue; }
      if (rn2[q] < 0.25 * best[q]) { best[q] = rn2[q]; stall[q] = 0; }
      else if (++stall[q] >= 2) { act[q] = 0; scale[q] = 0.0; continue; }
      scale[q] = std::sqrt(rn2[q]);
      any = true;
    }
    if (trace)
      std::fprintf(stderr, "[cpm ir] outer %d it %d relres[0] %.3e worst %.3e\n", nout, it_total,
                   relres_of(rn2[0], fn2[0]), worst_relres(rn2, fn2));
    if (!any) break;
    CPM_CUDA_TRY(cudaMemcpyAsync(d_scale, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    ir_rhs_kernel<<<g, 256, 0, st>>>(N, c->NS, rhs_w, nrhs, ld, d_scale, w->r64, w->f32);
    CPM_CUDA_TRY(cudaMemsetAsync(w->xd, 0, sizeof(double) * (size_t)N * ld, st));
    cpm_count_launches(c, 1);
    int it = 0, rs = 0;
    bool broke = false;
    rc = bicgstab<float, double>(c, ap32, form32, m, n, w->f32, w->xd, w, inner_tol,
                                 std::min(inner_maxit, maxit - it_total), check_every, &it, &rs, &broke, st);
    if (rc) return rc;
    it_total += it;
    nrs += rs;
    // keep the correction only where the FP64 residual went down; a column
    // whose FP32 solve made it worse is left for the FP64 finish
    ir_candidate_kernel<<<g, 256, 0, st>>>(N, nrhs, ld, d_scale, w->xd, x, w->fs);
    cpm_count_launches(c, 1);
    ++nout;
    std::vector<double> rn2_prev = rn2;
    rc = residual64(c, ap64, m, n, f, w->fs, w, wrow, rn2, fn2, st);
    if (rc) return rc;
    std::vector<double> acc(nrhs, 0.0);
    bool rejected = false;
    for (int q = 0; q < nrhs; ++q) {
      if (scale[q] == 0.0) { rn2[q] = rn2_prev[q]; continue; }
      if (std::isfinite(rn2[q]) && rn2[q] < rn2_prev[q]) {
        acc[q] = 1.0;
      } else {
        rejected = true;
        act[q] = 0;
        rn2[q] = rn2_prev[q];
      }
    }
    CPM_CUDA_TRY(cudaMemcpyAsync(d_scale, acc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    accept_kernel<<<g, 256, 0, st>>>(N, nrhs, ld, d_scale, w->fs, x);
    cpm_count_launches(c, 1);
    if (rejected) {
      // r64 must hold the residual of x for the next outer step
      rc = residual64(c, ap64, m, n, f, x, w, wrow, rn2, fn2, st);
      if (rc) return rc;
    }
  }
  *iters = it_total;
  *outers = nout;
  *restarts = nrs;
  return CPM_OK;
}

static cpm_status solve_impl(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                             int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t st) {
  cpm_solve_opts opts{1e-10, 10000, CPM_SOLVE_FP64, 1e-2, 200, 16, CPM_NORM_SCALED, 1000};
  if (o) opts = *o;
  if (opts.tol <= 0) opts.tol = 1e-10;
  if (opts.maxit <= 0) opts.maxit = 10000;
  if (opts.inner_tol <= 0 || opts.inner_tol >= 1) opts.inner_tol = 1e-2;
  if (opts.max_refine <= 0) opts.max_refine = 200;
  if (opts.check_every <= 0) opts.check_every = 16;
  if (opts.inner_maxit <= 0) opts.inner_maxit = 1000;
  if (opts.norm != CPM_NORM_PLAIN) opts.norm = CPM_NORM_SCALED;
  const bool scaled = (opts.norm == CPM_NORM_SCALED);
  const bool trace = std::getenv("CPM_SOLVE_TRACE") != nullptr;
  const int64_t N = c->NS + c->NC;
  // Jacobi value of the PDE rows: 1/(m + n diag L) (Sec. 5.4)
  const double dS = 1.0 / (m + n * (-2.0 * c->dim / (c->h * c->h)));
  // residual weight of the PDE rows; the adjoint (iterated right-preconditioned,
  // see below) is measured on its unscaled residual, the iteration's own
  const double wrow = (scaled && !adjoint) ? dS : 1.0;
  SolveWork *&w = adjoint ? c->solve_adj : c->solve;
  cpm_status rc;
  int iters = 0, restarts = 0, refinements = 0, iters64 = 0;
  bool broke = false;
  std::vector<double> rn2, fn2;
  ApplyFn<double> ap64 = adjoint ? cpm_apply_transpose_scaled_T<double> : cpm_apply_scaled_T<double>;
  // scaled: BiCGSTAB on (W A) x = W f, so its recursive residual is the
  // measured one; plain: the paper's right-preconditioned form.  The adjoint
  // always iterates right-preconditioned, A^T W mu = g with lambda = W mu: this
  // is the transpose of the row-scaled forward system, whereas scaling the rows
  // of A^T leaves the BC rows with O(1/h^2) couplings and BiCGSTAB breaks down.
  const bool left = scaled && !adjoint;
  KrylovForm form = left ? KrylovForm{1.0, dS, 4000.0, 0.0f} : KrylovForm{dS, 1.0, 4000.0, 0.0f};
  if (opts.mode == CPM_SOLVE_FP64) {
    rc = get_work(c, w, N, nrhs, ld, sizeof(double));
    if (rc) return rc;
    const double *rhs = f;
    if (left) {
      scale_rows64_kernel<<<cpm_grid(N * nrhs, 256), 256, 0, st>>>(N, c->NS, nrhs, ld, dS, f, w->fs);
      cpm_count_launches(c, 1);
      rhs = w->fs;
    }
    // the recursively updated residual drifts from f - A x near the rounding
    // level; while the true residual is above tol, restart from the current x
    double prev_worst = INFINITY;
    for (int pass = 0; pass < 6; ++pass) {
      int it = 0, rs = 0;
      rc = bicgstab<double>(c, ap64, form, m, n, rhs, x, w, opts.tol, opts.maxit - iters, opts.check_every, &it, &rs,
                            &broke, st);
      if (rc) return rc;
      iters += it;
      iters64 += it;
      restarts += rs;
      rc = residual64(c, ap64, m, n, f, x, w, wrow, rn2, fn2, st);
      if (rc) return rc;
      double worst = worst_relres(rn2, fn2);
      // stop at the attainable accuracy: a restart that does not halve the worst
      // true residual gains nothing more
      if (worst <= opts.tol || broke || iters >= opts.maxit || !(worst < 0.5 * prev_worst)) break;
      prev_worst = worst;
    }
  } else if (opts.mode == CPM_SOLVE_FP32_IR) {
    ApplyFn<float> ap32 = adjoint ? cpm_apply_transpose_scaled_T<float> : cpm_apply_scaled_T<float>;
    // the FP32 iteration always runs on the row-scaled system (its residual is
    // balanced); the requested norm decides acceptance and convergence
    KrylovForm form32 = adjoint ? KrylovForm{dS, 1.0, 4000.0, 0.5f} : KrylovForm{1.0, dS, 4000.0, 0.5f};
    rc = get_work(c, w, N, nrhs, ld, sizeof(float));
    if (rc) return rc;
    rc = ir_restarted(c, ap64, ap32, form32, m, n, f, x, w, wrow, adjoint ? 1.0 : dS, opts.tol, opts.inner_tol, opts.inner_maxit,
                      opts.maxit, opts.max_refine, opts.check_every, trace, &iters, &refinements, &restarts, rn2, fn2,
                      st);
    if (rc) return rc;
    if (!(worst_relres(rn2, fn2) <= opts.tol) && iters < opts.maxit) {
      // FP64 finish from the current iterate for the columns the FP32 phase
      // left above tol (columns already converged stay frozen)
      if (trace) std::fprintf(stderr, "[cpm] FP64 finish from relres %.3e\n", worst_relres(rn2, fn2));
      SolveWork *&w64 = adjoint ? c->solve_adj64 : c->solve64;
      rc = get_work(c, w64, N, nrhs, ld, sizeof(double));
      if (rc) return rc;
      const double *rhs = f;
      if (left) {
        scale_rows64_kernel<<<cpm_grid(N * nrhs, 256), 256, 0, st>>>(N, c->NS, nrhs, ld, dS, f, w64->fs);
        cpm_count_launches(c, 1);
        rhs = w64->fs;
      }
      int it = 0, rs = 0;
      broke = false;
      rc = bicgstab<double>(c, ap64, form, m, n, rhs, x, w64, opts.tol, opts.maxit - iters, opts.check_every, &it,
                            &rs, &broke, st);
      if (rc) return rc;
      iters += it;
      iters64 += it;
      restarts += rs;
      rc = residual64(c, ap64, m, n, f, x, w64, wrow, rn2, fn2, st);
      if (rc) return rc;
    }
  } else {
    return CPM_ERR_ARG;
  }
  double relres = worst_relres(rn2, fn2);
  cpm_status out = CPM_OK;
  if (!(relres <= opts.tol)) out = broke ? CPM_ERR_BREAKDOWN : CPM_ERR_NOT_CONVERGED;
  if (stats) {
    stats->iterations = iters;
    stats->refinements = refinements;
    stats->restarts = restarts;
    stats->relres = relres;
    stats->status = out;
    stats->fp64_iterations = iters64;
  }
  return out;
}

cpm_status cpm_internal_solve(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                              int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t st) {
  return solve_impl(c, adjoint, m, n, f, x, nrhs, ld, o, stats, st);
}
