// krylov.cu -- preconditioned BiCGSTAB on the device (Sec. 5.4), in FP64 or in
// FP32 with FP64 reliable updates.
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
// The FP32 form (iterative refinement in its "reliable update" shape): the
// Krylov vectors and the operator are FP32, the solution x and the true
// residual f - A x are FP64.  The FP32 iterate is a correction that is folded
// into x whenever the FP32 recursive residual has dropped by a factor delta
// since the last fold (or after a fixed number of iterations); then the FP64
// residual is recomputed and replaces the FP32 recursive one.  Unlike
// restarting an inner solve at every refinement, the Krylov recurrences
// continue across folds, so the slowly converging smooth modes keep their
// progress.  Convergence is decided on the FP64 residual only.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
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
    for (int64_t i = lo + sub; i < hi; i += rows_per) {
      int64_t o = i * ld + r;
      double wi = (i < NS) ? wpde : 1.0;
      acc0 += wi * ((double)a0[o] * (double)b0[o]);
      if (nq > 1) acc1 += wi * ((double)a1[o] * (double)b1[o]);
      if (nq > 2) acc2 += wi * ((double)a2[o] * (double)b2[o]);
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
//                      [14] |r|^2 at the last reliable update (FP32 form)
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

// FP32 form: after a reliable update, per column: new |r|^2, activity, and a
// restart of the recurrences for columns that broke down
__global__ void scal_reliable_kernel(double *sc, const double *rn2, const double *act, const double *replaced,
                                     const double *reset, int nrhs) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  double *s = sc + r * NSC;
  s[5] = act[r];
  if (replaced[r] != 0.0 && rn2[r] >= 0.0) {
    s[9] = rn2[r];
    s[14] = rn2[r];
    if (rn2[r] < s[11]) { s[11] = rn2[r]; s[12] = 0.0; }
  }
  if (reset[r] != 0.0) {
    s[0] = 1.0; s[1] = 1.0; s[2] = 1.0; s[6] = 0.0; s[10] = 0.0; s[13] = 0.0;
    s[7] += 1.0;
  }
}

// FP32 form with a measuring norm other than the iteration's: set |r|^2 of the
// replaced columns from a fresh dot product
__global__ void scal_setr_kernel(double *sc, const double *dots, const double *replaced, int nrhs) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  if (replaced[r] == 0.0) return;
  double *s = sc + r * NSC;
  s[9] = dots[r];
  s[14] = dots[r];
  s[11] = dots[r];
  s[12] = 0.0;
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
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
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
    ph[o] = dinv_of<T>(i, NS, dS) * pv;
  }
}

// s = r - alpha v;  sh = D s
template <typename T>
__global__ void upd_s_kernel(const double *sc, int64_t N, int64_t NS, int nrhs, int64_t ld, T dS, const T *r,
                             const T *v, T *s_, T *sh) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    const double *s = sc + c * NSC;
    if (s[5] == 0.0) continue;
    int64_t o = i * ld + c;
    T sv = r[o] - T(s[1]) * v[o];
    s_[o] = sv;
    sh[o] = dinv_of<T>(i, NS, dS) * sv;
  }
}

// x += alpha ph + omega sh;  r = s - omega t
template <typename T>
__global__ void upd_xr_kernel(const double *sc, int64_t N, int nrhs, int64_t ld, T *x, T *r, const T *ph, const T *sh,
                              const T *s_, const T *t) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    const double *s = sc + c * NSC;
    if (s[5] == 0.0) continue;
    int64_t o = i * ld + c;
    T al = T(s[1]), om = T(s[2]);
    x[o] = x[o] + al * ph[o] + om * sh[o];
    r[o] = s_[o] - om * t[o];
  }
}

// r = f - r (r holds A x);  rhat = r;  p = v = 0
template <typename T>
__global__ void init_r_kernel(int64_t N, int nrhs, int64_t ld, const T *f, T *r, T *rh, T *p, T *v) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
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
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    int64_t o = i * ld + c;
    r[o] = f[o] - r[o];
  }
}

// out = W f (PDE rows scaled by dS)
__global__ void scale_rows64_kernel(int64_t N, int64_t NS, int nrhs, int64_t ld, double dS, const double *f,
                                    double *out) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    int64_t o = i * ld + c;
    out[o] = (i < NS) ? dS * f[o] : f[o];
  }
}

// candidate of a reliable update: xc = x + x32 (every column)
__global__ void candidate_kernel(int64_t N, int nrhs, int64_t ld, const double *x, const float *x32, double *xc) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    int64_t o = i * ld + c;
    xc[o] = x[o] + (double)x32[o];
  }
}

// columns with acc != 0 take the candidate; columns with drop != 0 restart x32
__global__ void accept_kernel(int64_t N, int nrhs, int64_t ld, const double *acc, const double *drop,
                              const double *xc, double *x, float *x32) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    int64_t o = i * ld + c;
    if (acc[c] != 0.0) x[o] = xc[o];
    if (drop[c] != 0.0) x32[o] = 0.0f;
  }
}

// r32 = W r64 for the active columns; columns that restart also take
// rhat = r32 and p = v = 0
__global__ void replace_r_kernel(int64_t N, int64_t NS, double wrow, float mix, int nrhs, int64_t ld,
                                 const double *act, const double *reset, const double *r64, float *r32, float *rh,
                                 float *p, float *v) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    if (act[c] == 0.0) continue;
    int64_t o = i * ld + c;
    float rv = (float)(((i < NS) ? wrow : 1.0) * r64[o]);
    r32[o] = rv;
    if (reset[c] != 0.0) {
      rh[o] = rv * shadow_weight(i, c, mix);
      p[o] = 0.0f;
      v[o] = 0.0f;
    }
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
  float *x32 = nullptr;     // FP32 correction since the last reliable update
  double *part = nullptr, *dots = nullptr, *sc = nullptr;
  double *h_pinned = nullptr;  // host mirror of sc
  double *d_cols = nullptr;    // per-column host-set arrays: [4][nrhs]
};

static void free_work(SolveWork *w) {
  if (!w) return;
  for (auto &p : w->vec) cudaFree(p);
  cudaFree(w->r64); cudaFree(w->fs); cudaFree(w->x32);
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
  if (elem == (int)sizeof(float)) CPM_CUDA_TRY(cudaMalloc(&w->x32, (size_t)N * ld * sizeof(float)));
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
template <typename T>
static cpm_status iteration(cpm_ctx *c, ApplyFn<T> apply, const KrylovForm &form, double m, double n, T *x,
                            SolveWork *w, double tol, int decide, cudaStream_t st) {
  const int64_t N = c->NS + c->NC, NS = c->NS;
  const int nrhs = w->nrhs;
  const int64_t ld = w->ld;
  T *r = (T *)w->vec[0], *rh = (T *)w->vec[1], *p = (T *)w->vec[2], *v = (T *)w->vec[3], *s = (T *)w->vec[4],
    *t = (T *)w->vec[5], *ph = (T *)w->vec[6], *sh = (T *)w->vec[7];
  const T dS = T(form.right);
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
  upd_xr_kernel<T><<<g, 256, 0, st>>>(w->sc, N, nrhs, ld, x, r, ph, sh, s, t);
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
template <typename T>
static cpm_status bicgstab(cpm_ctx *c, ApplyFn<T> apply, const KrylovForm &form, double m, double n, const T *f, T *x,
                           SolveWork *w, double tol, int maxit, int check_every, int *iters, int *restarts,
                           bool *broke, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  const int nrhs = w->nrhs;
  const int64_t ld = w->ld;
  T *r = (T *)w->vec[0], *rh = (T *)w->vec[1], *p = (T *)w->vec[2], *v = (T *)w->vec[3];
  const unsigned g = cpm_grid(N * nrhs, 256);
  cpm_status rc = apply(c, m, n, form.rowscale, x, r, nrhs, ld, st);
  if (rc) return rc;
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
      rc = iteration<T>(c, apply, form, m, n, x, w, tol, 1, st);
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

// FP32 BiCGSTAB with FP64 reliable updates (see the file comment)
static cpm_status bicgstab_reliable(cpm_ctx *c, ApplyFn<double> ap64, ApplyFn<float> ap32, const KrylovForm &form,
                                    double m, double n, const double *f, double *x, SolveWork *w, double wrow,
                                    double wfp32,
                                    double tol, double delta, int max_between, int maxit, int max_updates,
                                    int check_every, bool trace, int *iters, int *updates, int *restarts, bool *broke,
                                    std::vector<double> &rn2, std::vector<double> &fn2, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  const int nrhs = w->nrhs;
  const int64_t ld = w->ld;
  float *r = (float *)w->vec[0], *rh = (float *)w->vec[1], *p = (float *)w->vec[2], *v = (float *)w->vec[3];
  float *x32 = w->x32;
  const unsigned g = cpm_grid(N * nrhs, 256);
  double *d_rn2 = w->d_cols, *d_act = w->d_cols + nrhs, *d_reset = w->d_cols + 2 * nrhs;
  std::vector<double> act(nrhs, 1.0), reset(nrhs, 1.0), best(nrhs, INFINITY);
  std::vector<int> since_best(nrhs, 0);
  cpm_status rc = residual64(c, ap64, m, n, f, x, w, wrow, rn2, fn2, st);
  if (rc) return rc;
  CPM_CUDA_TRY(cudaMemsetAsync(x32, 0, sizeof(float) * (size_t)N * ld, st));
  // scalars: |W f|^2 from the FP64 pass, |r|^2 from the replaced residual
  CPM_CUDA_TRY(cudaMemcpyAsync(w->dots, rn2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
  CPM_CUDA_TRY(cudaMemcpyAsync(w->dots + nrhs, fn2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
  scal_init_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs, 0.0);
  cpm_count_launches(c, 1);
  int it = 0, last_update = 0, nupd = 0, nrestart = 0;
  *broke = false;
  bool do_update = true;  // the first "update" installs r32 = W r64, rhat = r32
  std::vector<double> acc(nrhs, 0.0), replace(nrhs, 1.0), drop(nrhs, 0.0);
  std::vector<int> nreject(nrhs, 0);
  while (true) {
    if (do_update) {
      if (nupd > 0) {
        // fold x32 into x only where the FP64 residual of x + x32 decreased;
        // elsewhere the correction is dropped and the recurrences restart
        candidate_kernel<<<g, 256, 0, st>>>(N, nrhs, ld, x, x32, w->fs);
        cpm_count_launches(c, 1);
        std::vector<double> rn2_prev = rn2;
        rc = residual64(c, ap64, m, n, f, w->fs, w, wrow, rn2, fn2, st);
        if (rc) return rc;
        bool rejected = false;
        for (int q = 0; q < nrhs; ++q) {
          bool ok = act[q] != 0.0 && std::isfinite(rn2[q]) && rn2[q] < rn2_prev[q];
          acc[q] = ok ? 1.0 : 0.0;
          if (ok) {
            nreject[q] = 0;
            replace[q] = 1.0;
          } else if (act[q] != 0.0) {
            // not folded: BiCGSTAB spikes are often temporary, so the FP32
            // iteration goes on unchanged; after three rejections in a row the
            // correction is dropped and the recurrences restart from x
            rejected = true;
            replace[q] = 0.0;
            if (++nreject[q] >= 3) {
              nreject[q] = 0;
              reset[q] = 1.0;
              replace[q] = 1.0;
              ++nrestart;
            }
            if (trace && q == 0)
              std::fprintf(stderr, "[cpm reliable] column 0: fold rejected (fp32 |r|/|r0| %.3e)%s\n",
                           std::sqrt(w->h_pinned[9] / w->h_pinned[14]), reset[q] != 0.0 ? ", restart" : "");
          }
        }
        // x takes the candidate where accepted; x32 restarts where accepted or
        // reset (a reset column also needs its residual replaced)
        for (int q = 0; q < nrhs; ++q) {
          drop[q] = (acc[q] != 0.0 || reset[q] != 0.0) ? 1.0 : 0.0;
          if (reset[q] != 0.0) replace[q] = 1.0;
        }
        CPM_CUDA_TRY(cudaMemcpyAsync(d_act, acc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
        CPM_CUDA_TRY(cudaMemcpyAsync(d_reset, drop.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
        accept_kernel<<<g, 256, 0, st>>>(N, nrhs, ld, d_act, d_reset, w->fs, x, x32);
        cpm_count_launches(c, 1);
        if (rejected) {
          rc = residual64(c, ap64, m, n, f, x, w, wrow, rn2, fn2, st);
          if (rc) return rc;
        }
      }
      bool any = false;
      for (int q = 0; q < nrhs; ++q) {
        if (act[q] == 0.0) continue;
        double rr = relres_of(rn2[q], fn2[q]);
        if (rr <= tol) { act[q] = 0.0; continue; }
        // a column whose FP64 residual has not halved in 4 folds has reached
        // what the FP32 phase can do; the FP64 phase takes it from here
        if (rn2[q] < 0.25 * best[q]) { best[q] = rn2[q]; since_best[q] = 0; }
        else if (++since_best[q] > 4) { act[q] = 0.0; continue; }
        any = true;
      }
      if (trace)
        std::fprintf(stderr, "[cpm reliable] update %d it %d relres[0] %.3e fp32 |r|/|r0| %.3e\n", nupd, it,
                     relres_of(rn2[0], fn2[0]), nupd ? std::sqrt(w->h_pinned[9] / w->h_pinned[14]) : 1.0);
      ++nupd;
      last_update = it;
      if (!any || nupd > max_updates) break;
      // the residual is replaced for columns whose x changed (accepted or
      // restarted); a rejected column keeps its FP32 recursive residual
      for (int q = 0; q < nrhs; ++q) drop[q] = (act[q] != 0.0 && replace[q] != 0.0) ? 1.0 : 0.0;
      CPM_CUDA_TRY(cudaMemcpyAsync(d_rn2, rn2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      CPM_CUDA_TRY(cudaMemcpyAsync(d_act, drop.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      CPM_CUDA_TRY(cudaMemcpyAsync(d_reset, reset.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      replace_r_kernel<<<g, 256, 0, st>>>(N, c->NS, wfp32, form.shadow_mix, nrhs, ld, d_act, d_reset, w->r64, r, rh, p,
                                          v);
      cpm_count_launches(c, 1);
      // the FP32 recursive residual restarts from the replaced one (which is
      // already W r, so its plain norm is the weighted norm)
      std::vector<double> rs2(nrhs);
      for (int q = 0; q < nrhs; ++q) rs2[q] = (wfp32 == wrow) ? rn2[q] : -1.0;
      CPM_CUDA_TRY(cudaMemcpyAsync(d_rn2, rs2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      for (int q = 0; q < nrhs; ++q) acc[q] = act[q];
      CPM_CUDA_TRY(cudaMemcpyAsync(w->d_cols + 3 * nrhs, acc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice,
                                   st));
      scal_reliable_kernel<<<1, 256, 0, st>>>(w->sc, d_rn2, w->d_cols + 3 * nrhs, d_act, d_reset, nrhs);
      cpm_count_launches(c, 1);
      if (wfp32 != wrow) {
        // the FP32 residual norm differs from the measured one: take it from r32
        dots<float>(w, 1, r, r, nullptr, nullptr, nullptr, nullptr, N, st);
        scal_setr_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, d_act, nrhs);
        cpm_count_launches(c, 1);
      }
      std::fill(replace.begin(), replace.end(), 1.0);
      std::fill(reset.begin(), reset.end(), 0.0);
      do_update = false;
    }
    if (it >= maxit) break;
    int steps = std::min(check_every, maxit - it);
    for (int k = 0; k < steps; ++k) {
      rc = iteration<float>(c, ap32, form, m, n, x32, w, tol, 0, st);
      if (rc) return rc;
    }
    CPM_CUDA_TRY(cudaGetLastError());
    it += steps;
    rc = read_scalars(w, st);
    if (rc) return rc;
    for (int q = 0; q < nrhs; ++q) {
      if (act[q] == 0.0) continue;
      const double *sq = w->h_pinned + q * NSC;
      // recursive residual dropped by delta since the last update, or reached
      // the tolerance: fold and replace; broke down or diverged: also restart
      if (sq[9] <= delta * delta * sq[14] || std::sqrt(sq[9]) <= tol * std::sqrt(sq[8])) do_update = true;
      if (sq[9] > 1e4 * sq[14]) do_update = true;  // the FP32 iteration is running away
      if (sq[10] != 0.0 || sq[13] != 0.0 || sq[5] == 0.0) {
        do_update = true;
        reset[q] = 1.0;
        ++nrestart;
      }
    }
    if (it - last_update >= max_between) do_update = true;
    if (nrestart > 40) { *broke = true; break; }
  }
  // fold what is left where it helps
  {
    candidate_kernel<<<g, 256, 0, st>>>(N, nrhs, ld, x, x32, w->fs);
    cpm_count_launches(c, 1);
    std::vector<double> rn2_prev = rn2;
    rc = residual64(c, ap64, m, n, f, w->fs, w, wrow, rn2, fn2, st);
    if (rc) return rc;
    bool rejected = false;
    for (int q = 0; q < nrhs; ++q) {
      acc[q] = (std::isfinite(rn2[q]) && rn2[q] <= rn2_prev[q]) ? 1.0 : 0.0;
      if (acc[q] == 0.0) rejected = true;
    }
    std::vector<double> ones(nrhs, 1.0);
    CPM_CUDA_TRY(cudaMemcpyAsync(d_act, acc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    CPM_CUDA_TRY(cudaMemcpyAsync(d_reset, ones.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    accept_kernel<<<g, 256, 0, st>>>(N, nrhs, ld, d_act, d_reset, w->fs, x, x32);
    cpm_count_launches(c, 1);
    if (rejected) {
      rc = residual64(c, ap64, m, n, f, x, w, wrow, rn2, fn2, st);
      if (rc) return rc;
    }
  }
  *iters = it;
  *updates = nupd;
  *restarts = nrestart;
  return CPM_OK;
}

static cpm_status solve_impl(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                             int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t st) {
  cpm_solve_opts opts{1e-10, 10000, CPM_SOLVE_FP64, 0.1, 200, 16, CPM_NORM_SCALED, 1000};
  if (o) opts = *o;
  if (opts.tol <= 0) opts.tol = 1e-10;
  if (opts.maxit <= 0) opts.maxit = 10000;
  if (opts.inner_tol <= 0 || opts.inner_tol >= 1) opts.inner_tol = 0.1;
  if (opts.max_refine <= 0) opts.max_refine = 200;
  if (opts.check_every <= 0) opts.check_every = 16;
  if (opts.inner_maxit <= 0) opts.inner_maxit = 1000;
  if (opts.norm != CPM_NORM_PLAIN) opts.norm = CPM_NORM_SCALED;
  const bool scaled = (opts.norm == CPM_NORM_SCALED);
  const bool trace = std::getenv("CPM_SOLVE_TRACE") != nullptr;
  const int64_t N = c->NS + c->NC;
  // Jacobi value of the PDE rows: 1/(m + n diag L) (Sec. 5.4)
  const double dS = 1.0 / (m + n * (-2.0 * c->dim / (c->h * c->h)));
  const double wrow = scaled ? dS : 1.0;  // residual weight of the PDE rows
  SolveWork *&w = adjoint ? c->solve_adj : c->solve;
  cpm_status rc;
  int iters = 0, restarts = 0, refinements = 0;
  bool broke = false;
  std::vector<double> rn2, fn2;
  ApplyFn<double> ap64 = adjoint ? cpm_apply_transpose_scaled_T<double> : cpm_apply_scaled_T<double>;
  // scaled: BiCGSTAB on (W A) x = W f, so its recursive residual is the
  // measured one; plain: the paper's right-preconditioned form
  KrylovForm form = scaled ? KrylovForm{1.0, dS, 4000.0, 0.0f} : KrylovForm{dS, 1.0, 4000.0, 0.0f};
  if (opts.mode == CPM_SOLVE_FP64) {
    rc = get_work(c, w, N, nrhs, ld, sizeof(double));
    if (rc) return rc;
    const double *rhs = f;
    if (scaled) {
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
    rc = get_work(c, w, N, nrhs, ld, sizeof(float));
    if (rc) return rc;
    ApplyFn<float> ap32 = adjoint ? cpm_apply_transpose_scaled_T<float> : cpm_apply_scaled_T<float>;
    // the FP32 iteration always runs on the row-scaled system (its residual is
    // balanced); the requested norm decides acceptance and convergence
    KrylovForm form32{1.0, dS, 4000.0, 0.5f};
    rc = bicgstab_reliable(c, ap64, ap32, form32, m, n, f, x, w, wrow, dS, opts.tol, opts.inner_tol, opts.inner_maxit,
                           opts.maxit, opts.max_refine, opts.check_every, trace, &iters, &refinements, &restarts,
                           &broke, rn2, fn2, st);
    if (rc) return rc;
    if (!(worst_relres(rn2, fn2) <= opts.tol) && iters < opts.maxit) {
      // FP64 finish from the current iterate for the columns the FP32 phase
      // left above tol (columns already converged stay frozen)
      if (trace) std::fprintf(stderr, "[cpm] FP64 finish from relres %.3e\n", worst_relres(rn2, fn2));
      SolveWork *&w64 = adjoint ? c->solve_adj64 : c->solve64;
      rc = get_work(c, w64, N, nrhs, ld, sizeof(double));
      if (rc) return rc;
      const double *rhs = f;
      if (scaled) {
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
  }
  return out;
}

cpm_status cpm_internal_solve(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                              int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t st) {
  return solve_impl(c, adjoint, m, n, f, x, nrhs, ld, o, stats, st);
}
