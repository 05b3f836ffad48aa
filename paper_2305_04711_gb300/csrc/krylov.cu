// krylov.cu -- preconditioned BiCGSTAB on the device (Sec. 5.4) and FP32 inner
// solves inside FP64 iterative refinement.
//
// The solver is van der Vorst's BiCGSTAB with right preconditioning by the
// diagonal of m I + n diag(L) on PDE rows and 1 on BC rows (Sec. 5.4).  All
// right-hand sides of a batch ([N][ld] layout) iterate together, each with its
// own scalars (rho, alpha, omega) kept in device memory, so a whole iteration
// runs without a host round trip; the host looks at the convergence flags every
// `check_every` iterations.  Dot products are deterministic: fixed-size block
// partials reduced in a fixed order by one block.  A right-hand side whose
// relative residual reaches the tolerance is frozen.  A near-zero rho restarts
// that right-hand side's shadow residual (r_hat = r); too many restarts is a
// breakdown.
#include <cmath>
#include <cstring>
#include <vector>

#include "apply.cuh"
#include "cpm_internal.cuh"
#include "krylov.cuh"

namespace {

constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs: fixed, so reductions are deterministic
constexpr int RED_THREADS = 256;

// partial sums of up to 3 dot products per column: out[blk][q][r]
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) dots_kernel(const T *__restrict__ a0, const T *__restrict__ b0,
                                                           const T *__restrict__ a1, const T *__restrict__ b1,
                                                           const T *__restrict__ a2, const T *__restrict__ b2, int nq,
                                                           int64_t N, int nrhs, int64_t ld, double *part) {
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
      acc0 += (double)a0[o] * (double)b0[o];
      if (nq > 1) acc1 += (double)a1[o] * (double)b1[o];
      if (nq > 2) acc2 += (double)a2[o] * (double)b2[o];
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
//                      [8] fnorm2 [9] rnorm2 [10] breakdown
constexpr int NSC = 11;

__global__ void scal_init_kernel(double *sc, const double *dots /* (r,r),(f,f) */, int nrhs, double tol) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  double *s = sc + r * NSC;
  s[0] = 1.0; s[1] = 1.0; s[2] = 1.0; s[3] = 0.0; s[4] = 0.0;
  s[6] = 0.0; s[7] = 0.0; s[10] = 0.0;
  double fn2 = dots[nrhs + r];
  s[8] = fn2 > 0.0 ? fn2 : 1.0;
  s[9] = dots[r];
  s[5] = (sqrt(s[9]) <= tol * sqrt(s[8])) ? 0.0 : 1.0;
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

__global__ void scal_conv_kernel(double *sc, const double *dots, int nrhs, double tol) {
  int r = threadIdx.x;
  if (r >= nrhs) return;
  double *s = sc + r * NSC;
  if (s[5] == 0.0) return;
  s[9] = dots[r];
  s[0] = s[3];
  if (!isfinite(s[9])) { s[10] = 1.0; s[5] = 0.0; return; }
  if (sqrt(s[9]) <= tol * sqrt(s[8])) s[5] = 0.0;
}

// ---- fused vector updates ---------------------------------------------------
template <typename T>
__device__ __forceinline__ T dinv_of(int64_t i, int64_t NS, T dS) { return (i < NS) ? dS : T(1); }

// p = restart ? r : r + beta (p - omega v);  ph = D p;  (restart: rhat = r)
template <typename T>
__global__ void upd_p_kernel(const double *sc, int64_t N, int64_t NS, int nrhs, int64_t ld, T dS, const T *r, T *rh,
                             T *p, const T *v, T *ph) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    const double *s = sc + c * NSC;
    if (s[5] == 0.0) continue;
    int64_t o = i * ld + c;
    T pv;
    if (s[6] != 0.0) {
      rh[o] = r[o];
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

// ---- mixed precision helpers -----------------------------------------------
// r64 = f - r64 (r64 holds A x); also writes r32 = r64 * inv_norm (per column, later)
__global__ void residual64_kernel(int64_t N, int nrhs, int64_t ld, const double *f, double *r) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    int64_t o = i * ld + c;
    r[o] = f[o] - r[o];
  }
}

__global__ void scale_to32_kernel(int64_t N, int nrhs, int64_t ld, const double *r, const double *nrm2,
                                  const double *active, float *r32, float *x32) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    int64_t o = i * ld + c;
    double n = sqrt(nrm2[c]);
    r32[o] = (n > 0.0 && active[c] != 0.0) ? (float)(r[o] / n) : 0.0f;
    x32[o] = 0.0f;
  }
}

__global__ void update64_kernel(int64_t N, int nrhs, int64_t ld, const double *nrm2, const float *d32, double *x,
                                const double *active) {
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < N * nrhs;
       tid += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = tid / nrhs;
    int c = (int)(tid - i * nrhs);
    if (active[c] == 0.0) continue;
    int64_t o = i * ld + c;
    x[o] += sqrt(nrm2[c]) * (double)d32[o];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
struct SolveWork {
  int nrhs = 0;
  int64_t ld = 0;
  int elem = 0;  // bytes per element of the Krylov vectors
  void *vec[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double *r64 = nullptr, *t64 = nullptr;  // FP64 residual / product (IR mode)
  void *x32 = nullptr;  // FP32 inner right-hand side (IR mode)
  void *d32 = nullptr;  // FP32 inner solution (IR mode)
  double *part = nullptr, *dots = nullptr, *sc = nullptr;
  double *h_pinned = nullptr;  // host mirror of sc (+ spare)
  double *active64 = nullptr;  // per column outer-active flags (IR)
};

static void free_work(SolveWork *w) {
  if (!w) return;
  for (auto &p : w->vec) cudaFree(p);
  cudaFree(w->r64); cudaFree(w->t64); cudaFree(w->x32); cudaFree(w->d32); cudaFree(w->part); cudaFree(w->dots); cudaFree(w->sc);
  cudaFree(w->active64);
  if (w->h_pinned) cudaFreeHost(w->h_pinned);
  delete w;
}

void cpm_free_solve(cpm_ctx *c) {
  free_work(c->solve);
  free_work(c->solve_adj);
  c->solve = nullptr;
  c->solve_adj = nullptr;
}

static cpm_status get_work(SolveWork *&w, int64_t N, int nrhs, int64_t ld, int elem, bool ir) {
  if (w && w->nrhs == nrhs && w->ld == ld && w->elem == elem && (!ir || w->r64)) return CPM_OK;
  free_work(w);
  w = new SolveWork;
  w->nrhs = nrhs; w->ld = ld; w->elem = elem;
  size_t vb = (size_t)N * (size_t)ld * (size_t)elem;
  for (auto &p : w->vec) CPM_CUDA_TRY(cudaMalloc(&p, vb));
  if (ir) {
    CPM_CUDA_TRY(cudaMalloc(&w->r64, (size_t)N * ld * sizeof(double)));
    CPM_CUDA_TRY(cudaMalloc(&w->t64, (size_t)N * ld * sizeof(double)));
    CPM_CUDA_TRY(cudaMalloc(&w->x32, (size_t)N * ld * sizeof(float)));
    CPM_CUDA_TRY(cudaMalloc(&w->d32, (size_t)N * ld * sizeof(float)));
  }
  CPM_CUDA_TRY(cudaMalloc(&w->part, sizeof(double) * RED_BLOCKS * 3 * nrhs));
  CPM_CUDA_TRY(cudaMalloc(&w->dots, sizeof(double) * 3 * nrhs));
  CPM_CUDA_TRY(cudaMalloc(&w->sc, sizeof(double) * NSC * nrhs));
  CPM_CUDA_TRY(cudaMalloc(&w->active64, sizeof(double) * nrhs));
  CPM_CUDA_TRY(cudaMallocHost(&w->h_pinned, sizeof(double) * (NSC + 3) * nrhs));
  return CPM_OK;
}

template <typename T>
static void dots(SolveWork *w, int nq, const T *a0, const T *b0, const T *a1, const T *b1, const T *a2, const T *b2,
                 int64_t N, cudaStream_t st) {
  dots_kernel<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a0, b0, a1, b1, a2, b2, nq, N, w->nrhs, w->ld, w->part);
  reduce_parts_kernel<<<1, 256, 0, st>>>(w->part, RED_BLOCKS, nq, w->nrhs, w->dots);
}

template <typename T>
using ApplyFn = cpm_status (*)(cpm_ctx *, double, double, const T *, T *, int, int64_t, cudaStream_t);

// BiCGSTAB on A x = f in precision T; x holds the initial guess.  Returns the
// number of iterations in *iters; per-column scalars stay in w->sc.
template <typename T>
static cpm_status bicgstab(cpm_ctx *c, ApplyFn<T> apply, double m, double n, const T *f, T *x, SolveWork *w,
                           double tol, int maxit, int check_every, int *iters, int *restarts, bool *broke,
                           cudaStream_t st) {
  const int64_t N = c->NS + c->NC, NS = c->NS;
  const int nrhs = w->nrhs;
  const int64_t ld = w->ld;
  T *r = (T *)w->vec[0], *rh = (T *)w->vec[1], *p = (T *)w->vec[2], *v = (T *)w->vec[3], *s = (T *)w->vec[4],
    *t = (T *)w->vec[5], *ph = (T *)w->vec[6], *sh = (T *)w->vec[7];
  const T dS = T(1.0 / (m + n * (-2.0 * c->dim / (c->h * c->h))));
  const unsigned g = cpm_grid(N * nrhs, 256);
  cpm_status rc = apply(c, m, n, x, r, nrhs, ld, st);
  if (rc) return rc;
  init_r_kernel<T><<<g, 256, 0, st>>>(N, nrhs, ld, f, r, rh, p, v);
  dots<T>(w, 2, r, r, f, f, nullptr, nullptr, N, st);
  scal_init_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs, tol);
  int it = 0;
  *broke = false;
  while (true) {
    // host check of the flags
    CPM_CUDA_TRY(cudaMemcpyAsync(w->h_pinned, w->sc, sizeof(double) * NSC * nrhs, cudaMemcpyDeviceToHost, st));
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
    bool any = false;
    int rs = 0;
    for (int q = 0; q < nrhs; ++q) {
      const double *sq = w->h_pinned + q * NSC;
      if (sq[5] != 0.0) any = true;
      if (sq[10] != 0.0) *broke = true;
      rs += (int)sq[7];
    }
    *restarts = rs;
    if (!any || it >= maxit) break;
    int steps = std::min(check_every, maxit - it);
    for (int k = 0; k < steps; ++k) {
      dots<T>(w, 2, rh, r, rh, rh, nullptr, nullptr, N, st);
      scal_rho_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs);
      upd_p_kernel<T><<<g, 256, 0, st>>>(w->sc, N, NS, nrhs, ld, dS, r, rh, p, v, ph);
      rc = apply(c, m, n, ph, v, nrhs, ld, st);
      if (rc) return rc;
      dots<T>(w, 1, rh, v, nullptr, nullptr, nullptr, nullptr, N, st);
      scal_alpha_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs);
      upd_s_kernel<T><<<g, 256, 0, st>>>(w->sc, N, NS, nrhs, ld, dS, r, v, s, sh);
      rc = apply(c, m, n, sh, t, nrhs, ld, st);
      if (rc) return rc;
      dots<T>(w, 2, t, s, t, t, nullptr, nullptr, N, st);
      scal_omega_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs);
      upd_xr_kernel<T><<<g, 256, 0, st>>>(w->sc, N, nrhs, ld, x, r, ph, sh, s, t);
      dots<T>(w, 1, r, r, nullptr, nullptr, nullptr, nullptr, N, st);
      scal_conv_kernel<<<1, 256, 0, st>>>(w->sc, w->dots, nrhs, tol);
    }
    CPM_CUDA_TRY(cudaGetLastError());
    it += steps;
  }
  *iters = it;
  return CPM_OK;
}

// FP64 residual r = f - A x and its squared norms (f,f), (r,r) per column
static cpm_status residual64(cpm_ctx *c, ApplyFn<double> apply, double m, double n, const double *f, const double *x,
                             SolveWork *w, std::vector<double> &rn2, std::vector<double> &fn2, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  cpm_status rc = apply(c, m, n, x, w->r64, w->nrhs, w->ld, st);
  if (rc) return rc;
  residual64_kernel<<<cpm_grid(N * w->nrhs, 256), 256, 0, st>>>(N, w->nrhs, w->ld, f, w->r64);
  dots<double>(w, 2, w->r64, w->r64, f, f, nullptr, nullptr, N, st);
  CPM_CUDA_TRY(cudaMemcpyAsync(w->h_pinned, w->dots, sizeof(double) * 2 * w->nrhs, cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  rn2.assign(w->h_pinned, w->h_pinned + w->nrhs);
  fn2.assign(w->h_pinned + w->nrhs, w->h_pinned + 2 * w->nrhs);
  return CPM_OK;
}

static cpm_status solve_impl(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                             int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t st) {
  cpm_solve_opts opts{1e-10, 10000, CPM_SOLVE_FP64, 1e-4, 30, 16};
  if (o) opts = *o;
  if (opts.tol <= 0) opts.tol = 1e-10;
  if (opts.maxit <= 0) opts.maxit = 10000;
  if (opts.inner_tol <= 0) opts.inner_tol = 1e-4;
  if (opts.max_refine <= 0) opts.max_refine = 30;
  if (opts.check_every <= 0) opts.check_every = 16;
  const int64_t N = c->NS + c->NC;
  SolveWork *&w = adjoint ? c->solve_adj : c->solve;
  cpm_status rc;
  int iters = 0, restarts = 0, refinements = 0;
  bool broke = false;
  double relres = 0.0;
  std::vector<double> rn2, fn2;
  if (opts.mode == CPM_SOLVE_FP64) {
    rc = get_work(w, N, nrhs, ld, sizeof(double), true);
    if (rc) return rc;
    ApplyFn<double> ap = adjoint ? cpm_apply_transpose_T<double> : cpm_apply_T<double>;
    rc = bicgstab<double>(c, ap, m, n, f, x, w, opts.tol, opts.maxit, opts.check_every, &iters, &restarts, &broke, st);
    if (rc) return rc;
    rc = residual64(c, ap, m, n, f, x, w, rn2, fn2, st);
    if (rc) return rc;
  } else if (opts.mode == CPM_SOLVE_FP32_IR) {
    rc = get_work(w, N, nrhs, ld, sizeof(float), true);
    if (rc) return rc;
    ApplyFn<double> ap64 = adjoint ? cpm_apply_transpose_T<double> : cpm_apply_T<double>;
    ApplyFn<float> ap32 = adjoint ? cpm_apply_transpose_T<float> : cpm_apply_T<float>;
    std::vector<double> act(nrhs, 1.0);
    rc = residual64(c, ap64, m, n, f, x, w, rn2, fn2, st);
    if (rc) return rc;
    while (true) {
      bool any = false;
      relres = 0.0;
      for (int q = 0; q < nrhs; ++q) {
        double fnq = fn2[q] > 0 ? std::sqrt(fn2[q]) : 1.0;
        double rr = std::sqrt(rn2[q]) / fnq;
        relres = std::max(relres, rr);
        act[q] = (rr > opts.tol) ? 1.0 : 0.0;
        any = any || act[q] != 0.0;
      }
      if (!any || refinements >= opts.max_refine || iters >= opts.maxit) break;
      ++refinements;
      // inner: A32 d = r / |r| (columns already converged stay at d = 0)
      CPM_CUDA_TRY(cudaMemcpyAsync(w->active64, act.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      CPM_CUDA_TRY(cudaMemcpyAsync(w->dots, rn2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      // keep a copy of |r|^2 in t64 (dots is reused by the inner solve)
      CPM_CUDA_TRY(cudaMemcpyAsync(w->t64, w->dots, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, st));
      float *rhs32 = (float *)w->x32;
      float *d32 = (float *)w->d32;
      scale_to32_kernel<<<cpm_grid(N * nrhs, 256), 256, 0, st>>>(N, nrhs, ld, w->r64, w->t64, w->active64, rhs32,
                                                                  d32);
      int it_in = 0, rs_in = 0;
      bool broke_in = false;
      int inner_max = opts.maxit - iters;
      rc = bicgstab<float>(c, ap32, m, n, rhs32, d32, w, opts.inner_tol, inner_max, opts.check_every, &it_in, &rs_in,
                           &broke_in, st);
      if (rc) return rc;
      iters += it_in;
      restarts += rs_in;
      update64_kernel<<<cpm_grid(N * nrhs, 256), 256, 0, st>>>(N, nrhs, ld, w->t64, d32, x, w->active64);
      rc = residual64(c, ap64, m, n, f, x, w, rn2, fn2, st);
      if (rc) return rc;
    }
  } else {
    return CPM_ERR_ARG;
  }
  relres = 0.0;
  for (int q = 0; q < nrhs; ++q) {
    double fnq = fn2[q] > 0 ? std::sqrt(fn2[q]) : 1.0;
    relres = std::max(relres, std::sqrt(rn2[q]) / fnq);
  }
  cpm_status out = CPM_OK;
  if (relres > opts.tol) out = broke ? CPM_ERR_BREAKDOWN : CPM_ERR_NOT_CONVERGED;
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
