// krylov.cu -- preconditioned BiCGSTAB on the device (Sec. 5.4), in FP64 or as
// FP32 inner solves of a mixed-precision iterative refinement.
//
// The solver is van der Vorst's BiCGSTAB with the diagonal D of m I + n diag(L)
// on PDE rows and 1 on BC rows as preconditioner (Sec. 5.4).  Two forms:
//  * plain (default, the paper's): right-preconditioned, A D mu = f with
//    x = D mu; the recursive residual is the unscaled f - A x, and the
//    stopping test is |f - A x|_2 <= tol |f|_2 per right-hand side;
//  * scaled: BiCGSTAB on the row-scaled system (W A) x = W f, W = D^-1, whose
//    residual is the Jacobi-scaled one.
// D never becomes a vector pass: the operator applies it as a column (right)
// or row (left) factor of the PDE entries, and the solution update folds it in.
//
// One iteration is five vector kernels and two operator products:
//   p  = r + beta (p - omega v)            (shadow restart: rhat = w r, p = r)
//   v  = A D p;  (rhat, v) -> alpha        (dot kernel, last block finishes)
//   s  = r - alpha v
//   t  = A D s;  (t, s), (t, t) -> omega
//   x += D (alpha p + omega s);  r = s - omega t;
//        (r, r), (rhat, r), (rhat, rhat), (w r, r) -> convergence, rho, beta
// Every dot product is reduced deterministically: a fixed grid of blocks, each
// reducing its rows in a fixed order (warp shuffles, then shared memory) to a
// partial per right-hand side, and the last block to arrive (atomic ticket)
// summing the partials in block order and updating the per-right-hand-side
// scalars (rho, alpha, omega, beta, convergence flags) on the device.  The
// iterations therefore need no host round trip; the host reads the flags every
// `check_every` iterations, and on an internal stream replays those iteration
// groups from a captured CUDA graph.  All right-hand sides of a batch ([N][ld]
// layout) iterate together with their own scalars; a right-hand side that
// converges is frozen.
//
// The FP32 form is mixed-precision iterative refinement: FP32 BiCGSTAB (FP32
// operator in its difference form, FP32 Krylov vectors) on the correction
// equation, the correction added to the FP64 solution; every time a column's
// FP32 residual has fallen by inner_tol the FP64 residual f - A x restarts it in
// a fresh Krylov space (see ir_refine).  Convergence is decided
// on the FP64 residual only; a column that stops gaining finishes in FP64.
//
// Workspaces are reserved by cpm_set_boundary / cpm_reserve; solves allocate
// nothing.
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

constexpr int KT = 512;    // threads per block of the vector kernels
constexpr int NQMAX = 4;   // dot products reduced by one kernel at most
// elements per thread in flight in the vector loops (16 bytes of each vector)
template <typename T>
constexpr int unroll_of() { return (sizeof(T) == 8) ? 2 : 4; }

// per right-hand side scalar slots
enum {
  S_RHO_OLD = 0, S_ALPHA, S_OMEGA, S_RHO, S_BETA, S_ACTIVE, S_RESTART, S_NRESTART, S_FN2, S_RN2, S_BROKE,
  S_BEST, S_STALL, S_STOPPED, S_RN2_0, S_ITERS, NSC
};

enum { ST_OUT = 0, ST_INIT, ST_ALPHA, ST_OMEGA, ST_XR };

struct Red {
  double *part;      // [G][NQMAX][nrhs] block partials
  unsigned *ticket;  // arrival counter (reset by the last block)
  double *sc;        // [nrhs][NSC]
  double *out;       // [NQMAX][nrhs] reduced dot products (ST_OUT / ST_INIT)
  int nrhs;
};

struct Conv {
  double tol;     // relative tolerance on the iterated system's residual
  double stall;   // iterations without the residual halving before giving up
  float mix;      // shadow = r o (1 + mix u) (shadow 0; mix 0: the classical rhat = r)
  int shadow;     // 0: rhat from r as above; 1: rhat = u, independent of r
  unsigned seed;  // of the hash u
};

// a fixed hash u(i, c, seed) in [-1, 1]
__device__ __forceinline__ float hash_unit(int64_t i, int c, unsigned seed) {
  uint64_t k = (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)c * 0xD1B54A32D192ED03ull +
               (uint64_t)seed * 0x94D049BB133111EBull;
  k ^= k >> 31; k *= 0xBF58476D1CE4E5B9ull; k ^= k >> 29;
  return (float)((k >> 40) & 0xFFFFFF) * (2.0f / 16777215.0f) - 1.0f;
}

// The shadow residual rhat of a (re)start, given the residual r there.
// rhat = r is the classical choice, but when r is supported on few rows (a
// right-hand side on the BC rows only) A r lives elsewhere and (rhat, A r) = 0:
// the first step breaks down.  A random rhat (shadow 1) meets every row; its
// (rhat, r) ~ |rhat| |r| / sqrt(N) is still far above the rounding of the dot
// products.  `restarts` selects a fresh hash after a near-breakdown.
__device__ __forceinline__ float shadow_of(const Conv &cv, int64_t i, int c, float r, unsigned restarts) {
  if (cv.shadow == 1) return hash_unit(i, c, cv.seed + restarts);
  if (cv.mix == 0.0f) return r;
  return r * (1.0f + cv.mix * hash_unit(i, c, 0u));
}
__device__ __forceinline__ double shadow_of(const Conv &cv, int64_t i, int c, double r, unsigned restarts) {
  if (cv.shadow == 1) return (double)hash_unit(i, c, cv.seed + restarts);
  if (cv.mix == 0.0f) return r;
  return r * (1.0 + (double)cv.mix * (double)hash_unit(i, c, 0u));
}

// ---- deterministic block reduction -----------------------------------------
// Thread t of a block owns column c = t % nrhs and rows sub, sub + rows_per,
// ... of the block's share (sub = t / nrhs, rows_per = KT / nrhs).
template <int NQ>
__device__ __forceinline__ bool block_publish(const double (&acc)[NQ], const Red &R) {
  __shared__ double sh[NQ][KT];
  __shared__ bool s_last;
  const int t = threadIdx.x, nrhs = R.nrhs;
  if (nrhs < 32 && (32 % nrhs) == 0) {
    // lanes with equal column combine by xor shuffles, then the warps in order
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = acc[q];
    for (int off = 16; off >= nrhs; off >>= 1)
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    const int lane = t & 31, w = t >> 5;
    if (lane < nrhs)
#pragma unroll
      for (int q = 0; q < NQ; ++q) sh[q][w * nrhs + lane] = v[q];
    __syncthreads();
    if (t < nrhs)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int k = 0; k < KT / 32; ++k) s += sh[q][k * nrhs + t];
        R.part[((int64_t)blockIdx.x * NQMAX + q) * nrhs + t] = s;
      }
  } else {
    const int rows_per = KT / nrhs;
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[q][t] = acc[q];
    __syncthreads();
    if (t < nrhs)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int k = 0; k < rows_per; ++k) s += sh[q][k * nrhs + t];
        R.part[((int64_t)blockIdx.x * NQMAX + q) * nrhs + t] = s;
      }
  }
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = (atomicAdd(R.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  return s_last;
}

__device__ void stage_finish(int stage, const Red &R, const Conv &cv, int c, const double *d) {
  double *s = R.sc + c * NSC;
  if (stage == ST_OUT) return;
  if (stage == ST_INIT) {
    const double fn2 = d[1] > 0.0 ? d[1] : 1.0;
    s[S_FN2] = fn2;
    s[S_RN2] = d[0]; s[S_BEST] = d[0]; s[S_RN2_0] = d[0];
    s[S_RHO] = d[2]; s[S_RHO_OLD] = 1.0; s[S_ALPHA] = 1.0; s[S_OMEGA] = 1.0; s[S_BETA] = 0.0;
    s[S_RESTART] = 0.0; s[S_NRESTART] = 0.0; s[S_BROKE] = 0.0; s[S_STALL] = 0.0; s[S_STOPPED] = 0.0;
    s[S_ITERS] = 0.0;
    const bool fin = isfinite(d[0]);
    s[S_ACTIVE] = (!fin || sqrt(d[0]) <= cv.tol * sqrt(fn2)) ? 0.0 : 1.0;
    if (!fin) s[S_STOPPED] = 1.0;
    return;
  }
  if (s[S_ACTIVE] == 0.0) return;
  if (stage == ST_ALPHA) {
    if (d[0] == 0.0 || !isfinite(d[0])) { s[S_BROKE] = 1.0; s[S_ACTIVE] = 0.0; return; }
    s[S_ALPHA] = s[S_RHO] / d[0];
    return;
  }
  if (stage == ST_OMEGA) {
    const double om = (d[1] > 0.0) ? d[0] / d[1] : 0.0;
    s[S_OMEGA] = om;
    if (om == 0.0 || !isfinite(om)) { s[S_BROKE] = 1.0; s[S_ACTIVE] = 0.0; }
    return;
  }
  // ST_XR: residual bookkeeping, then rho and beta of the next iteration
  s[S_ITERS] += 1.0;
  const double rn2 = d[0];
  s[S_RN2] = rn2;
  if (!isfinite(rn2) || rn2 > 1e16 * s[S_BEST]) { s[S_STOPPED] = 1.0; s[S_ACTIVE] = 0.0; return; }
  if (sqrt(rn2) <= cv.tol * sqrt(s[S_FN2])) { s[S_ACTIVE] = 0.0; return; }
  if (rn2 < 0.25 * s[S_BEST]) { s[S_BEST] = rn2; s[S_STALL] = 0.0; }
  else {
    s[S_STALL] += 1.0;
    if (s[S_STALL] > cv.stall) { s[S_STOPPED] = 1.0; s[S_ACTIVE] = 0.0; return; }
  }
  double rho = d[1];
  s[S_RESTART] = 0.0;
  if (fabs(rho) <= 1e-28 * sqrt(d[2]) * sqrt(rn2) || rho == 0.0) {
    // restart from a new shadow residual (the one the XR pass dotted with r
    // as d[3]): p = r, rho = (rhat', r)
    s[S_RESTART] = 1.0;
    s[S_NRESTART] += 1.0;
    if (s[S_NRESTART] > 20.0) { s[S_BROKE] = 1.0; s[S_ACTIVE] = 0.0; return; }
    rho = d[3];
    s[S_RHO] = 1.0; s[S_ALPHA] = 1.0; s[S_OMEGA] = 1.0;
  }
  s[S_BETA] = (rho / s[S_RHO]) * (s[S_ALPHA] / s[S_OMEGA]);
  s[S_RHO_OLD] = s[S_RHO];
  s[S_RHO] = rho;
}

// the last block: sum the partials in block order (a warp per (q, c), lanes
// strided over the blocks, then an xor-shuffle tree, identical in every lane)
template <int NQ>
__device__ void finish_reduce(int stage, const Red &R, const Conv &cv) {
  __shared__ double sd[NQMAX][256];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nrhs = R.nrhs;
  const int G = gridDim.x;
  __threadfence();
  for (int pr = w; pr < NQ * nrhs; pr += KT / 32) {
    const int q = pr / nrhs, c = pr - q * nrhs;
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += __ldcg(R.part + ((int64_t)b * NQMAX + q) * nrhs + c);
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) sd[q][c] = s;
  }
  __syncthreads();
  if (t < nrhs) {
    double d[NQMAX] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < NQ; ++q) d[q] = sd[q][t];
    if (stage == ST_OUT || stage == ST_INIT)
#pragma unroll
      for (int q = 0; q < NQ; ++q) R.out[q * nrhs + t] = d[q];
    stage_finish(stage, R, cv, t, d);
  }
  if (t == 0) *R.ticket = 0u;
}

// grid-stride element loop with UNR elements per thread in flight; the body
// functor loads into its element state, then updates and accumulates.  Runs
// of 16 products are summed in T, the runs in FP64 (for FP32 vectors this
// keeps the FP64 pipe, 1/64 of the FP32 rate here, off the hot loop).
template <typename T, int NQ, class Body>
__device__ __forceinline__ void vloop(const Body &body, int64_t N, int nrhs, int64_t ld, double (&acc)[NQ]) {
  constexpr int UNR = unroll_of<T>();
  const int c = threadIdx.x % nrhs, sub = threadIdx.x / nrhs, rows_per = KT / nrhs;
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  if (sub >= rows_per || !body.on(c)) return;
  body.init(c);
  const int64_t stride = (int64_t)gridDim.x * rows_per;
  T run[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) run[q] = T(0);
  int k = 0;
  for (int64_t i0 = (int64_t)blockIdx.x * rows_per + sub; i0 < N; i0 += UNR * stride) {
    typename Body::Elt e[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < N) body.load(e[u], i, i * ld + c);
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < N) body.apply(e[u], i, i * ld + c, run);
    }
    k += UNR;
    if (k >= 16) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) { acc[q] += (double)run[q]; run[q] = T(0); }
      k = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] += (double)run[q];
}

// ---- iteration kernels -------------------------------------------------------
template <typename T>
struct PBody {
  const double *sc; Conv cv;
  const T *__restrict__ r; T *__restrict__ rh; T *__restrict__ p; const T *__restrict__ v;
  mutable int c_; mutable bool restart; mutable unsigned nres; mutable T beta, omega;
  struct Elt { T r, p, v; };
  __device__ bool on(int c) const { return sc[c * NSC + S_ACTIVE] != 0.0; }
  __device__ void init(int c) const {
    c_ = c;
    restart = sc[c * NSC + S_RESTART] != 0.0;
    nres = (unsigned)sc[c * NSC + S_NRESTART];
    beta = T(sc[c * NSC + S_BETA]);
    omega = T(sc[c * NSC + S_OMEGA]);
  }
  __device__ void load(Elt &e, int64_t, int64_t o) const {
    e.r = r[o];
    if (!restart) { e.p = p[o]; e.v = v[o]; }
  }
  __device__ void apply(Elt &e, int64_t i, int64_t o, T (&)[1]) const {
    if (restart) {
      rh[o] = shadow_of(cv, i, c_, e.r, nres);
      p[o] = e.r;
    } else {
      p[o] = e.r + beta * (e.p - omega * e.v);
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(KT, 2) kp_kernel(const double *sc, Conv cv, int64_t N, int nrhs, int64_t ld,
                                                const T *r, T *rh, T *p, const T *v) {
  PBody<T> b{sc, cv, r, rh, p, v};
  double acc[1];
  vloop<T, 1>(b, N, nrhs, ld, acc);
}

template <typename T>
struct SBody {
  const double *sc;
  const T *__restrict__ r; const T *__restrict__ v; T *__restrict__ s;
  mutable T alpha;
  struct Elt { T r, v; };
  __device__ bool on(int c) const { return sc[c * NSC + S_ACTIVE] != 0.0; }
  __device__ void init(int c) const { alpha = T(sc[c * NSC + S_ALPHA]); }
  __device__ void load(Elt &e, int64_t, int64_t o) const { e.r = r[o]; e.v = v[o]; }
  __device__ void apply(Elt &e, int64_t, int64_t o, T (&)[1]) const { s[o] = e.r - alpha * e.v; }
};

template <typename T>
__global__ void __launch_bounds__(KT, 2) ks_kernel(const double *sc, int64_t N, int nrhs, int64_t ld, const T *r,
                                                const T *v, T *s) {
  SBody<T> b{sc, r, v, s};
  double acc[1];
  vloop<T, 1>(b, N, nrhs, ld, acc);
}

// (a, b) [and (a, a)] with a stage finish
template <typename T, int NQ>
struct DotBody {
  const double *sc;
  const T *__restrict__ a; const T *__restrict__ b;
  struct Elt { T a, b; };
  __device__ bool on(int c) const { return sc == nullptr || sc[c * NSC + S_ACTIVE] != 0.0; }
  __device__ void init(int) const {}
  __device__ void load(Elt &e, int64_t, int64_t o) const { e.a = a[o]; if (NQ > 1 || b != a) e.b = b[o]; else e.b = e.a; }
  __device__ void apply(Elt &e, int64_t, int64_t, T (&run)[NQ]) const {
    run[0] += e.a * e.b;
    if (NQ > 1) run[NQ - 1] += e.a * e.a;
  }
};

template <typename T, int NQ>
__global__ void __launch_bounds__(KT, 2) dot_kernel(Red R, Conv cv, int stage, int64_t N, int64_t ld, const T *a,
                                                 const T *b) {
  DotBody<T, NQ> body{R.sc, a, b};
  double acc[NQ];
  vloop<T, NQ>(body, N, R.nrhs, ld, acc);
  if (block_publish<NQ>(acc, R)) finish_reduce<NQ>(stage, R, cv);
}

// x += D (alpha p + omega s);  r = s - omega t;  the XR dot products
template <typename T, typename TX>
struct XRBody {
  const double *sc; Conv cv; int64_t NS; T cs;
  TX *__restrict__ x; T *__restrict__ r; const T *__restrict__ rh; const T *__restrict__ p;
  const T *__restrict__ s; const T *__restrict__ t;
  mutable int c_; mutable unsigned nres; mutable T alpha, omega;
  struct Elt { TX x; T rh, p, s, t; };
  __device__ bool on(int c) const { return sc[c * NSC + S_ACTIVE] != 0.0; }
  __device__ void init(int c) const {
    c_ = c;
    nres = (unsigned)sc[c * NSC + S_NRESTART] + 1u;
    alpha = T(sc[c * NSC + S_ALPHA]);
    omega = T(sc[c * NSC + S_OMEGA]);
  }
  __device__ void load(Elt &e, int64_t, int64_t o) const {
    e.x = x[o]; e.rh = rh[o]; e.p = p[o]; e.s = s[o]; e.t = t[o];
  }
  __device__ void apply(Elt &e, int64_t i, int64_t o, T (&run)[4]) const {
    const T d = (i < NS) ? cs : T(1);
    x[o] = e.x + TX(d * (alpha * e.p + omega * e.s));
    const T rn = e.s - omega * e.t;
    r[o] = rn;
    run[0] += rn * rn;
    run[1] += e.rh * rn;
    run[2] += e.rh * e.rh;
    // (rhat', r) for the shadow residual a restart would take
    run[3] += shadow_of(cv, i, c_, rn, nres) * rn;
  }
};

template <typename T, typename TX>
__global__ void __launch_bounds__(KT, 2) kxr_kernel(Red R, Conv cv, int64_t N, int64_t NS, T cs, int64_t ld, TX *x,
                                                 T *r, const T *rh, const T *p, const T *s, const T *t) {
  XRBody<T, TX> body{R.sc, cv, NS, cs, x, r, rh, p, s, t};
  double acc[4];
  vloop<T, 4>(body, N, R.nrhs, ld, acc);
  if (block_publish<4>(acc, R)) finish_reduce<4>(ST_XR, R, cv);
}

// r = f - r (r holds A x, or nothing when x = 0);  rhat = shadow of r;
// p = v = 0;  (r, r), (f, f), (rhat, r) -> the initial scalars
template <typename T>
struct InitBody {
  const T *__restrict__ f; T *__restrict__ r; T *__restrict__ rh; T *__restrict__ p; T *__restrict__ v;
  bool x_zero; Conv cv;
  mutable int c_;
  struct Elt { T f, r; };
  __device__ bool on(int) const { return true; }
  __device__ void init(int c) const { c_ = c; }
  __device__ void load(Elt &e, int64_t, int64_t o) const { e.f = f[o]; e.r = x_zero ? T(0) : r[o]; }
  __device__ void apply(Elt &e, int64_t i, int64_t o, T (&run)[3]) const {
    const T rv = e.f - e.r;
    const T sh = shadow_of(cv, i, c_, rv, 0u);
    r[o] = rv; rh[o] = sh; p[o] = T(0); v[o] = T(0);
    run[0] += rv * rv;
    run[1] += e.f * e.f;
    run[2] += sh * rv;
  }
};

template <typename T>
__global__ void __launch_bounds__(KT, 2) init_kernel(Red R, Conv cv, int64_t N, int64_t ld, bool x_zero, const T *f,
                                                  T *r, T *rh, T *p, T *v) {
  InitBody<T> body{f, r, rh, p, v, x_zero, cv};
  double acc[3];
  vloop<T, 3>(body, N, R.nrhs, ld, acc);
  if (block_publish<3>(acc, R)) finish_reduce<3>(ST_INIT, R, cv);
}

// ---- FP64 residual -----------------------------------------------------------
// r = f - r (r holds A x) and the weighted norms |W r|^2, |W f|^2 with W = wrow
// on PDE rows and 1 on BC rows
struct ResidBody {
  const double *__restrict__ f; double *__restrict__ r; int64_t NS; double w2, v2;
  struct Elt { double f, r; };
  __device__ bool on(int) const { return true; }
  __device__ void init(int) const {}
  __device__ void load(Elt &e, int64_t, int64_t o) const { e.f = f[o]; e.r = r[o]; }
  __device__ void apply(Elt &e, int64_t i, int64_t o, double (&run)[3]) const {
    const double rv = e.f - e.r;
    r[o] = rv;
    const bool pde = i < NS;
    run[0] += (pde ? w2 : 1.0) * (rv * rv);
    run[1] += (pde ? w2 : 1.0) * (e.f * e.f);
    run[2] += (pde ? v2 : 1.0) * (rv * rv);
  }
};

// r = f - r and, per column, |W r|^2, |W f|^2 (W = sqrt(w2) on PDE rows) and
// |V r|^2 (V = sqrt(v2) on PDE rows; the norm of an iterated system)
__global__ void __launch_bounds__(KT, 2) resid_kernel(Red R, int64_t N, int64_t NS, double w2, double v2, int64_t ld,
                                                   const double *f, double *r) {
  ResidBody body{f, r, NS, w2, v2};
  double acc[3];
  vloop<double, 3>(body, N, R.nrhs, ld, acc);
  Conv cv{0.0, 0.0, 0.0f, 0, 0u};
  if (block_publish<3>(acc, R)) finish_reduce<3>(ST_OUT, R, cv);
}

// y = x o xi with xi(i, c) = +-1 from a fixed hash: the model of the rounding
// of x to FP64 (independent relative perturbations of each entry)
__global__ void sign_perturb_kernel(int64_t N, int nrhs, int64_t ld, const double *x, double *y) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    uint64_t k = (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)c * 0xD1B54A32D192ED03ull + 0x2545F4914F6CDD1Dull;
    k ^= k >> 31; k *= 0xBF58476D1CE4E5B9ull; k ^= k >> 29;
    const int64_t o = i * ld + c;
    y[o] = ((k >> 40) & 1ull) ? x[o] : -x[o];
  }
}

// |W y|^2 per column (W = wrow on PDE rows, 1 on BC rows)
struct WNormBody {
  const double *__restrict__ y; int64_t NS; double w2;
  struct Elt { double y; };
  __device__ bool on(int) const { return true; }
  __device__ void init(int) const {}
  __device__ void load(Elt &e, int64_t, int64_t o) const { e.y = y[o]; }
  __device__ void apply(Elt &e, int64_t i, int64_t, double (&run)[1]) const {
    run[0] += ((i < NS) ? w2 : 1.0) * (e.y * e.y);
  }
};

__global__ void __launch_bounds__(KT, 2) wnorm_kernel(Red R, int64_t N, int64_t NS, double w2, int64_t ld,
                                                      const double *y) {
  WNormBody body{y, NS, w2};
  double acc[1];
  vloop<double, 1>(body, N, R.nrhs, ld, acc);
  Conv cv{0.0, 0.0, 0.0f, 0, 0u};
  if (block_publish<1>(acc, R)) finish_reduce<1>(ST_OUT, R, cv);
}

// out = W f (PDE rows scaled by dS)
__global__ void scale_rows64_kernel(int64_t N, int64_t NS, int nrhs, int64_t ld, double dS, const double *f,
                                    double *out) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    out[o] = (i < NS) ? dS * f[o] : f[o];
  }
}

// refinement step: FP32 right-hand side W r / scale per selected column (scale
// 0: a column left out, zero right-hand side) and a zero correction d
__global__ void ir_rhs_kernel(int64_t N, int64_t NS, double wrow, int nrhs, int64_t ld, const double *scale,
                              const double *r64, float *f32, float *d32) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    double sc = scale[c];
    f32[o] = (sc > 0.0) ? (float)(((i < NS) ? wrow : 1.0) * r64[o] / sc) : 0.0f;
    d32[o] = 0.0f;
  }
}

// x += s_c d: the FP32 correction of an inner solve into the FP64 solution
// (s = nullptr: every column with s_c = 1; s_c = -1 takes a correction back)
__global__ void ir_add_kernel(int64_t N, int nrhs, int64_t ld, const double *s, const float *d32, double *x) {
  CPM_ROWS_COLS_LOOP(N, nrhs, i, c) {
    int64_t o = i * ld + c;
    const double sc = s ? s[c] : 1.0;
    if (sc != 0.0) x[o] += sc * (double)d32[o];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
struct GraphKey {
  const void *fn = nullptr;
  double m = 0, n = 0, rs = 0, cs = 0, tol = 0, stall = 0;
  float mix = 0;
  int shadow = 0;
  unsigned seed = 0;
  const void *x = nullptr, *vecs = nullptr;
  int nrhs = 0, steps = 0, elem = 0, xelem = 0, G = 0;
  int64_t ld = 0;
  bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

struct SolveWork {
  int64_t N = 0, ld = 0;     // reserved rows and leading dimension
  bool has32 = false;
  double *v64[6] = {};       // FP64 Krylov vectors (FP64 solves, FP64 finish of FP32_IR)
  float *v32[6] = {};        // FP32 Krylov vectors (FP32_IR inner solves)
  float *d32 = nullptr;      // FP32_IR correction of one inner solve
  double *r64 = nullptr;     // FP64 residual
  double *xc = nullptr;      // FP64 scratch of the rounding-floor estimate
  double *part = nullptr, *sc = nullptr, *out = nullptr, *cols = nullptr;
  unsigned *ticket = nullptr;
  double *h_pin = nullptr;   // host mirror: [NSC * ld] scalars, then [NQMAX * ld] dots
  int G = 0;                 // blocks of the vector kernels (fixed: deterministic reductions)
  cudaGraphExec_t gexec = nullptr;
  GraphKey gkey;
  int64_t glaunches = 0;     // kernels per replay
  bool graphs_ok = true;
};

static void free_work(SolveWork *w) {
  if (!w) return;
  for (auto p : w->v64) cudaFree(p);
  for (auto p : w->v32) cudaFree(p);
  cudaFree(w->d32);
  cudaFree(w->r64); cudaFree(w->xc);
  cudaFree(w->part); cudaFree(w->sc); cudaFree(w->out); cudaFree(w->cols); cudaFree(w->ticket);
  if (w->h_pin) cudaFreeHost(w->h_pin);
  if (w->gexec) cudaGraphExecDestroy(w->gexec);
  delete w;
}

void cpm_free_solve(cpm_ctx *c) {
  free_work(c->solve);
  c->solve = nullptr;
}

// Reserve the solve workspace for N x ld (FP64 vectors always; FP32 inner
// vectors and the refinement buffers with `fp32`).  The only allocation of the
// solve path; called from cpm_set_boundary and cpm_reserve.
cpm_status cpm_reserve_solve(cpm_ctx *c, int64_t ld, bool fp32) {
  const int64_t N = c->NS + c->NC;
  SolveWork *w = c->solve;
  if (w && w->N == N && w->ld >= ld && (w->has32 || !fp32)) return CPM_OK;
  if (w) { ld = std::max(ld, w->ld); fp32 = fp32 || w->has32; }
  free_work(w);
  c->solve = nullptr;
  w = new SolveWork;
  w->N = N; w->ld = ld; w->has32 = fp32;
  const size_t n = (size_t)std::max<int64_t>(N, 1) * (size_t)ld;
  cpm_status rc = CPM_OK;
  auto al = [&](void **p, size_t bytes) {
    if (rc == CPM_OK && cudaMalloc(p, bytes) != cudaSuccess) { (void)cudaGetLastError(); rc = CPM_ERR_OOM; }
  };
  for (auto &p : w->v64) al((void **)&p, n * sizeof(double));
  al((void **)&w->r64, n * sizeof(double));
  if (fp32) {
    for (auto &p : w->v32) al((void **)&p, n * sizeof(float));
    al((void **)&w->d32, n * sizeof(float));
    al((void **)&w->xc, n * sizeof(double));
  }
  w->G = 2 * c->nsm;
  // partials for up to 4 blocks per SM (the autotuner's widest choice)
  al((void **)&w->part, sizeof(double) * (size_t)(4 * c->nsm) * NQMAX * ld);
  al((void **)&w->sc, sizeof(double) * NSC * ld);
  al((void **)&w->out, sizeof(double) * NQMAX * ld);
  al((void **)&w->cols, sizeof(double) * 4 * ld);
  al((void **)&w->ticket, sizeof(unsigned));
  if (rc == CPM_OK && cudaMallocHost((void **)&w->h_pin, sizeof(double) * (NSC + NQMAX) * ld) != cudaSuccess) {
    (void)cudaGetLastError();
    rc = CPM_ERR_OOM;
  }
  if (rc == CPM_OK && cudaMemset(w->ticket, 0, sizeof(unsigned)) != cudaSuccess) rc = CPM_ERR_CUDA;
  if (rc != CPM_OK) { free_work(w); return rc; }
  c->solve = w;
  return CPM_OK;
}

namespace {

// operator product with a PDE-row scale R and a PDE-entry scale C: v = R A C u
// (or R A^T C u)
template <typename T>
using ApplyFn = cpm_status (*)(cpm_ctx *, double, double, double, double, const T *, T *, int, int64_t,
                               cudaStream_t);

template <typename T>
struct Op {
  ApplyFn<T> fn;
  double m, n, rowscale, colscale;
  cpm_status operator()(cpm_ctx *c, const T *u, T *v, int nrhs, int64_t ld, cudaStream_t st, bool plain_cols) const {
    return fn(c, m, n, rowscale, plain_cols ? 1.0 : colscale, u, v, nrhs, ld, st);
  }
};

template <typename T>
struct Vecs { T *r, *rh, *p, *v, *s, *t; };

Red red_of(SolveWork *w, int nrhs) { return Red{w->part, w->ticket, w->sc, w->out, nrhs}; }

// one BiCGSTAB iteration for all active columns (device only)
template <typename T, typename TX>
cpm_status iteration(cpm_ctx *c, const Op<T> &op, TX *x, const Vecs<T> &V, SolveWork *w, int nrhs, int64_t ld,
                     const Conv &cv, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  const Red R = red_of(w, nrhs);
  const unsigned G = (unsigned)w->G;
  kp_kernel<T><<<G, KT, 0, st>>>(w->sc, cv, N, nrhs, ld, V.r, V.rh, V.p, V.v);
  cpm_status rc = op(c, V.p, V.v, nrhs, ld, st, false);
  if (rc) return rc;
  dot_kernel<T, 1><<<G, KT, 0, st>>>(R, cv, ST_ALPHA, N, ld, V.rh, V.v);
  ks_kernel<T><<<G, KT, 0, st>>>(w->sc, N, nrhs, ld, V.r, V.v, V.s);
  rc = op(c, V.s, V.t, nrhs, ld, st, false);
  if (rc) return rc;
  dot_kernel<T, 2><<<G, KT, 0, st>>>(R, cv, ST_OMEGA, N, ld, V.t, V.s);
  kxr_kernel<T, TX><<<G, KT, 0, st>>>(R, cv, N, c->NS, T(op.colscale), ld, x, V.r, V.rh, V.p, V.s, V.t);
  cpm_count_launches(c, 5);
  return CPM_OK;
}

cpm_status read_scalars(SolveWork *w, int nrhs, cudaStream_t st) {
  CPM_CUDA_TRY(cudaMemcpyAsync(w->h_pin, w->sc, sizeof(double) * NSC * nrhs, cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  return CPM_OK;
}

// `steps` iterations: replayed from a cached graph when the group is a full
// one and nothing is being profiled, launched directly otherwise
template <typename T, typename TX>
cpm_status iterations(cpm_ctx *c, const Op<T> &op, TX *x, const Vecs<T> &V, SolveWork *w, int nrhs, int64_t ld,
                      const Conv &cv, int steps, bool graph, cudaStream_t st) {
  if (graph && w->graphs_ok && !c->prof.on) {
    GraphKey k;
    std::memset(&k, 0, sizeof(k));
    k.fn = (const void *)op.fn; k.m = op.m; k.n = op.n; k.rs = op.rowscale; k.cs = op.colscale;
    k.tol = cv.tol; k.stall = cv.stall; k.mix = cv.mix; k.shadow = cv.shadow; k.seed = cv.seed;
    k.x = x; k.vecs = V.r; k.nrhs = nrhs; k.steps = steps;
    k.elem = (int)sizeof(T); k.xelem = (int)sizeof(TX); k.ld = ld; k.G = w->G;
    if (!(w->gexec && w->gkey == k)) {
      if (w->gexec) { cudaGraphExecDestroy(w->gexec); w->gexec = nullptr; }
      const int64_t before = c->prof.launches;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      cpm_status rc = CPM_OK;
      if (e == cudaSuccess) {
        for (int s = 0; s < steps && rc == CPM_OK; ++s) rc = iteration<T, TX>(c, op, x, V, w, nrhs, ld, cv, st);
        e = cudaStreamEndCapture(st, &g);
      }
      if (rc == CPM_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&w->gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      w->glaunches = c->prof.launches - before;
      c->prof.launches = before;
      if (rc != CPM_OK || e != cudaSuccess) {
        // capture not available here: plain launches from now on
        (void)cudaGetLastError();
        if (w->gexec) { cudaGraphExecDestroy(w->gexec); w->gexec = nullptr; }
        w->graphs_ok = false;
        if (rc != CPM_OK) return rc;
        return iterations<T, TX>(c, op, x, V, w, nrhs, ld, cv, steps, false, st);
      }
      w->gkey = k;
    }
    CPM_CUDA_TRY(cudaGraphLaunch(w->gexec, st));
    cpm_count_launches(c, (int)w->glaunches);
    return CPM_OK;
  }
  for (int s = 0; s < steps; ++s) {
    cpm_status rc = iteration<T, TX>(c, op, x, V, w, nrhs, ld, cv, st);
    if (rc) return rc;
  }
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}

// BiCGSTAB iterations for all active columns until none is active or maxit:
// the host reads the per-column flags every check_every iterations
template <typename T, typename TX>
cpm_status krylov_run(cpm_ctx *c, const Op<T> &op, TX *x, const Vecs<T> &V, SolveWork *w, int nrhs, int64_t ld,
                      const Conv &cv, int maxit, int check_every, int *iters, int *restarts, bool *broke,
                      cudaStream_t st) {
  int it = 0;
  const bool graph = std::getenv("CPM_NO_GRAPHS") == nullptr;
  const bool trace = std::getenv("CPM_SOLVE_TRACE") != nullptr;
  while (true) {
    cpm_status rc = read_scalars(w, nrhs, st);
    if (rc) return rc;
    bool any = false;
    int nrestart = 0, nact = 0, nbroke = 0, nstop = 0;
    double worst = 0.0;
    for (int q = 0; q < nrhs; ++q) {
      const double *sq = w->h_pin + q * NSC;
      if (sq[S_ACTIVE] != 0.0) { any = true; ++nact; }
      if (sq[S_BROKE] != 0.0) { *broke = true; ++nbroke; }
      if (sq[S_STOPPED] != 0.0) ++nstop;
      nrestart += (int)sq[S_NRESTART];
      worst = std::max(worst, std::sqrt(sq[S_RN2] / sq[S_FN2]));
    }
    *restarts = nrestart;
    if (trace)
      std::fprintf(stderr, "[cpm it] %d recursive relres[0] %.3e worst %.3e active %d broke %d stopped %d restarts %d\n",
                   it, std::sqrt(w->h_pin[S_RN2] / w->h_pin[S_FN2]), worst, nact, nbroke, nstop, nrestart);
    if (!any || it >= maxit) break;
    const int steps = std::min(check_every, maxit - it);
    rc = iterations<T, TX>(c, op, x, V, w, nrhs, ld, cv, steps, graph && steps == check_every, st);
    if (rc) return rc;
    it += steps;
  }
  *iters = it;
  return CPM_OK;
}

// BiCGSTAB on the iterated system (op) with right-hand side f; x holds the
// initial guess (x_zero: x = 0, which a wider accumulator TX requires)
template <typename T, typename TX>
cpm_status bicgstab(cpm_ctx *c, const Op<T> &op, const T *f, TX *x, bool x_zero, const Vecs<T> &V, SolveWork *w,
                    int nrhs, int64_t ld, const Conv &cv, int maxit, int check_every, int *iters, int *restarts,
                    bool *broke, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  const Red R = red_of(w, nrhs);
  cpm_status rc = CPM_OK;
  if (!x_zero) {
    if constexpr (std::is_same<T, TX>::value) {
      rc = op(c, x, V.r, nrhs, ld, st, true);  // r = R A x (x in the original variables)
      if (rc) return rc;
    } else {
      return CPM_ERR_ARG;
    }
  }
  init_kernel<T><<<(unsigned)w->G, KT, 0, st>>>(R, cv, N, ld, x_zero, f, V.r, V.rh, V.p, V.v);
  cpm_count_launches(c, 1);
  *broke = false;
  return krylov_run<T, TX>(c, op, x, V, w, nrhs, ld, cv, maxit, check_every, iters, restarts, broke, st);
}

// FP64 residual r64 = f - A x and its squared weighted norms per column:
// |W r|^2 and |W f|^2 with W = diag(wrow on PDE rows, 1 on BC rows)
cpm_status residual64(cpm_ctx *c, ApplyFn<double> fn, double m, double n, const double *f, const double *x,
                      SolveWork *w, int nrhs, int64_t ld, double wrow, std::vector<double> &rn2,
                      std::vector<double> &fn2, cudaStream_t st, double vrow = 1.0,
                      std::vector<double> *rv2 = nullptr) {
  const int64_t N = c->NS + c->NC;
  cpm_status rc = fn(c, m, n, 1.0, 1.0, x, w->r64, nrhs, ld, st);
  if (rc) return rc;
  resid_kernel<<<(unsigned)w->G, KT, 0, st>>>(red_of(w, nrhs), N, c->NS, wrow * wrow, vrow * vrow, ld, f, w->r64);
  cpm_count_launches(c, 1);
  CPM_CUDA_TRY(cudaMemcpyAsync(w->h_pin, w->out, sizeof(double) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  rn2.assign(w->h_pin, w->h_pin + nrhs);
  fn2.assign(w->h_pin + nrhs, w->h_pin + 2 * nrhs);
  if (rv2) rv2->assign(w->h_pin + 2 * nrhs, w->h_pin + 3 * nrhs);
  return CPM_OK;
}

double relres_of(double rn2, double fn2) {
  double fnq = fn2 > 0 ? std::sqrt(fn2) : 1.0;
  double rr = std::sqrt(rn2) / fnq;
  return std::isfinite(rr) ? rr : INFINITY;
}

// The FP64 rounding floor of the true residual: storing the exact solution in
// FP64 perturbs each entry by up to half an ulp, and the operator amplifies
// that noise by about its row norm (O(1/h^2) on PDE rows), so the relative
// residual of any FP64 x cannot fall much below
//   floor = (u / sqrt 3) |W A (x o xi)|_2 / |W f|_2,   u = 2^-53,
// with xi a fixed random +-1 vector (the rounding model: independent relative
// errors of variance u^2 / 3).  A column converges when its true relative
// residual is at most max(tol, 4 floor).  Needs two [N][ld] FP64 scratch vectors.
cpm_status floor64(cpm_ctx *c, ApplyFn<double> fn, double m, double n, const double *x, double *y, double *Ay,
                   SolveWork *w, int nrhs, int64_t ld, double wrow, const std::vector<double> &fn2,
                   std::vector<double> &floors, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  sign_perturb_kernel<<<cpm_grid(N * nrhs, 256), 256, 0, st>>>(N, nrhs, ld, x, y);
  cpm_status rc = fn(c, m, n, 1.0, 1.0, y, Ay, nrhs, ld, st);
  if (rc) return rc;
  wnorm_kernel<<<(unsigned)w->G, KT, 0, st>>>(red_of(w, nrhs), N, c->NS, wrow * wrow, ld, Ay);
  cpm_count_launches(c, 2);
  CPM_CUDA_TRY(cudaMemcpyAsync(w->h_pin, w->out, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  const double u = std::ldexp(1.0, -53);
  floors.resize(nrhs);
  for (int q = 0; q < nrhs; ++q) floors[q] = (u / std::sqrt(3.0)) * relres_of(w->h_pin[q], fn2[q]);
  return CPM_OK;
}

// converged: within tol, or within four times the rounding floor
bool done_col(double rn2, double fn2, double tol, double floor_q) {
  const double r = relres_of(rn2, fn2);
  return r <= tol || r <= 4.0 * floor_q;
}

double worst_relres(const std::vector<double> &rn2, const std::vector<double> &fn2) {
  double worst = 0.0;
  for (size_t q = 0; q < rn2.size(); ++q) worst = std::max(worst, relres_of(rn2[q], fn2[q]));
  return worst;
}

// Mixed-precision iterative refinement: FP32 BiCGSTAB on the correction
// equation (the iterated form of A d = r), d accumulated in FP32 and added to
// the FP64 solution x at each refinement.  Whenever a column's recursive FP32 residual has dropped by
// `delta` relative to the start of the inner solve, the host computes the FP64
// residual r = f - A x (difference-form product, accurate to the FP64 rounding
// of local differences), stops the columns that meet tol there, and restarts
// the FP32 iteration of the others from r (scaled as the iterated form needs)
// with a fresh Krylov space: p = 0 and a random shadow residual.  Keeping p and
// rhat across the refinement (residual replacement) was tried and lets FP32
// BiCGSTAB drift into large residual spikes on fine torus grids after a few
// hundred iterations (the bi-orthogonality of an old shadow residual is lost in
// FP32), whereas fresh inner solves of about a hundred iterations each reduce
// the FP64 residual by delta steadily.  The random shadow matters: the first
// residual lives on the BC rows only, so rhat = r gives (rhat, A r) = 0.  A
// column whose FP64 residual fails to fall over three refinements is left for
// the FP64 finish.  rhs_w weights the PDE rows of the FP32 residual: the scaling
// of the left-scaled form, or 1 for a right-preconditioned form.
cpm_status ir_refine(cpm_ctx *c, ApplyFn<double> ap64, const Op<float> &op32, double m, double n,
                       const double *f, double *x, SolveWork *w, int nrhs, int64_t ld, double wrow, double rhs_w,
                       double tol, double delta, int maxit, int max_repl, int check_every, bool trace, int *iters,
                       int *nrepl_out, int *restarts, std::vector<double> &rn2, std::vector<double> &fn2,
                       std::vector<double> &floors, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  const unsigned g = cpm_grid(N * nrhs, 256);
  Vecs<float> V{w->v32[0], w->v32[1], w->v32[2], w->v32[3], w->v32[4], w->v32[5]};
  float *f32 = w->v32[5];  // first right-hand side: read by the init kernel before t is written
  Conv cv{delta, 400.0, 0.0f, 1, 1u};
  const Red R = red_of(w, nrhs);
  std::vector<double> flag(nrhs, 0.0), prev(nrhs, INFINITY);
  std::vector<int> stall(nrhs, 0), taken(nrhs, 0);
  floors.assign(nrhs, 0.0);
  // the residual in the iterated system's norm (rhs_w on the PDE rows) decides
  // whether a refinement step is kept: the plain norm may rise while the
  // residual moves off the BC rows
  std::vector<double> rv2, rv2_old;
  cpm_status rc = residual64(c, ap64, m, n, f, x, w, nrhs, ld, wrow, rn2, fn2, st, rhs_w, &rv2);
  if (rc) return rc;
  int it_total = 0, nrep = 0, nrs = 0;
  while (true) {
    // the rounding floor matters once the residual nears the tolerance
    if (worst_relres(rn2, fn2) > tol && worst_relres(rn2, fn2) < 1e3 * tol) {
      rc = floor64(c, ap64, m, n, x, w->xc, w->v64[0], w, nrhs, ld, wrow, fn2, floors, st);
      if (rc) return rc;
    }
    bool any = false;
    for (int q = 0; q < nrhs; ++q) {
      flag[q] = 0.0;
      if (done_col(rn2[q], fn2[q], tol, floors[q])) continue;
      // a refinement that does not halve the residual is a stall (the first
      // ones may raise the plain norm: the residual moves off the BC rows);
      // three in a row leave the column to the FP64 finish
      if (stall[q] >= 3) continue;
      if (rn2[q] < 0.25 * prev[q]) stall[q] = 0;
      else if (!taken[q] && ++stall[q] >= 3) continue;
      taken[q] = 0;
      prev[q] = rn2[q];
      flag[q] = 1.0;
      any = true;
    }
    if (trace)
      std::fprintf(stderr, "[cpm ir] refinement %d it %d relres[0] %.3e worst %.3e\n", nrep, it_total,
                   relres_of(rn2[0], fn2[0]), worst_relres(rn2, fn2));
    if (!any || it_total >= maxit || nrep >= max_repl) break;
    CPM_CUDA_TRY(cudaMemcpyAsync(w->cols, flag.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    // r = W r64 on the selected columns (0 elsewhere), d = 0, a fresh Krylov
    // space; the correction accumulates in FP32 (it is needed to about delta)
    ir_rhs_kernel<<<g, 256, 0, st>>>(N, c->NS, rhs_w, nrhs, ld, w->cols, w->r64, f32, w->d32);
    // each step draws its own shadow residual, so that a step taken back is
    // not repeated identically
    cv.seed = 1u + 7919u * (unsigned)nrep;
    init_kernel<float><<<(unsigned)w->G, KT, 0, st>>>(R, cv, N, ld, true, f32, V.r, V.rh, V.p, V.v);
    cpm_count_launches(c, 2);
    ++nrep;
    int it = 0, rs = 0;
    bool broke = false;
    rc = krylov_run<float, float>(c, op32, w->d32, V, w, nrhs, ld, cv, maxit - it_total, check_every, &it, &rs,
                                  &broke, st);
    if (rc) return rc;
    ir_add_kernel<<<g, 256, 0, st>>>(N, nrhs, ld, nullptr, w->d32, x);
    cpm_count_launches(c, 1);
    it_total += it;
    nrs += rs;
    rv2_old = rv2;
    rc = residual64(c, ap64, m, n, f, x, w, nrhs, ld, wrow, rn2, fn2, st, rhs_w, &rv2);
    if (rc) return rc;
    // a step that raised its column's residual (an inner solve that drifted
    // off the true residual) is taken back and counts as a stall
    bool back = false;
    for (int q = 0; q < nrhs; ++q) {
      flag[q] = 0.0;
      if (!(rv2[q] <= rv2_old[q])) {
        flag[q] = -1.0;
        ++stall[q];
        taken[q] = 1;
        back = true;
      }
    }
    if (back) {
      if (trace) std::fprintf(stderr, "[cpm ir] steps taken back after refinement %d\n", nrep);
      CPM_CUDA_TRY(cudaMemcpyAsync(w->cols, flag.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      ir_add_kernel<<<g, 256, 0, st>>>(N, nrhs, ld, w->cols, w->d32, x);
      cpm_count_launches(c, 1);
      rc = residual64(c, ap64, m, n, f, x, w, nrhs, ld, wrow, rn2, fn2, st, rhs_w, &rv2);
      if (rc) return rc;
    }
  }
  *iters = it_total;
  *nrepl_out = nrep;
  *restarts = nrs;
  return CPM_OK;
}

// FP64 BiCGSTAB passes from the current x: the recursively updated residual
// drifts from f - A x near the rounding level, so while the true residual is
// above tol the iteration restarts from the current x, as long as a pass still
// lowers the worst true residual by 10 %
cpm_status fp64_passes(cpm_ctx *c, ApplyFn<double> ap64, bool left, double dS, double m, double n, const double *f,
                       double *x, SolveWork *w, int nrhs, int64_t ld, double wrow, double tol, int maxit,
                       int check_every, int *iters, int *restarts, bool *broke, std::vector<double> &rn2,
                       std::vector<double> &fn2, std::vector<double> &floors, cudaStream_t st) {
  const int64_t N = c->NS + c->NC;
  Vecs<double> V{w->v64[0], w->v64[1], w->v64[2], w->v64[3], w->v64[4], w->v64[5]};
  const Op<double> op = left ? Op<double>{ap64, m, n, dS, 1.0} : Op<double>{ap64, m, n, 1.0, dS};
  Conv cv{tol, 4000.0, 0.0f, 0, 0u};  // classical rhat = r (restarted on a first-step breakdown)
  double prev_worst = INFINITY;
  for (int pass = 0; pass < 8; ++pass) {
    const double *rhs = f;
    if (left) {
      // W f into the t slot, which the initial residual reads before t is written
      scale_rows64_kernel<<<cpm_grid(N * nrhs, 256), 256, 0, st>>>(N, c->NS, nrhs, ld, dS, f, V.t);
      cpm_count_launches(c, 1);
      rhs = V.t;
    }
    int it = 0, rs = 0;
    cpm_status rc = bicgstab<double, double>(c, op, rhs, x, false, V, w, nrhs, ld, cv, maxit - *iters, check_every,
                                             &it, &rs, broke, st);
    if (rc) return rc;
    *iters += it;
    *restarts += rs;
    rc = residual64(c, ap64, m, n, f, x, w, nrhs, ld, wrow, rn2, fn2, st);
    if (rc) return rc;
    const double worst = worst_relres(rn2, fn2);
    if (worst > tol) {
      // t and s are free between passes
      rc = floor64(c, ap64, m, n, x, V.t, V.s, w, nrhs, ld, wrow, fn2, floors, st);
      if (rc) return rc;
    }
    bool all = true;
    double fmin = INFINITY;
    for (int q = 0; q < nrhs; ++q) {
      const bool d = done_col(rn2[q], fn2[q], tol, floors[q]);
      all = all && d;
      if (!d) fmin = std::min(fmin, floors[q]);
    }
    // a further pass while the last one still gained 10 %; its recursion need
    // not go below the rounding floor, where the true residual cannot follow
    // a breakdown ends the pass, not the solve: the next pass restarts from x
    if (all || *iters >= maxit || !(worst < 0.9 * prev_worst)) break;
    if (std::isfinite(fmin)) cv.tol = std::max(tol, 0.5 * fmin);
    prev_worst = worst;
  }
  return CPM_OK;
}

cpm_status solve_impl(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                      int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t st) {
  cpm_solve_opts opts{1e-10, 10000, CPM_SOLVE_FP64, 1e-1, 200, 16, CPM_NORM_PLAIN, 1000};
  if (o) opts = *o;
  if (opts.tol <= 0) opts.tol = 1e-10;
  if (opts.maxit <= 0) opts.maxit = 10000;
  if (opts.inner_tol <= 0 || opts.inner_tol >= 1) opts.inner_tol = 1e-1;
  if (opts.max_refine <= 0) opts.max_refine = 200;
  if (opts.check_every <= 0) opts.check_every = 16;
  if (opts.inner_maxit <= 0) opts.inner_maxit = 1000;
  if (opts.norm != CPM_NORM_SCALED) opts.norm = CPM_NORM_PLAIN;
  const bool scaled = (opts.norm == CPM_NORM_SCALED);
  const bool trace = std::getenv("CPM_SOLVE_TRACE") != nullptr;
  SolveWork *w = c->solve;
  const int64_t N = c->NS + c->NC;
  if (!w || w->N != N || ld > w->ld) return CPM_ERR_CAPACITY;
  if (opts.mode == CPM_SOLVE_FP32_IR && !w->has32) return CPM_ERR_CAPACITY;
  // Jacobi value of the PDE rows: 1/(m + n diag L) (Sec. 5.4)
  const double dS = 1.0 / (m + n * (-2.0 * c->dim / (c->h * c->h)));
  // residual weight of the PDE rows; the adjoint (iterated right-preconditioned,
  // see below) is measured on its unscaled residual, the iteration's own
  const double wrow = (scaled && !adjoint) ? dS : 1.0;
  cpm_status rc;
  int iters = 0, restarts = 0, refinements = 0, iters64 = 0;
  bool broke = false;
  std::vector<double> rn2, fn2, floors(nrhs, 0.0);
  ApplyFn<double> ap64 = adjoint ? cpm_apply_transpose_rc_T<double> : cpm_apply_rc_T<double>;
  // scaled: BiCGSTAB on (W A) x = W f, so its recursive residual is the
  // measured one; plain: the paper's right-preconditioned form.  The adjoint
  // always iterates right-preconditioned, A^T W mu = g with lambda = W mu: this
  // is the transpose of the row-scaled forward system, whereas scaling the rows
  // of A^T leaves the BC rows with O(1/h^2) couplings and BiCGSTAB breaks down.
  const bool left = scaled && !adjoint;
  CPM_CUDA_TRY(cudaMemsetAsync(w->ticket, 0, sizeof(unsigned), st));
  w->G = c->nsm * ((c->tune.vec_blocks_per_sm >= 1 && c->tune.vec_blocks_per_sm <= 4) ? c->tune.vec_blocks_per_sm : 2);
  // the initial residual: a right-hand side (or guess) that is not finite is
  // rejected before any iteration
  rc = residual64(c, ap64, m, n, f, x, w, nrhs, ld, wrow, rn2, fn2, st);
  if (rc) return rc;
  for (int q = 0; q < nrhs; ++q)
    if (!std::isfinite(fn2[q]) || !std::isfinite(rn2[q])) {
      if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->relres = NAN;
        stats->status = CPM_ERR_ARG;
      }
      return CPM_ERR_ARG;
    }
  if (opts.mode == CPM_SOLVE_FP64) {
    rc = fp64_passes(c, ap64, left, dS, m, n, f, x, w, nrhs, ld, wrow, opts.tol, opts.maxit, opts.check_every, &iters,
                     &restarts, &broke, rn2, fn2, floors, st);
    if (rc) return rc;
    iters64 = iters;
  } else if (opts.mode == CPM_SOLVE_FP32_IR) {
    ApplyFn<float> ap32 = adjoint ? cpm_apply_transpose_rc_T<float> : cpm_apply_rc_T<float>;
    // the FP32 iteration runs on the row-scaled system (its residual is
    // balanced), the adjoint right-preconditioned; the requested norm decides
    // acceptance and convergence
    const Op<float> op32 = adjoint ? Op<float>{ap32, m, n, 1.0, dS} : Op<float>{ap32, m, n, dS, 1.0};
    rc = ir_refine(c, ap64, op32, m, n, f, x, w, nrhs, ld, wrow, adjoint ? 1.0 : dS, opts.tol, opts.inner_tol,
                     opts.maxit, opts.max_refine, opts.check_every, trace, &iters, &refinements, &restarts, rn2, fn2,
                     floors, st);
    if (rc) return rc;
    bool all = true;
    for (int q = 0; q < nrhs; ++q) all = all && done_col(rn2[q], fn2[q], opts.tol, floors[q]);
    if (!all && iters < opts.maxit) {
      // FP64 finish from the current iterate for the columns the FP32 phase
      // left above tol
      if (trace) std::fprintf(stderr, "[cpm] FP64 finish from relres %.3e\n", worst_relres(rn2, fn2));
      int it64 = 0;
      rc = fp64_passes(c, ap64, left, dS, m, n, f, x, w, nrhs, ld, wrow, opts.tol, opts.maxit - iters,
                       opts.check_every, &it64, &restarts, &broke, rn2, fn2, floors, st);
      if (rc) return rc;
      iters += it64;
      iters64 += it64;
    }
  } else {
    return CPM_ERR_ARG;
  }
  double relres = worst_relres(rn2, fn2), floor_max = 0.0;
  bool conv = true;
  for (int q = 0; q < nrhs; ++q) {
    conv = conv && done_col(rn2[q], fn2[q], opts.tol, floors[q]);
    floor_max = std::max(floor_max, floors[q]);
  }
  cpm_status out = CPM_OK;
  if (!conv) out = broke ? CPM_ERR_BREAKDOWN : CPM_ERR_NOT_CONVERGED;
  // a bounded wait of the fused single right-hand side product that gave up
  // (its device flag; set-up leaves the flags clear) voids the products
  unsigned herr = 0;
  CPM_CUDA_TRY(cudaMemcpyAsync(&herr, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr & CPM_DEVERR_WAIT) {
    CPM_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), st));
    out = CPM_ERR_TIMEOUT;
  }
  if (stats) {
    stats->iterations = iters;
    stats->refinements = refinements;
    stats->restarts = restarts;
    stats->relres = relres;
    stats->status = out;
    stats->fp64_iterations = iters64;
    stats->relres_floor = floor_max;
  }
  return out;
}

}  // namespace

cpm_status cpm_internal_solve(cpm_ctx *c, bool adjoint, double m, double n, const double *f, double *x, int nrhs,
                              int64_t ld, const cpm_solve_opts *o, cpm_solve_stats *stats, cudaStream_t caller) {
  // run on the internal stream, ordered after the caller's prior work and
  // before its later work
  cudaStream_t st = c->istream ? c->istream : caller;
  if (st != caller) {
    CPM_CUDA_TRY(cudaEventRecord(c->ev_join[0], caller));
    CPM_CUDA_TRY(cudaStreamWaitEvent(st, c->ev_join[0], 0));
  }
  cpm_status rc = solve_impl(c, adjoint, m, n, f, x, nrhs, ld, o, stats, st);
  if (st != caller) {
    cudaError_t e1 = cudaEventRecord(c->ev_join[1], st);
    cudaError_t e2 = cudaStreamWaitEvent(caller, c->ev_join[1], 0);
    if (rc == CPM_OK && (e1 != cudaSuccess || e2 != cudaSuccess)) rc = cpm_internal_cuda_err(e1 ? e1 : e2);
  }
  return rc;
}

// Timing of the Krylov vector kernels for the autotuner: `reps` launches of the
// two-product dot kernel over the workspace's first two vectors of precision
// prec with G blocks (no scalar state is touched).  Returns milliseconds per
// launch.
cpm_status cpm_time_vector_kernels(cpm_ctx *c, int prec, int nrhs, int64_t ld, int G, int reps, cudaStream_t st,
                                   double *ms) {
  SolveWork *w = c->solve;
  if (!w || ld > w->ld || (prec == CPM_PREC_FP32 && !w->has32) || G < 1 || G > 4 * c->nsm) return CPM_ERR_CAPACITY;
  const int64_t N = c->NS + c->NC;
  Red R = red_of(w, nrhs);
  const Conv cv{0.0, 0.0, 0.0f, 0, 0u};
  cudaEvent_t e0, e1;
  CPM_CUDA_TRY(cudaEventCreate(&e0));
  CPM_CUDA_TRY(cudaEventCreate(&e1));
  CPM_CUDA_TRY(cudaMemsetAsync(w->ticket, 0, sizeof(unsigned), st));
  auto launch = [&]() {
    if (prec == CPM_PREC_FP32)
      dot_kernel<float, 2><<<(unsigned)G, KT, 0, st>>>(R, cv, ST_OUT, N, ld, w->v32[0], w->v32[1]);
    else
      dot_kernel<double, 2><<<(unsigned)G, KT, 0, st>>>(R, cv, ST_OUT, N, ld, w->v64[0], w->v64[1]);
  };
  R.sc = nullptr;  // the dot bodies then include every column
  launch();
  cudaEventRecord(e0, st);
  for (int k = 0; k < reps; ++k) launch();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cpm_internal_cuda_err(e);
  *ms = (double)t / reps;
  return CPM_OK;
}

cpm_status cpm_solve_buffers_of(cpm_ctx *c, int prec, cpm_solve_buffers *b) {
  SolveWork *w = c->solve;
  if (!w || (prec == CPM_PREC_FP32 && !w->has32)) return CPM_ERR_CAPACITY;
  if (prec == CPM_PREC_FP32) { b->u = w->v32[0]; b->v = w->v32[1]; }
  else { b->u = w->v64[0]; b->v = w->v64[1]; }
  return CPM_OK;
}

