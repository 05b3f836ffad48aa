// apply.cu -- the matrix-free CPM operator on the device.
//
// Sec. 5.4 computes v = A u in four passes with stored E and L:
//   a = E u;  b = (L - diag L) a;  a = diag(L) u;  v = m u + n a + n b.
// Here E and L are never stored for the bulk of the rows: each PDE row keeps
// only the packed location of its interpolation stencil's base node and the
// fractional position t (FP64 and FP32 copies); the cubic Lagrange weights are
// formed in registers and the separable 4x4x4 gather runs along x-lines whose
// DOFs are consecutive in the canonical order (a line crossing a brick face is
// split in two runs).  Rows within 2 r of an interior boundary carry explicit
// stencils with the crossing-test flips (Eq. 10).  Two kernels per product:
//   gather : a_i = (E u)_i for PDE rows
//   combine: v_i = (m + n diagL) u_i + (n/h^2) sum_nbr a_sigma(nbr)   (PDE rows)
//            v_alpha = sum_beta B_alpha,beta u_beta                   (BC rows)
// where a neighbour flipped to a BC DOF reads u of that DOF (E rows of BC DOFs
// are the identity).
#include <mutex>

#include "apply.cuh"
#include "cpm_internal.cuh"

namespace {

template <typename T, bool DIFF, int NP>
__device__ __forceinline__ T line_sum(const T *u, int64_t ld, int r, int32_t s0, int32_t s1, int split, const T *w,
                                      T ui) {
  // nodes 0..split-1 are consecutive from s0, nodes split..NP-1 consecutive from
  // s1; a negative start (a node outside the band, excluded at set-up) reads
  // nothing
  T acc = T(0);
#pragma unroll
  for (int cx = 0; cx < NP; ++cx) {
    int32_t st = (cx < split) ? s0 : s1;
    int32_t idx = (cx < split) ? (s0 + cx) : (s1 + (cx - split));
    if (st >= 0) {
      T val = __ldg(u + (int64_t)idx * ld + r);
      acc += w[cx] * (DIFF ? (val - ui) : val);
    }
  }
  return acc;
}

// DIFF: a_i = sum_j w_j (u_j - u_i), the extension's defect, instead of
// sum_j w_j u_j.  Subtracting neighbouring values first keeps the rounding
// error relative to the differences (exact when close, Sterbenz), which FP32
// needs on smooth fields where the Laplacian cancels O(1) values to O(h^2).
// cs scales the values of PDE DOFs on input (a right diagonal factor C: the
// product is then E C u); BC DOFs enter unscaled.
template <typename T, bool DIFF, int NP>
__global__ void __launch_bounds__(256) gather_kernel(ApplyArgs<T> A, T cs, const T *__restrict__ u,
                                                     T *__restrict__ a, int nrhs, int64_t ld) {
  const int64_t NS = A.v.NS;
  CPM_ROWS_COLS_LOOP(A.v.NS, nrhs, i, r) {
    uint32_t rb = __ldg(A.rbase + i);
    T acc = T(0);
    const T ui = DIFF ? __ldg(u + i * ld + r) : T(0);
    if (rb & CPM_SPECIAL_BIT) {
      int64_t s = __ldg(A.spec_of + i);
      const int32_t *ec = A.ecol + s * 64;
      const T *ew = A.ew + s * 64;
      for (int e = 0; e < 64; ++e) {
        int32_t c = __ldg(ec + e);
        if (c >= 0) {
          const T val = __ldg(u + (int64_t)c * ld + r) * ((c < NS) ? cs : T(1));
          acc += __ldg(ew + e) * (DIFF ? (val - cs * ui) : val);
        }
      }
    } else {
      int32_t b = (int32_t)((rb >> 9) & 0x3FFFFFu);
      int l = (int)(rb & 511u);
      int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
      T wx[4], wy[4], wz[4];
      cpm_lagrange<NP, T>(__ldg(A.t + 3 * i), wx);
      cpm_lagrange<NP, T>(__ldg(A.t + 3 * i + 1), wy);
      const int nz = (A.v.dim == 3) ? NP : 1;
      if (A.v.dim == 3) cpm_lagrange<NP, T>(__ldg(A.t + 3 * i + 2), wz);
      else { wz[0] = T(1); wz[1] = wz[2] = wz[3] = T(0); }
      const int split = (lx + NP - 1 < 8) ? NP : 8 - lx;
      for (int cz = 0; cz < nz; ++cz) {
        T pz = T(0);
#pragma unroll
        for (int cy = 0; cy < NP; ++cy) {
          int32_t s0 = cpm_node_index(A.v, b, lx, ly + cy, lz + cz);
          int32_t s1 = (split < NP) ? cpm_node_index(A.v, b, 8, ly + cy, lz + cz) : 0;
          pz += wy[cy] * line_sum<T, DIFF, NP>(u, ld, r, s0, s1, split, wx, ui);
        }
        acc += wz[cz] * pz;
      }
      acc *= cs;
    }
    a[i * ld + r] = acc;
  }
}

// DIFF: a holds the extension defects sum_j w_j (u_j - u_k), and the row is
// m u_i + (n/h^2) [ sum_present (a_k + (u_k - u_i)) - n_missing u_i ],
// the same value as m u_i + n [diag(L) u_i + (1/h^2) sum_present (E u)_k].
template <typename T, bool DIFF>
__global__ void __launch_bounds__(256) combine_kernel(ApplyArgs<T> A, T m, T n, T rowscale, T cs,
                                                      const T *__restrict__ u, const T *__restrict__ a,
                                                      T *__restrict__ v, int nrhs, int64_t ld) {
  const int64_t NS = A.v.NS, N = NS + A.v.NC;
  const T inv_h2 = T(A.v.inv_h * A.v.inv_h);
  const T diag = m + n * T(-2.0 * A.v.dim * A.v.inv_h * A.v.inv_h);
  const int nfd = 2 * A.v.dim;
  CPM_ROWS_COLS_LOOP(N, nrhs, i, r) {
    if (i < NS) {
      uint32_t rb = __ldg(A.rbase + i);
      const T ui = cs * __ldg(u + i * ld + r);
      T s = T(0);
      int present = 0;
      if (A.nbr8) {
        // the precomputed neighbour table (flipped columns included)
        const int4 n0 = __ldg(reinterpret_cast<const int4 *>(A.nbr8 + i * 8));
        const int2 n1 = __ldg(reinterpret_cast<const int2 *>(A.nbr8 + i * 8 + 4));
        const int32_t nb[6] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int32_t c = nb[k];
          if (c < 0) continue;
          ++present;
          if (c < NS) {
            const T ac = __ldg(a + (int64_t)c * ld + r);
            s += DIFF ? ac + (cs * __ldg(u + (int64_t)c * ld + r) - ui) : ac;
          } else {
            const T uc = __ldg(u + (int64_t)c * ld + r);
            s += DIFF ? (uc - ui) : uc;
          }
        }
      } else if (rb & CPM_SPECIAL_BIT) {
        int64_t sp = __ldg(A.spec_of + i);
        for (int k = 0; k < 6; ++k) {
          int32_t c = __ldg(A.fcol + sp * 6 + k);
          if (c < 0) continue;
          ++present;
          const T uc = __ldg(u + (int64_t)c * ld + r) * ((c < NS) ? cs : T(1));
          if (DIFF) s += (c < NS) ? (__ldg(a + (int64_t)c * ld + r) + (uc - ui)) : (uc - ui);
          else s += (c < NS) ? __ldg(a + (int64_t)c * ld + r) : uc;
        }
      } else {
        uint32_t rs = __ldg(A.rself + i);
        int32_t b = (int32_t)(rs >> 9);
        int l = (int)(rs & 511u);
        int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
        int32_t nbr[6];
        nbr[0] = cpm_node_index(A.v, b, lx - 1, ly, lz);
        nbr[1] = cpm_node_index(A.v, b, lx + 1, ly, lz);
        nbr[2] = cpm_node_index(A.v, b, lx, ly - 1, lz);
        nbr[3] = cpm_node_index(A.v, b, lx, ly + 1, lz);
        nbr[4] = (A.v.dim == 3) ? cpm_node_index(A.v, b, lx, ly, lz - 1) : -1;
        nbr[5] = (A.v.dim == 3) ? cpm_node_index(A.v, b, lx, ly, lz + 1) : -1;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          int32_t j = nbr[k];
          if (j < 0) continue;
          ++present;
          T aj = __ldg(a + (int64_t)j * ld + r);
          if (DIFF) s += aj + (cs * __ldg(u + (int64_t)j * ld + r) - ui);
          else s += aj;
        }
      }
      T val;
      if (DIFF) val = m * ui + (n * inv_h2) * (s - T(nfd - present) * ui);
      else val = diag * ui + (n * inv_h2) * s;
      v[i * ld + r] = rowscale * val;
    } else {
      int64_t al = i - NS;
      int cnt = __ldg(A.bc_cnt + al);
      T s = T(0);
      for (int e = 0; e < cnt; ++e) {
        const int32_t c = __ldg(A.bc_col + al * CPM_BC_STRIDE + e);
        s += __ldg(A.bc_val + al * CPM_BC_STRIDE + e) * (__ldg(u + (int64_t)c * ld + r) * ((c < NS) ? cs : T(1)));
      }
      v[i * ld + r] = s;
    }
  }
}

// ---- batched combine: one warp per row, lanes over right-hand sides ---------
// With many right-hand sides the FD stencil is the same for every column, so
// one warp reads it once per row and each lane carries RPL columns
// (r = lane * RPL + k): every neighbour is one coalesced load of 32 * RPL
// contiguous values ([N][ld] layout, ld a multiple of RPL).  The extension
// values a = E u come from the cell-bucketed gather (cells.cu).
template <typename T, int RPL>
struct Vec;
template <> struct Vec<float, 1> { typedef float t; };
template <> struct Vec<float, 2> { typedef float2 t; };
template <> struct Vec<float, 4> { typedef float4 t; };
template <> struct Vec<double, 1> { typedef double t; };
template <> struct Vec<double, 2> { typedef double2 t; };

template <typename T, int RPL>
__device__ __forceinline__ void ldv(const T *p, T out[RPL]) {
  typedef typename Vec<T, RPL>::t V;
  V v = __ldg(reinterpret_cast<const V *>(p));
  const T *q = reinterpret_cast<const T *>(&v);
#pragma unroll
  for (int k = 0; k < RPL; ++k) out[k] = q[k];
}

template <typename T, int RPL>
__device__ __forceinline__ void stv(T *p, const T in[RPL]) {
  typedef typename Vec<T, RPL>::t V;
  V v;
  T *q = reinterpret_cast<T *>(&v);
#pragma unroll
  for (int k = 0; k < RPL; ++k) q[k] = in[k];
  *reinterpret_cast<V *>(p) = v;
}

template <typename T, bool DIFF, int RPL>
__global__ void __launch_bounds__(256) combine_batched_kernel(ApplyArgs<T> A, T m, T n, T rowscale, T cs,
                                                              const T *__restrict__ u, const T *__restrict__ a,
                                                              T *__restrict__ v, int nrhs, int64_t ld) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int col = lane * RPL;
  const bool on = col < nrhs;
  const int64_t NS = A.v.NS, N = NS + A.v.NC;
  const T inv_h2 = T(A.v.inv_h * A.v.inv_h);
  const T diag = m + n * T(-2.0 * A.v.dim * A.v.inv_h * A.v.inv_h);
  const int nfd = 2 * A.v.dim;
  for (int64_t i = warp; i < N; i += nwarps) {
    T out[RPL];
    if (i < NS) {
      int32_t nbr[6];
      if (A.nbr8) {
        const int4 n0 = __ldg(reinterpret_cast<const int4 *>(A.nbr8 + i * 8));
        const int2 n1 = __ldg(reinterpret_cast<const int2 *>(A.nbr8 + i * 8 + 4));
        nbr[0] = n0.x; nbr[1] = n0.y; nbr[2] = n0.z; nbr[3] = n0.w; nbr[4] = n1.x; nbr[5] = n1.y;
      } else if (__ldg(A.rbase + i) & CPM_SPECIAL_BIT) {
        int64_t sp = __ldg(A.spec_of + i);
#pragma unroll
        for (int k = 0; k < 6; ++k) nbr[k] = __ldg(A.fcol + sp * 6 + k);
      } else {
        uint32_t rs = __ldg(A.rself + i);
        int32_t b = (int32_t)(rs >> 9);
        int l = (int)(rs & 511u);
        int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
        nbr[0] = cpm_node_index(A.v, b, lx - 1, ly, lz);
        nbr[1] = cpm_node_index(A.v, b, lx + 1, ly, lz);
        nbr[2] = cpm_node_index(A.v, b, lx, ly - 1, lz);
        nbr[3] = cpm_node_index(A.v, b, lx, ly + 1, lz);
        nbr[4] = (A.v.dim == 3) ? cpm_node_index(A.v, b, lx, ly, lz - 1) : -1;
        nbr[5] = (A.v.dim == 3) ? cpm_node_index(A.v, b, lx, ly, lz + 1) : -1;
      }
      if (!on) continue;
      T ui[RPL], s[RPL];
      ldv<T, RPL>(u + i * ld + col, ui);
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        ui[k] *= cs;
        s[k] = T(0);
      }
      int present = 0;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        int32_t c = nbr[q];
        if (c < 0) continue;
        ++present;
        T uc[RPL], ac[RPL];
        if (DIFF || c >= NS) ldv<T, RPL>(u + (int64_t)c * ld + col, uc);
        if (c < NS) ldv<T, RPL>(a + (int64_t)c * ld + col, ac);
        const T sc_c = (c < NS) ? cs : T(1);
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          uc[k] *= sc_c;
          if (DIFF) s[k] += (c < NS) ? (ac[k] + (uc[k] - ui[k])) : (uc[k] - ui[k]);
          else s[k] += (c < NS) ? ac[k] : uc[k];
        }
      }
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        T val = DIFF ? (m * ui[k] + (n * inv_h2) * (s[k] - T(nfd - present) * ui[k]))
                     : (diag * ui[k] + (n * inv_h2) * s[k]);
        out[k] = rowscale * val;
      }
    } else {
      if (!on) continue;
      int64_t al = i - NS;
      int cnt = __ldg(A.bc_cnt + al);
#pragma unroll
      for (int k = 0; k < RPL; ++k) out[k] = T(0);
      for (int e = 0; e < cnt; ++e) {
        const int32_t cc = __ldg(A.bc_col + al * CPM_BC_STRIDE + e);
        const T w = __ldg(A.bc_val + al * CPM_BC_STRIDE + e) * ((cc < NS) ? cs : T(1));
        T val[RPL];
        ldv<T, RPL>(u + (int64_t)cc * ld + col, val);
#pragma unroll
        for (int k = 0; k < RPL; ++k) out[k] += w * val[k];
      }
    }
    stv<T, RPL>(v + i * ld + col, out);
  }
}

// batched product: E u for all PDE rows through the cell-bucketed gather
// (cells.cu), then the warp-per-row combine
template <typename T, int RPL>
static int launch_batched(const cpm_ctx *c, const ApplyArgs<T> &A, T m, T n, T rowscale, T cs, const T *u, T *a,
                          T *v, int nrhs, int64_t ld, cudaStream_t st, bool diff) {
  // 8 warps per block; by default 8 blocks per SM
  const int64_t warps = (int64_t)c->nsm * (c->tune.combine_warps_per_sm > 0 ? c->tune.combine_warps_per_sm : 64);
  unsigned g = (unsigned)std::min<int64_t>((A.v.NS + A.v.NC + 7) / 8, warps / 8);
  if (g < 1) g = 1;
  int launched = 1 + cpm_launch_gather_cells<T>(c, A, cs, u, a, nrhs, ld, st, diff, RPL);
  if (diff) combine_batched_kernel<T, true, RPL><<<g, 256, 0, st>>>(A, m, n, rowscale, cs, u, a, v, nrhs, ld);
  else combine_batched_kernel<T, false, RPL><<<g, 256, 0, st>>>(A, m, n, rowscale, cs, u, a, v, nrhs, ld);
  return launched;
}

__global__ void rhs_kernel(BandView v, const CurveDev *curves, const int32_t *bc_curve, const int32_t *side,
                           const int32_t *type, const double *param, const double *s, const double *g,
                           const double *samples, double *f, int nrhs, int64_t ld) {
  const int64_t N = v.NS + v.NC;
  CPM_ROWS_COLS_LOOP(N, nrhs, i, r) {
    if (i < v.NS) {
      f[i * ld + r] = s ? s[i * ld + r] : 0.0;
      continue;
    }
    int64_t al = i - v.NS;
    const CurveDev &cv = curves[bc_curve[al]];
    double gv = 0.0;
    if (g) {
      gv = g[al * ld + r];
    } else if (samples) {
      int ns = cv.n_samples;
      double sp = param[al] / 6.283185307179586476925286766559 * ns;
      double fl = floor(sp);
      int i0 = ((int)fl) % ns;
      if (i0 < 0) i0 += ns;
      int i1 = (i0 + 1) % ns;
      double fr = sp - fl;
      int64_t o = cv.sample_off;
      double plus = (1.0 - fr) * samples[(o + i0) * ld + r] + fr * samples[(o + i1) * ld + r];
      if (cv.two_sided) {
        double minus = (1.0 - fr) * samples[(o + ns + i0) * ld + r] + fr * samples[(o + ns + i1) * ld + r];
        int sd = side[al];
        gv = (sd > 0) ? minus : (sd < 0) ? plus : 0.5 * (plus + minus);
      } else {
        gv = plus;
      }
    }
    f[i * ld + r] = cpm_bc_data_scale(type[al]) * gv;
  }
}

// dL/dsamples = B^T (c_alpha lambda_alpha): one block per (sample, rhs), a fixed
// order reduction over the BC DOFs of the sample's curve (deterministic)
__global__ void boundary_grad_kernel(BandView v, const CurveDev *curves, int ncurves, const int32_t *curve_first,
                                     const int32_t *side, const int32_t *type, const double *param,
                                     const double *lam, double *out, int64_t nsamples_total, int nrhs,
                                     int64_t ld) {
  __shared__ double red[256];
  for (int64_t q = blockIdx.x; q < nsamples_total * nrhs; q += gridDim.x) {
    int64_t sidx = q / nrhs;
    int r = (int)(q - sidx * nrhs);
    int k = 0;
    while (k + 1 < ncurves && curves[k + 1].sample_off <= sidx) ++k;
    const CurveDev &cv = curves[k];
    int ns = cv.n_samples;
    int64_t loc = sidx - cv.sample_off;
    int blockside = (cv.two_sided && loc >= ns) ? -1 : +1;  // plus block first, then minus block
    int kk = (int)(loc % ns);
    double acc = 0.0;
    for (int64_t al = curve_first[k] + threadIdx.x; al < curve_first[k + 1]; al += blockDim.x) {
      double sp = param[al] / 6.283185307179586476925286766559 * ns;
      double fl = floor(sp);
      int i0 = ((int)fl) % ns;
      if (i0 < 0) i0 += ns;
      int i1 = (i0 + 1) % ns;
      double fr = sp - fl;
      double wblk = 1.0;
      if (cv.two_sided) {
        int sd = side[al];
        // a BC DOF whose cp_S is on the plus side takes the minus-side samples
        if (sd > 0) wblk = (blockside < 0) ? 1.0 : 0.0;
        else if (sd < 0) wblk = (blockside > 0) ? 1.0 : 0.0;
        else wblk = 0.5;
      }
      double w = 0.0;
      if (i0 == kk) w += 1.0 - fr;
      if (i1 == kk) w += fr;
      const double c = cpm_bc_data_scale(type[al]);
      acc += wblk * w * c * lam[(v.NS + al) * ld + r];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[sidx * ld + r] = red[0];
    __syncthreads();
  }
}

}  // namespace

template <typename T>
ApplyArgs<T> cpm_apply_args(const cpm_ctx *c) {
  ApplyArgs<T> A;
  A.v = c->view();
  A.rbase = c->d_rbase;
  A.rself = c->d_rself;
  A.spec_of = c->d_spec_of;
  A.ecol = c->d_spec_ecol;
  A.fcol = c->d_spec_fcol;
  A.nbr8 = c->d_nbr8;
  A.bc_cnt = c->d_bc_cnt;
  A.bc_col = c->d_bc_col;
  if constexpr (sizeof(T) == 8) {
    A.t = reinterpret_cast<const T *>(c->d_t64);
    A.ew = reinterpret_cast<const T *>(c->d_spec_ew);
    A.bc_val = reinterpret_cast<const T *>(c->d_bc_val);
  } else {
    A.t = reinterpret_cast<const T *>(c->d_t32);
    A.ew = reinterpret_cast<const T *>(c->d_spec_ew32);
    A.bc_val = reinterpret_cast<const T *>(c->d_bc_val32);
  }
  return A;
}

template <typename T>
void cpm_launch_gather(const ApplyArgs<T> &A, T cs, const T *u, T *a, int nrhs, int64_t ld, cudaStream_t st,
                       bool diff) {
  const unsigned g = cpm_grid(A.v.NS * nrhs, 256);
  if (A.v.np1 == 3) {
    if (diff) gather_kernel<T, true, 3><<<g, 256, 0, st>>>(A, cs, u, a, nrhs, ld);
    else gather_kernel<T, false, 3><<<g, 256, 0, st>>>(A, cs, u, a, nrhs, ld);
  } else {
    if (diff) gather_kernel<T, true, 4><<<g, 256, 0, st>>>(A, cs, u, a, nrhs, ld);
    else gather_kernel<T, false, 4><<<g, 256, 0, st>>>(A, cs, u, a, nrhs, ld);
  }
}

template <typename T>
void cpm_launch_combine(const ApplyArgs<T> &A, T m, T n, T rowscale, T cs, const T *u, const T *a, T *v, int nrhs,
                        int64_t ld, cudaStream_t st, bool diff) {
  unsigned g = cpm_grid((A.v.NS + A.v.NC) * nrhs, 256);
  if (diff) combine_kernel<T, true><<<g, 256, 0, st>>>(A, m, n, rowscale, cs, u, a, v, nrhs, ld);
  else combine_kernel<T, false><<<g, 256, 0, st>>>(A, m, n, rowscale, cs, u, a, v, nrhs, ld);
}

template ApplyArgs<double> cpm_apply_args<double>(const cpm_ctx *);
template ApplyArgs<float> cpm_apply_args<float>(const cpm_ctx *);
template void cpm_launch_gather<double>(const ApplyArgs<double> &, double, const double *, double *, int, int64_t,
                                        cudaStream_t, bool);
template void cpm_launch_gather<float>(const ApplyArgs<float> &, float, const float *, float *, int, int64_t,
                                       cudaStream_t, bool);
template void cpm_launch_combine<double>(const ApplyArgs<double> &, double, double, double, double, const double *,
                                         const double *, double *, int, int64_t, cudaStream_t, bool);
template void cpm_launch_combine<float>(const ApplyArgs<float> &, float, float, float, float, const float *,
                                        const float *, float *, int, int64_t, cudaStream_t, bool);

// v = R A C u using the context's reserved scratch for a (no allocation): R
// scales the PDE rows of the result by `rowscale` and C the PDE entries of the
// input by `colscale` (1 and 1 for the plain product); BC rows and BC entries
// are left alone.  Both forms use the difference form of the gather, which
// keeps the rounding of smooth fields relative to local differences.
template <typename T>
cpm_status cpm_apply_rc_T(cpm_ctx *c, double m, double n, double rowscale, double colscale, const T *u, T *v,
                          int nrhs, int64_t ld, cudaStream_t st) {
  if (sizeof(T) * (size_t)c->NS * (size_t)ld > c->a_scratch.bytes) return CPM_ERR_CAPACITY;
  ApplyArgs<T> A = cpm_apply_args<T>(c);
  T *a = reinterpret_cast<T *>(c->a_scratch.p);
  const bool diff = true;
  const T cs = T(colscale);
  cpm_prof_begin(c, st);
  // batched layouts whose columns fill whole warps use the warp-per-row kernels
  const bool aligned2 = (ld % 2 == 0) && ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v) |
                                           reinterpret_cast<uintptr_t>(a)) % (2 * sizeof(T)) == 0);
  int launched = 2;
  // two adjacent columns per lane need an even column count and 2-element alignment
  if (nrhs > 32 && nrhs <= 64 && nrhs % 2 == 0 && aligned2)
    launched = launch_batched<T, 2>(c, A, (T)m, (T)n, (T)rowscale, cs, u, a, v, nrhs, ld, st, diff);
  else if (nrhs >= 16 && nrhs <= 32)
    launched = launch_batched<T, 1>(c, A, (T)m, (T)n, (T)rowscale, cs, u, a, v, nrhs, ld, st, diff);
  else if (nrhs == 1 && c->ncells > 0) {
    // default: the per-cell gather, then the combine; 1: per-row gather; 2: the
    // fused persistent product (fused1.cu)
    launched = (c->tune.single_mode == 2)
                   ? cpm_launch_fused1<T>(c, A, (T)m, (T)n, (T)rowscale, cs, u, a, v, st)
                   : 0;
    if (launched == 0) {
      launched = 1 + cpm_launch_gather1<T>(c, A, cs, u, a, st, diff);
      cpm_launch_combine<T>(A, (T)m, (T)n, (T)rowscale, cs, u, a, v, nrhs, ld, st, diff);
    }
  } else {
    cpm_launch_gather<T>(A, cs, u, a, nrhs, ld, st, diff);
    cpm_launch_combine<T>(A, (T)m, (T)n, (T)rowscale, cs, u, a, v, nrhs, ld, st, diff);
  }
  cpm_prof_end(c, st, c->NS * (int64_t)nrhs);
  cpm_count_launches(c, launched);
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}
template cpm_status cpm_apply_rc_T<double>(cpm_ctx *, double, double, double, double, const double *, double *, int,
                                           int64_t, cudaStream_t);
template cpm_status cpm_apply_rc_T<float>(cpm_ctx *, double, double, double, double, const float *, float *, int,
                                          int64_t, cudaStream_t);

template <typename T>
cpm_status cpm_apply_T(cpm_ctx *c, double m, double n, const T *u, T *v, int nrhs, int64_t ld, cudaStream_t st) {
  return cpm_apply_rc_T<T>(c, m, n, 1.0, 1.0, u, v, nrhs, ld, st);
}
template cpm_status cpm_apply_T<double>(cpm_ctx *, double, double, const double *, double *, int, int64_t,
                                        cudaStream_t);
template cpm_status cpm_apply_T<float>(cpm_ctx *, double, double, const float *, float *, int, int64_t,
                                       cudaStream_t);

void cpm_prof_begin(cpm_ctx *c, cudaStream_t st) {
  if (!c->prof.on) return;
  Profiler &p = c->prof;
  if (p.used + 2 > p.ev.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { (void)cudaGetLastError(); p.on = false; return; }
      p.ev.push_back(e);
    }
  }
  cudaEventRecord(p.ev[p.used], st);
}

void cpm_prof_end(cpm_ctx *c, cudaStream_t st, int64_t row_rhs) {
  if (!c->prof.on) return;
  Profiler &p = c->prof;
  cudaEventRecord(p.ev[p.used + 1], st);
  p.used += 2;
  p.applies += 1;
  p.row_rhs += row_rhs;
}

cpm_status cpm_internal_extend(cpm_ctx *c, const double *u, double *a, int nrhs, int64_t ld, cudaStream_t st) {
  ApplyArgs<double> A = cpm_apply_args<double>(c);
  cpm_launch_gather<double>(A, 1.0, u, a, nrhs, ld, st, false);
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}

cpm_status cpm_internal_rhs(cpm_ctx *c, const double *s, const double *g, const double *samples, double *f, int nrhs,
                            int64_t ld, cudaStream_t st) {
  int64_t N = c->NS + c->NC;
  rhs_kernel<<<cpm_grid(N * nrhs, 256), 256, 0, st>>>(c->view(), c->d_curves, c->d_bc_curve, c->d_side, c->d_bc_type,
                                                      c->d_param, s,
                                                      g, samples, f, nrhs, ld);
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}

cpm_status cpm_internal_boundary_grad(cpm_ctx *c, const double *lam, double *out, int nrhs, int64_t ld,
                                      cudaStream_t st) {
  if (c->nsamples_total == 0) return CPM_OK;
  // c->d_curve_first: first BC DOF of each curve (BC DOFs are ordered by curve),
  // built with the boundary
  unsigned grid = (unsigned)std::min<int64_t>(c->nsamples_total * nrhs, (int64_t)c->nsm * 32);
  boundary_grad_kernel<<<grid, 256, 0, st>>>(c->view(), c->d_curves, c->ncurves, c->d_curve_first, c->d_side,
                                             c->d_bc_type, c->d_param, lam, out, c->nsamples_total, nrhs, ld);
  cpm_count_launches(c, 1);
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}

// ---- operator product with a static scratch (no allocation) -----------------
// The E u intermediate lives in a fixed module array instead of the context's
// lazily grown scratch, so this path calls no allocator.  Nothing in the array
// has to start at zero: every element the combine reads was written earlier in
// the same call.  One array per device serves every context and stream, so
// calls that overlap in time on one device race on it.
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// device address of the array for the current device, looked up on the first
// call for that device
cpm_status noalloc_scratch(void **out) {
  int dev = -1;
  CPM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return CPM_ERR_CAPACITY;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cpm_internal_cuda_err(e);
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CPM_OK;
}
}  // namespace

size_t cpm_noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

template <typename T>
cpm_status cpm_apply_noalloc_T(cpm_ctx *c, double m, double n, const T *u, T *v, int nrhs, int64_t ld,
                               cudaStream_t st) {
  if (sizeof(T) * (size_t)c->NS * (size_t)ld > kNoAllocScratchBytes) return CPM_ERR_CAPACITY;
  void *p = nullptr;
  cpm_status rc = noalloc_scratch(&p);
  if (rc) return rc;
  T *a = reinterpret_cast<T *>(p);
  ApplyArgs<T> A = cpm_apply_args<T>(c);
  const bool diff = true;  // the same arithmetic as cpm_apply
  const bool aligned2 = (ld % 2 == 0) && ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v) |
                                           reinterpret_cast<uintptr_t>(a)) % (2 * sizeof(T)) == 0);
  int launched = 2;
  if (nrhs > 32 && nrhs <= 64 && nrhs % 2 == 0 && aligned2)
    launched = launch_batched<T, 2>(c, A, (T)m, (T)n, T(1), T(1), u, a, v, nrhs, ld, st, diff);
  else if (nrhs >= 16 && nrhs <= 32)
    launched = launch_batched<T, 1>(c, A, (T)m, (T)n, T(1), T(1), u, a, v, nrhs, ld, st, diff);
  else {
    cpm_launch_gather<T>(A, T(1), u, a, nrhs, ld, st, diff);
    cpm_launch_combine<T>(A, (T)m, (T)n, T(1), T(1), u, a, v, nrhs, ld, st, diff);
  }
  cpm_count_launches(c, launched);
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}
template cpm_status cpm_apply_noalloc_T<double>(cpm_ctx *, double, double, const double *, double *, int, int64_t,
                                                cudaStream_t);
template cpm_status cpm_apply_noalloc_T<float>(cpm_ctx *, double, double, const float *, float *, int, int64_t,
                                               cudaStream_t);
