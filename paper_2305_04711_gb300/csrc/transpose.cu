// transpose.cu -- v = R A^T u, the adjoint operator, as gathers (no atomics).
//
// With s = n / h^2 and d = m + n (-2 dim / h^2), a PDE row i of A reads
//   (A u)_i = d u_i + s sum_k a~_{c(i,k)},   a~_c = (E u)_c (c < N_S),  a~_alpha = u_alpha,
// where c(i,k) is the k-th FD neighbour of row i after the crossing-test flips
// (Eqs. 10-11) and (E u)_c = sum_e w_{c,e} u_{col(c,e)}; a BC row is
// (A u)_alpha = sum_e B_{alpha,e} u_{bcol(alpha,e)} (Sec. 4.3).  The transpose is
//   b_c   = s sum_{i : c(i,k) = c} lambda_i                      (PDE DOFs c)
//   y_j   = d lambda_j + sum_{c, e : col(c,e) = j} w_{c,e} b_c
//           + s sum_{i : c(i,k) = j >= N_S} lambda_i + sum_{alpha, e : bcol = j} B lambda_alpha.
// Kernel 1 forms b from the geometric FD neighbours of c, keeping those whose
// own neighbour slot pointing back at c was not flipped.  Kernel 2 gathers E^T b
// at each node from the (up to 4^dim) stencil cells whose node set contains it,
// with every row of those cells (the cell buckets of cells.cu), and adds the
// sparse remainder -- flipped FD entries, flipped E entries (moved from node j to
// its twin) and BC-row entries -- from a per-column list built at set-up.
#include <algorithm>

#include "apply.cuh"
#include "cpm_internal.cuh"
#include "util.cuh"

namespace {

// packed location (brick << 9 | local) of a node given relative to brick b
// (offsets within one brick step); -1 when that brick is not in the band
__device__ __forceinline__ int64_t loc_of(const BandView &v, int32_t b, int lx, int ly, int lz) {
  const int dx = lx >> 3, dy = ly >> 3, dz = lz >> 3;
  if (dx | dy | dz) {
    b = __ldg(v.bnbr + (int64_t)b * 27 + 13 + dx + 3 * dy + 9 * dz);
    if (b < 0) return -1;
  }
  return ((int64_t)b << 9) | (int64_t)((lz & 7) * 64 + (ly & 7) * 8 + (lx & 7));
}

// per PDE row its 1-D Lagrange factors along each axis ([NS][12]: x, y, z,
// 4 slots each, zeros past the np1 stencil nodes)
__global__ void w1d_kernel(int64_t NS, int dim, int np1, const double *t64, double *w64, float *w32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NS; i += (int64_t)gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      double w[4] = {1.0, 0.0, 0.0, 0.0};
      if (a < dim) cpm_lagrange_rt<double>(np1, t64[3 * i + a], w);
      for (int k = 0; k < 4; ++k) {
        w64[i * 12 + 4 * a + k] = w[k];
        w32[i * 12 + 4 * a + k] = (float)w[k];
      }
    }
  }
}

__global__ void cellid_kernel(const uint32_t *cell_key, int64_t ncells, int32_t *cellid) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ncells; k += (int64_t)gridDim.x * blockDim.x)
    cellid[cell_key[k]] = (int32_t)k;
}

// ---- the sparse remainder, one list per column -------------------------------
// entry kinds: 0 flipped FD entry (y_target += s lambda_src), 1 flipped E entry
// (y_target += val b_src), 2 BC-row entry (y_target += val lambda_src)
struct TEntrySrc {
  const int32_t *spec_row; const int32_t *fcol; int64_t nspec;
  const int32_t *corr_row; const int32_t *corr_start; const int32_t *corr_node; const int32_t *corr_col;
  const double *corr_w; int64_t ncorr;
  const int32_t *bc_cnt; const int32_t *bc_col; const double *bc_val;
  int64_t NS, NC;
};

// pass 0 counts entries per target; pass 1 writes them at cursor positions
__global__ void tlist_kernel(TEntrySrc S, int pass, int32_t *count, int32_t *cursor, int32_t *t_src, int32_t *t_kind,
                             double *t_val) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  auto put = [&](int32_t target, int kind, int32_t src, double val) {
    if (pass == 0) {
      atomicAdd(count + target, 1);
    } else {
      int32_t p = atomicAdd(cursor + target, 1);
      t_src[p] = src;
      t_kind[p] = kind;
      t_val[p] = val;
    }
  };
  for (int64_t s = tid0; s < S.nspec; s += stride) {
    const int32_t i = S.spec_row[s];
    for (int k = 0; k < 6; ++k) {
      const int32_t cc = S.fcol[s * 6 + k];
      if (cc >= S.NS) put(cc, 0, i, 1.0);
    }
  }
  for (int64_t q = tid0; q < S.ncorr; q += stride) {
    const int32_t r = S.corr_row[q];
    for (int32_t e = S.corr_start[q]; e < S.corr_start[q + 1]; ++e) {
      put(S.corr_col[e], 1, r, S.corr_w[e]);
      put(S.corr_node[e], 1, r, -S.corr_w[e]);
    }
  }
  for (int64_t a = tid0; a < S.NC; a += stride) {
    const int64_t o = a * CPM_BC_STRIDE;
    for (int e = 0; e < S.bc_cnt[a]; ++e) put(S.bc_col[o + e], 2, (int32_t)(S.NS + a), S.bc_val[o + e]);
  }
}

// deterministic order inside each column list: by (kind, source)
__global__ void tlist_sort_kernel(const int32_t *ptr, int64_t N, int32_t *t_src, int32_t *t_kind, double *t_val,
                                  float *t_val32) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = ptr[j], e1 = ptr[j + 1];
    for (int32_t a = o + 1; a < e1; ++a) {
      const int32_t s = t_src[a], k = t_kind[a];
      const double v = t_val[a];
      const int64_t key = ((int64_t)k << 32) | (uint32_t)s;
      int32_t b = a - 1;
      while (b >= o && (((int64_t)t_kind[b] << 32) | (uint32_t)t_src[b]) > key) {
        t_src[b + 1] = t_src[b]; t_kind[b + 1] = t_kind[b]; t_val[b + 1] = t_val[b];
        --b;
      }
      t_src[b + 1] = s; t_kind[b + 1] = k; t_val[b + 1] = v;
    }
    for (int32_t a = o; a < e1; ++a) t_val32[a] = (float)t_val[a];
  }
}

template <typename T>
struct TArgs {
  BandView v;
  const uint32_t *rself;
  const T *w1d;  // [NS][12] per-axis Lagrange factors
  const int32_t *nbr8;
  const int32_t *cellid;
  const int32_t *cell_start;
  const int32_t *cell_rows;
  const int32_t *T_ptr;
  const int32_t *T_src;
  const int32_t *T_kind;
  const T *T_val;
  T *tblk;  // [ncells][64] per-cell blocks (one right-hand side), or nullptr
};

// b_c = s * sum of lambda over the rows whose unflipped FD slot points at c
// (cs: right diagonal factor on the PDE entries of lambda, as in the forward
// product: the kernels then apply A^T C)
template <typename T>
__global__ void __launch_bounds__(256) tb_kernel(TArgs<T> A, T s, const T *__restrict__ lam, T *__restrict__ bv,
                                                 int nrhs, int64_t ld) {
  const int nfd = 2 * A.v.dim;
  CPM_ROWS_COLS_LOOP(A.v.NS, nrhs, c, r) {
    const uint32_t rs = __ldg(A.rself + c);
    const int32_t b = (int32_t)(rs >> 9);
    const int l = (int)(rs & 511u);
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    T acc = T(0);
    for (int d = 0; d < nfd; ++d) {
      const int ax = d >> 1, sg = (d & 1) ? 1 : -1;
      const int32_t i = cpm_node_index(A.v, b, lx + (ax == 0 ? sg : 0), ly + (ax == 1 ? sg : 0),
                                       lz + (ax == 2 ? sg : 0));
      if (i < 0) continue;
      // row i's slot in the opposite direction points back at c unless flipped
      if (__ldg(A.nbr8 + (int64_t)i * 8 + (d ^ 1)) == (int32_t)c) acc += __ldg(lam + (int64_t)i * ld + r);
    }
    bv[c * ld + r] = s * acc;
  }
}

// One right-hand side: per stencil cell the block of its E^T b contributions,
// blk[cz*16 + cy*4 + cx] = sum over the cell's rows of w_x[cx] w_y[cy] w_z[cz] b_row,
// one thread per cell (the cell's rows share the 4x4x4 node set); the node
// gather below then reads one value per cell containing the node instead of
// revisiting every row of it.
template <typename T, int NP, int NZ>
__global__ void __launch_bounds__(128) tcell_kernel(TArgs<T> A, int64_t ncells, const T *__restrict__ bv) {
  for (int64_t cid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cid < ncells;
       cid += (int64_t)gridDim.x * blockDim.x) {
    T blk[NZ][NP][NP];
#pragma unroll
    for (int cz = 0; cz < NZ; ++cz)
#pragma unroll
      for (int cy = 0; cy < NP; ++cy)
#pragma unroll
        for (int cx = 0; cx < NP; ++cx) blk[cz][cy][cx] = T(0);
    const int32_t q1 = __ldg(A.cell_start + cid + 1);
    for (int32_t q = __ldg(A.cell_start + cid); q < q1; ++q) {
      const int64_t row = __ldg(A.cell_rows + q);
      const T *wr = A.w1d + row * 12;
      const T bb = __ldg(bv + row);
      T wx[NP], wy[NP], wz[NZ];
#pragma unroll
      for (int k = 0; k < NP; ++k) { wx[k] = __ldg(wr + k); wy[k] = __ldg(wr + 4 + k); }
#pragma unroll
      for (int k = 0; k < NZ; ++k) wz[k] = __ldg(wr + 8 + k);
#pragma unroll
      for (int cz = 0; cz < NZ; ++cz)
#pragma unroll
        for (int cy = 0; cy < NP; ++cy)
#pragma unroll
          for (int cx = 0; cx < NP; ++cx) blk[cz][cy][cx] += ((wx[cx] * wy[cy]) * wz[cz]) * bb;
    }
    T *out = A.tblk + cid * 64;
#pragma unroll
    for (int cz = 0; cz < NZ; ++cz)
#pragma unroll
      for (int cy = 0; cy < NP; ++cy)
#pragma unroll
        for (int cx = 0; cx < NP; ++cx) out[cz * 16 + cy * 4 + cx] = blk[cz][cy][cx];
  }
}

// y = R (d lambda_S + E^T b + remainder)
template <typename T>
__global__ void __launch_bounds__(256) ty_kernel(TArgs<T> A, T dg, T s, T rowscale, T cs, const T *__restrict__ lam,
                                                 const T *__restrict__ bv, T *__restrict__ y, int nrhs, int64_t ld) {
  const int64_t NS = A.v.NS, N = NS + A.v.NC;
  const int np1 = A.v.np1, nz = (A.v.dim == 3) ? np1 : 1;
  CPM_ROWS_COLS_LOOP(N, nrhs, j, r) {
    T acc = T(0);
    if (j < NS) {
      acc = (dg * cs) * __ldg(lam + j * ld + r);
      const uint32_t rs = __ldg(A.rself + j);
      const int32_t b = (int32_t)(rs >> 9);
      const int l = (int)(rs & 511u);
      const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
      for (int cz = 0; cz < nz; ++cz)
        for (int cy = 0; cy < np1; ++cy)
          for (int cx = 0; cx < np1; ++cx) {
            const int64_t key = loc_of(A.v, b, lx - cx, ly - cy, lz - cz);
            if (key < 0) continue;
            const int32_t cell = __ldg(A.cellid + key);
            if (cell < 0) continue;
            if (A.tblk) {
              // one right-hand side: the cell's block holds its rows' sum
              acc += A.tblk[(int64_t)cell * 64 + cz * 16 + cy * 4 + cx];
              continue;
            }
            const int32_t q1 = __ldg(A.cell_start + cell + 1);
            for (int32_t q = __ldg(A.cell_start + cell); q < q1; ++q) {
              const int64_t row = __ldg(A.cell_rows + q);
              const T *wr = A.w1d + row * 12;
              const T w = __ldg(wr + cx) * __ldg(wr + 4 + cy) * __ldg(wr + 8 + cz);
              acc += w * __ldg(bv + row * ld + r);
            }
          }
    }
    const int32_t e1 = __ldg(A.T_ptr + j + 1);
    for (int32_t e = __ldg(A.T_ptr + j); e < e1; ++e) {
      const int64_t src = __ldg(A.T_src + e);
      const int kind = __ldg(A.T_kind + e);
      if (kind == 0) acc += (s * cs) * __ldg(lam + src * ld + r);
      else if (kind == 1) acc += __ldg(A.T_val + e) * __ldg(bv + src * ld + r);
      else acc += __ldg(A.T_val + e) * __ldg(lam + src * ld + r);
    }
    y[j * ld + r] = (j < NS) ? rowscale * acc : acc;
  }
}

}  // namespace

cpm_status cpm_build_transpose(cpm_ctx *c) {
  cudaStream_t st = c->stream;
  cudaFree(c->d_T_ptr); cudaFree(c->d_T_row); cudaFree(c->d_T_kind); cudaFree(c->d_T_val); cudaFree(c->d_T_val32);
  cudaFree(c->d_cellid); cudaFree(c->d_w1d64); cudaFree(c->d_w1d32); cudaFree(c->d_tblk);
  c->d_w1d64 = nullptr; c->d_w1d32 = nullptr; c->d_tblk = nullptr;
  c->d_T_ptr = nullptr; c->d_T_row = nullptr; c->d_T_kind = nullptr; c->d_T_val = nullptr; c->d_T_val32 = nullptr;
  c->d_cellid = nullptr;
  c->transpose_ready = false;
  const int64_t N = c->NS + c->NC;
  const int64_t nkeys = c->nb * 512;
  int32_t *count = nullptr, *cursor = nullptr, *d_tot = nullptr;
  int32_t h_tot = 0;
  cpm_status rc = CPM_OK;
  TEntrySrc S{c->d_spec_row, c->d_spec_fcol, c->nspec, c->d_corr_row, c->d_corr_start, c->d_corr_node, c->d_corr_col,
              c->d_corr_w64, c->ncorr, c->d_bc_cnt, c->d_bc_col, c->d_bc_val, c->NS, c->NC};
  const unsigned gl = cpm_grid(std::max<int64_t>(std::max<int64_t>(c->nspec, c->ncorr), c->NC), 128);
#define TRY(x)                                             \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_) { rc = cpm_internal_cuda_err(e_); goto done; } \
  } while (0)
  TRY(cudaMalloc(&c->d_cellid, sizeof(int32_t) * std::max<int64_t>(nkeys, 1)));
  TRY(cudaMalloc(&c->d_tblk, sizeof(double) * 64 * std::max<int64_t>(c->ncells, 1)));
  TRY(cudaMemsetAsync(c->d_cellid, 0xFF, sizeof(int32_t) * std::max<int64_t>(nkeys, 1), st));
  TRY(cudaMalloc(&c->d_w1d64, sizeof(double) * 12 * std::max<int64_t>(c->NS, 1)));
  TRY(cudaMalloc(&c->d_w1d32, sizeof(float) * 12 * std::max<int64_t>(c->NS, 1)));
  w1d_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(c->NS, c->dim, c->p + 1, c->d_t64, c->d_w1d64, c->d_w1d32);
  if (c->ncells > 0)
    cellid_kernel<<<cpm_grid(c->ncells, 256), 256, 0, st>>>(c->d_cell_key, c->ncells, c->d_cellid);
  TRY(cudaMalloc(&count, sizeof(int32_t) * (N + 1)));
  TRY(cudaMalloc(&cursor, sizeof(int32_t) * (N + 1)));
  TRY(cudaMalloc(&d_tot, sizeof(int32_t)));
  TRY(cudaMalloc(&c->d_T_ptr, sizeof(int32_t) * (N + 1)));
  TRY(cudaMemsetAsync(count, 0, sizeof(int32_t) * (N + 1), st));
  tlist_kernel<<<gl, 128, 0, st>>>(S, 0, count, nullptr, nullptr, nullptr, nullptr);
  TRY(cpm_exclusive_scan(count, c->d_T_ptr, N + 1, d_tot, st));
  TRY(cudaMemcpyAsync(&h_tot, d_tot, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  c->nT = h_tot;
  TRY(cudaMalloc(&c->d_T_row, sizeof(int32_t) * std::max<int64_t>(c->nT, 1)));
  TRY(cudaMalloc(&c->d_T_kind, sizeof(int32_t) * std::max<int64_t>(c->nT, 1)));
  TRY(cudaMalloc(&c->d_T_val, sizeof(double) * std::max<int64_t>(c->nT, 1)));
  TRY(cudaMalloc(&c->d_T_val32, sizeof(float) * std::max<int64_t>(c->nT, 1)));
  TRY(cudaMemcpyAsync(cursor, c->d_T_ptr, sizeof(int32_t) * (N + 1), cudaMemcpyDeviceToDevice, st));
  if (c->nT > 0) {
    tlist_kernel<<<gl, 128, 0, st>>>(S, 1, nullptr, cursor, c->d_T_row, c->d_T_kind, c->d_T_val);
    tlist_sort_kernel<<<cpm_grid(N, 128), 128, 0, st>>>(c->d_T_ptr, N, c->d_T_row, c->d_T_kind, c->d_T_val,
                                                       c->d_T_val32);
  }
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(st));
  c->transpose_ready = true;
done:
#undef TRY
  cudaFree(count); cudaFree(cursor); cudaFree(d_tot);
  return rc;
}

template <typename T>
cpm_status cpm_apply_transpose_rc_T(cpm_ctx *c, double m, double n, double rowscale, double colscale, const T *u,
                                    T *v, int nrhs, int64_t ld, cudaStream_t st) {
  if (!c->transpose_ready) return CPM_ERR_STATE;
  if (sizeof(T) * (size_t)c->NS * (size_t)ld > c->b_scratch.bytes) return CPM_ERR_CAPACITY;
  TArgs<T> A;
  A.v = c->view();
  A.rself = c->d_rself;
  A.nbr8 = c->d_nbr8;
  A.cellid = c->d_cellid;
  A.cell_start = c->d_cell_start;
  A.cell_rows = c->d_cell_rows;
  A.T_ptr = c->d_T_ptr;
  A.T_src = c->d_T_row;
  A.T_kind = c->d_T_kind;
  if constexpr (sizeof(T) == 8) {
    A.w1d = reinterpret_cast<const T *>(c->d_w1d64);
    A.T_val = reinterpret_cast<const T *>(c->d_T_val);
  } else {
    A.w1d = reinterpret_cast<const T *>(c->d_w1d32);
    A.T_val = reinterpret_cast<const T *>(c->d_T_val32);
  }
  T *bv = reinterpret_cast<T *>(c->b_scratch.p);
  const double inv_h2 = 1.0 / (c->h * c->h);
  const T s = T(n * inv_h2), dg = T(m + n * (-2.0 * c->dim * inv_h2));
  const int64_t N = c->NS + c->NC;
  // one right-hand side: per-cell blocks of E^T b (reserved at set-up)
  A.tblk = (nrhs == 1 && ld == 1 && c->d_tblk && c->ncells > 0) ? reinterpret_cast<T *>(c->d_tblk) : nullptr;
  cpm_prof_begin(c, st);
  tb_kernel<T><<<cpm_grid(c->NS * nrhs, 256), 256, 0, st>>>(A, T(s * T(colscale)), u, bv, nrhs, ld);
  int launched = 2;
  if (A.tblk) {
    const unsigned gc = cpm_grid(c->ncells, 128);
    if (c->dim == 3) {
      if (c->p == 2) tcell_kernel<T, 3, 3><<<gc, 128, 0, st>>>(A, c->ncells, bv);
      else tcell_kernel<T, 4, 4><<<gc, 128, 0, st>>>(A, c->ncells, bv);
    } else {
      if (c->p == 2) tcell_kernel<T, 3, 1><<<gc, 128, 0, st>>>(A, c->ncells, bv);
      else tcell_kernel<T, 4, 1><<<gc, 128, 0, st>>>(A, c->ncells, bv);
    }
    ++launched;
  }
  ty_kernel<T><<<cpm_grid(N * nrhs, 256), 256, 0, st>>>(A, dg, s, T(rowscale), T(colscale), u, bv, v, nrhs, ld);
  cpm_prof_end(c, st, c->NS * (int64_t)nrhs);
  cpm_count_launches(c, launched);
  CPM_CUDA_TRY(cudaGetLastError());
  return CPM_OK;
}
template cpm_status cpm_apply_transpose_rc_T<double>(cpm_ctx *, double, double, double, double, const double *,
                                                     double *, int, int64_t, cudaStream_t);
template cpm_status cpm_apply_transpose_rc_T<float>(cpm_ctx *, double, double, double, double, const float *,
                                                    float *, int, int64_t, cudaStream_t);

template <typename T>
cpm_status cpm_apply_transpose_T(cpm_ctx *c, double m, double n, const T *u, T *v, int nrhs, int64_t ld,
                                 cudaStream_t st) {
  return cpm_apply_transpose_rc_T<T>(c, m, n, 1.0, 1.0, u, v, nrhs, ld, st);
}
template cpm_status cpm_apply_transpose_T<double>(cpm_ctx *, double, double, const double *, double *, int, int64_t,
                                                  cudaStream_t);
template cpm_status cpm_apply_transpose_T<float>(cpm_ctx *, double, double, const float *, float *, int, int64_t,
                                                 cudaStream_t);
