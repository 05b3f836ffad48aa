// cells.cu -- rows bucketed by the base node ("cell") of their interpolation
// stencil, and the cell-bucketed batched gather.
//
// All rows whose closest points fall in the same grid cell share the same
// 4x4x4 stencil nodes (Eq. 1); only their weights differ.  On a narrow band
// about 2 r / h ~ 8 rows share each cell.  With many right-hand sides the gather
// is bound by moving node values (64 nodes x nrhs per row), so one warp takes a
// whole cell: it loads the 64 nodes once and applies the separable weights of
// up to 8 of the cell's rows at a time (weights staged in shared memory).
//
// The buckets are built by a counting sort over the dense (brick, local) key
// space, with each bucket then ordered by row index, so the result does not
// depend on the scheduling of the atomics.  Only bulk rows are bucketed; rows
// with explicit (flipped) stencils near interior boundaries keep their own path.
#include <algorithm>

#include "apply.cuh"
#include "cpm_internal.cuh"
#include "util.cuh"

namespace {

__global__ void cell_count_kernel(const uint32_t *rbase, int64_t NS, int32_t *count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NS; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rb = rbase[i];
    if (rb & CPM_SPECIAL_BIT) continue;
    atomicAdd(count + rb, 1);
  }
}

__global__ void cell_scatter_kernel(const uint32_t *rbase, int64_t NS, int32_t *cursor, int32_t *rows) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NS; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rb = rbase[i];
    if (rb & CPM_SPECIAL_BIT) continue;
    int32_t p = atomicAdd(cursor + rb, 1);
    rows[p] = (int32_t)i;
  }
}

// per non-empty key: its cell id, start, and a deterministic (row-index) order
__global__ void cell_finish_kernel(const int32_t *count, const int32_t *offs, const int32_t *cellpos, int64_t nkeys,
                                   int32_t *rows, int32_t *cell_start, uint32_t *cell_key) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nkeys; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t n = count[k];
    if (n == 0) continue;
    int32_t c = cellpos[k], o = offs[k];
    cell_start[c] = o;
    cell_key[c] = (uint32_t)k;
    // insertion sort of the bucket (a few to a few dozen rows)
    for (int32_t a = o + 1; a < o + n; ++a) {
      int32_t v = rows[a], b = a - 1;
      while (b >= o && rows[b] > v) { rows[b + 1] = rows[b]; --b; }
      rows[b + 1] = v;
    }
  }
}

__global__ void flag_nonzero_kernel(const int32_t *count, int64_t n, int32_t *flag) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    flag[k] = count[k] != 0;
}

constexpr int CHUNK = 8;   // rows of a cell processed together
constexpr int WARPS = 8;   // warps per block

template <typename T, int RPL>
struct VecT;
template <> struct VecT<float, 1> { typedef float t; };
template <> struct VecT<float, 2> { typedef float2 t; };
template <> struct VecT<double, 1> { typedef double t; };
template <> struct VecT<double, 2> { typedef double2 t; };

template <typename T, int RPL>
__device__ __forceinline__ void ld(const T *p, T out[RPL]) {
  typedef typename VecT<T, RPL>::t V;
  V v = __ldg(reinterpret_cast<const V *>(p));
  const T *q = reinterpret_cast<const T *>(&v);
#pragma unroll
  for (int k = 0; k < RPL; ++k) out[k] = q[k];
}

template <typename T, int RPL>
__device__ __forceinline__ void st(T *p, const T in[RPL]) {
  typedef typename VecT<T, RPL>::t V;
  V v;
  T *q = reinterpret_cast<T *>(&v);
#pragma unroll
  for (int k = 0; k < RPL; ++k) q[k] = in[k];
  *reinterpret_cast<V *>(p) = v;
}

// One warp per cell.  DIFF (the FP32 form): the node values enter as
// differences to the cell's base-node value u_c, and each row adds u_c - u_i:
// sum_n w_n (u_n - u_i) = sum_n w_n (u_n - u_c) + (u_c - u_i) since sum_n w_n = 1,
// which keeps FP32 rounding relative to local differences.
template <typename T, bool DIFF, int RPL>
__global__ void __launch_bounds__(WARPS * 32) gather_cells_kernel(ApplyArgs<T> A, const int32_t *__restrict__ cstart,
                                                                  const uint32_t *__restrict__ ckey,
                                                                  const int32_t *__restrict__ crows, int64_t ncells,
                                                                  const T *__restrict__ u, T *__restrict__ a, int nrhs,
                                                                  int64_t ld_) {
  __shared__ T s_wx[WARPS][CHUNK][4];
  __shared__ T s_wyz[WARPS][CHUNK][16];
  __shared__ int32_t s_row[WARPS][CHUNK];
  __shared__ int32_t s_line[WARPS][16][2];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int col = lane * RPL;
  const bool on = col < nrhs;
  const int nz = (A.v.dim == 3) ? 4 : 1;
  const int nlines = 4 * nz;
  for (int64_t cid = warp; cid < ncells; cid += nwarps) {
    const uint32_t key = __ldg(ckey + cid);
    const int32_t b = (int32_t)(key >> 9);
    const int l = (int)(key & 511u);
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    const int split = (lx + 3 < 8) ? 4 : 8 - lx;
    if (lane < nlines) {
      int cy = lane & 3, cz = lane >> 2;
      s_line[wib][lane][0] = cpm_node_index(A.v, b, lx, ly + cy, lz + cz);
      s_line[wib][lane][1] = (split < 4) ? cpm_node_index(A.v, b, 8, ly + cy, lz + cz) : 0;
    }
    __syncwarp();
    T uc[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) uc[k] = T(0);
    if (DIFF && on && s_line[wib][0][0] >= 0) ld<T, RPL>(u + (int64_t)s_line[wib][0][0] * ld_ + col, uc);
    const int32_t r0 = __ldg(cstart + cid), r1 = __ldg(cstart + cid + 1);
    for (int32_t cs = r0; cs < r1; cs += CHUNK) {
      const int k = min(CHUNK, r1 - cs);
      if (lane < k) {
        int32_t row = __ldg(crows + cs + lane);
        s_row[wib][lane] = row;
        T wx[4], wy[4], wz[4];
        cpm_lagrange4<T>(__ldg(A.t + 3 * (int64_t)row), wx);
        cpm_lagrange4<T>(__ldg(A.t + 3 * (int64_t)row + 1), wy);
        if (A.v.dim == 3) cpm_lagrange4<T>(__ldg(A.t + 3 * (int64_t)row + 2), wz);
        else { wz[0] = T(1); wz[1] = wz[2] = wz[3] = T(0); }
#pragma unroll
        for (int q = 0; q < 4; ++q) s_wx[wib][lane][q] = wx[q];
#pragma unroll
        for (int q = 0; q < 16; ++q) s_wyz[wib][lane][q] = wy[q & 3] * wz[q >> 2];
      }
      __syncwarp();
      T acc[CHUNK][RPL];
#pragma unroll
      for (int j = 0; j < CHUNK; ++j)
#pragma unroll
        for (int q = 0; q < RPL; ++q) acc[j][q] = T(0);
      if (on) {
        for (int ln = 0; ln < nlines; ++ln) {
          const int32_t s0 = s_line[wib][ln][0], s1 = s_line[wib][ln][1];
          T d[4][RPL];
#pragma unroll
          for (int cx = 0; cx < 4; ++cx) {
            int32_t stt = (cx < split) ? s0 : s1;
            int32_t idx = (cx < split) ? (s0 + cx) : (s1 + (cx - split));
            if (stt >= 0) {
              ld<T, RPL>(u + (int64_t)idx * ld_ + col, d[cx]);
#pragma unroll
              for (int q = 0; q < RPL; ++q) if (DIFF) d[cx][q] -= uc[q];
            } else {
#pragma unroll
              for (int q = 0; q < RPL; ++q) d[cx][q] = T(0);
            }
          }
#pragma unroll
          for (int j = 0; j < CHUNK; ++j) {
            if (j < k) {
              const T wyz = s_wyz[wib][j][ln];
              const T w0 = s_wx[wib][j][0], w1 = s_wx[wib][j][1], w2 = s_wx[wib][j][2], w3 = s_wx[wib][j][3];
#pragma unroll
              for (int q = 0; q < RPL; ++q) {
                T line = w0 * d[0][q] + w1 * d[1][q] + w2 * d[2][q] + w3 * d[3][q];
                acc[j][q] += wyz * line;
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < CHUNK; ++j) {
          if (j < k) {
            const int64_t row = s_row[wib][j];
            if (DIFF) {
              T ui[RPL];
              ld<T, RPL>(u + row * ld_ + col, ui);
#pragma unroll
              for (int q = 0; q < RPL; ++q) acc[j][q] += uc[q] - ui[q];
            }
            st<T, RPL>(a + row * ld_ + col, acc[j]);
          }
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace

cpm_status cpm_build_cells(cpm_ctx *c) {
  cudaStream_t st = c->stream;
  cudaFree(c->d_cell_start); cudaFree(c->d_cell_rows); cudaFree(c->d_cell_key);
  c->d_cell_start = nullptr; c->d_cell_rows = nullptr; c->d_cell_key = nullptr;
  c->ncells = 0;
  c->nbulk = 0;
  const int64_t nkeys = c->nb * 512;
  int32_t *count = nullptr, *offs = nullptr, *flag = nullptr, *cellpos = nullptr, *d_tot = nullptr;
  int32_t h_tot = 0, h_cells = 0, nb32 = 0;
  cpm_status rc = CPM_OK;
#define TRY(x)                                             \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_) { rc = cpm_internal_cuda_err(e_); goto done; } \
  } while (0)
  TRY(cudaMalloc(&count, sizeof(int32_t) * nkeys));
  TRY(cudaMalloc(&offs, sizeof(int32_t) * nkeys));
  TRY(cudaMalloc(&flag, sizeof(int32_t) * nkeys));
  TRY(cudaMalloc(&cellpos, sizeof(int32_t) * nkeys));
  TRY(cudaMalloc(&d_tot, sizeof(int32_t)));
  TRY(cudaMemsetAsync(count, 0, sizeof(int32_t) * nkeys, st));
  cell_count_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(c->d_rbase, c->NS, count);
  TRY(cpm_exclusive_scan(count, offs, nkeys, d_tot, st));
  TRY(cudaMemcpyAsync(&h_tot, d_tot, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  flag_nonzero_kernel<<<cpm_grid(nkeys, 256), 256, 0, st>>>(count, nkeys, flag);
  TRY(cpm_exclusive_scan(flag, cellpos, nkeys, d_tot, st));
  TRY(cudaMemcpyAsync(&h_cells, d_tot, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  c->nbulk = h_tot;
  c->ncells = h_cells;
  nb32 = h_tot;
  TRY(cudaMalloc(&c->d_cell_rows, sizeof(int32_t) * std::max<int64_t>(c->nbulk, 1)));
  TRY(cudaMalloc(&c->d_cell_start, sizeof(int32_t) * (c->ncells + 1)));
  TRY(cudaMalloc(&c->d_cell_key, sizeof(uint32_t) * std::max<int64_t>(c->ncells, 1)));
  // scatter with a cursor copy of the offsets, then order each bucket
  TRY(cudaMemcpyAsync(flag, offs, sizeof(int32_t) * nkeys, cudaMemcpyDeviceToDevice, st));
  cell_scatter_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(c->d_rbase, c->NS, flag, c->d_cell_rows);
  cell_finish_kernel<<<cpm_grid(nkeys, 256), 256, 0, st>>>(count, offs, cellpos, nkeys, c->d_cell_rows,
                                                           c->d_cell_start, c->d_cell_key);
  TRY(cudaMemcpyAsync(c->d_cell_start + c->ncells, &nb32, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(st));
done:
#undef TRY
  cudaFree(count); cudaFree(offs); cudaFree(flag); cudaFree(cellpos); cudaFree(d_tot);
  return rc;
}

template <typename T>
void cpm_launch_gather_cells(const cpm_ctx *c, const ApplyArgs<T> &A, const T *u, T *a, int nrhs, int64_t ld,
                             cudaStream_t st, bool diff) {
  if (c->ncells == 0) return;
  unsigned g = (unsigned)std::min<int64_t>((c->ncells + WARPS - 1) / WARPS, 152 * 8);
  if (g < 1) g = 1;
  const int rpl = (nrhs > 32) ? 2 : 1;
  if (rpl == 2) {
    if (diff)
      gather_cells_kernel<T, true, 2><<<g, WARPS * 32, 0, st>>>(A, c->d_cell_start, c->d_cell_key, c->d_cell_rows,
                                                               c->ncells, u, a, nrhs, ld);
    else
      gather_cells_kernel<T, false, 2><<<g, WARPS * 32, 0, st>>>(A, c->d_cell_start, c->d_cell_key, c->d_cell_rows,
                                                                c->ncells, u, a, nrhs, ld);
  } else {
    if (diff)
      gather_cells_kernel<T, true, 1><<<g, WARPS * 32, 0, st>>>(A, c->d_cell_start, c->d_cell_key, c->d_cell_rows,
                                                               c->ncells, u, a, nrhs, ld);
    else
      gather_cells_kernel<T, false, 1><<<g, WARPS * 32, 0, st>>>(A, c->d_cell_start, c->d_cell_key, c->d_cell_rows,
                                                                c->ncells, u, a, nrhs, ld);
  }
}
template void cpm_launch_gather_cells<float>(const cpm_ctx *, const ApplyArgs<float> &, const float *, float *, int,
                                             int64_t, cudaStream_t, bool);
template void cpm_launch_gather_cells<double>(const cpm_ctx *, const ApplyArgs<double> &, const double *, double *,
                                              int, int64_t, cudaStream_t, bool);
