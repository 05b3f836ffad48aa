// cells.cu -- PDE rows bucketed by the base node ("cell") of their
// interpolation stencil, and the batched products built on the buckets.
//
// All rows whose closest points fall in the same grid cell share the same
// 4x4x4 stencil nodes (Eq. 1); only their weights differ.  On a narrow band
// several rows (about 2 r / h divided by the number of cells the surface
// crosses per normal line, ~5 in 3D) share each cell.  With many right-hand
// sides the extension E u is bound by moving node values, so one warp takes a
// whole cell: it holds the cell's node values for its columns in registers and
// applies the separable weights of every row of the cell to them.
//
// Rows near an interior boundary use the same cell gather; the entries their
// crossing test flipped (node j replaced by its BC twin, Sec. 4) are applied
// afterwards as a sparse correction w (u_twin - u_j) from a list built here.
//
// The buckets are built by a counting sort over the dense (brick, local) key
// space, with each bucket then ordered by row index, so the layout does not
// depend on the scheduling of the atomics.
#include <algorithm>

#include "apply.cuh"
#include "cpm_internal.cuh"
#include "util.cuh"

namespace {

__global__ void cell_count_kernel(const uint32_t *rbase, int64_t NS, int32_t *count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NS; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(count + (rbase[i] & ~CPM_SPECIAL_BIT), 1);
}

__global__ void cell_scatter_kernel(const uint32_t *rbase, int64_t NS, int32_t *cursor, int32_t *rows) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NS; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = atomicAdd(cursor + (rbase[i] & ~CPM_SPECIAL_BIT), 1);
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

__global__ void set_i32_kernel(int32_t *p, int32_t v) { *p = v; }

// FD neighbour columns of every PDE row (x-, x+, y-, y+, z-, z+; -1 where
// absent; the flipped columns for rows near interior boundaries), padded to 8
__global__ void nbr8_kernel(BandView v, const uint32_t *rself, const uint32_t *rbase, const int32_t *spec_of,
                            const int32_t *fcol, int32_t *nbr8) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.NS; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t o[8];
    if (rbase[i] & CPM_SPECIAL_BIT) {
      const int64_t sp = spec_of[i];
      for (int k = 0; k < 6; ++k) o[k] = fcol[sp * 6 + k];
    } else {
      const uint32_t rs = rself[i];
      const int32_t b = (int32_t)(rs >> 9);
      const int l = (int)(rs & 511u);
      const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
      o[0] = cpm_node_index(v, b, lx - 1, ly, lz);
      o[1] = cpm_node_index(v, b, lx + 1, ly, lz);
      o[2] = cpm_node_index(v, b, lx, ly - 1, lz);
      o[3] = cpm_node_index(v, b, lx, ly + 1, lz);
      o[4] = (v.dim == 3) ? cpm_node_index(v, b, lx, ly, lz - 1) : -1;
      o[5] = (v.dim == 3) ? cpm_node_index(v, b, lx, ly, lz + 1) : -1;
    }
    o[6] = o[7] = -1;
    int4 *dst = reinterpret_cast<int4 *>(nbr8 + i * 8);
    dst[0] = make_int4(o[0], o[1], o[2], o[3]);
    dst[1] = make_int4(o[4], o[5], o[6], o[7]);
  }
}

// node of stencil entry e (x fastest) of the row with packed base rb
__device__ __forceinline__ int32_t entry_node(const BandView &v, uint32_t rb, int e) {
  const int32_t b = (int32_t)((rb & ~CPM_SPECIAL_BIT) >> 9);
  const int l = (int)(rb & 511u);
  return cpm_node_index(v, b, (l & 7) + (e & 3), ((l >> 3) & 7) + ((e >> 2) & 3), (l >> 6) + (e >> 4));
}

// number of flipped interpolation entries of each special row
__global__ void corr_count_kernel(BandView v, const int32_t *spec_row, int64_t nspec, const uint32_t *rbase,
                                  const int32_t *ecol, int32_t *cnt) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nspec; s += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t rb = rbase[spec_row[s]];
    int n = 0;
    for (int e = 0; e < 64; ++e)
      if (cpm_in_stencil(e, v.np1, v.dim)) n += (ecol[s * 64 + e] != entry_node(v, rb, e));
    cnt[s] = n;
  }
}

__global__ void corr_fill_kernel(BandView v, const int32_t *spec_row, int64_t nspec, const uint32_t *rbase,
                                 const int32_t *ecol, const double *ew, const int32_t *cnt, const int32_t *offs,
                                 const int32_t *rowpos, int32_t *corr_row, int32_t *corr_start, int32_t *node,
                                 int32_t *col, double *w64, float *w32) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nspec; s += (int64_t)gridDim.x * blockDim.x) {
    if (cnt[s] == 0) continue;
    const int32_t i = spec_row[s];
    const uint32_t rb = rbase[i];
    corr_row[rowpos[s]] = i;
    corr_start[rowpos[s]] = offs[s];
    int32_t o = offs[s];
    for (int e = 0; e < 64; ++e) {
      if (!cpm_in_stencil(e, v.np1, v.dim)) continue;
      const int32_t j = entry_node(v, rb, e), ce = ecol[s * 64 + e];
      if (ce == j) continue;
      node[o] = j;
      col[o] = ce;
      w64[o] = ew[s * 64 + e];
      w32[o] = (float)ew[s * 64 + e];
      ++o;
    }
  }
}

constexpr int CHUNK = 8;   // rows of a cell whose weights are staged together
constexpr int WARPS = 8;   // warps per block

template <typename T, int R>
struct VecT;
template <> struct VecT<float, 1> { typedef float t; };
template <> struct VecT<float, 2> { typedef float2 t; };
template <> struct VecT<double, 1> { typedef double t; };
template <> struct VecT<double, 2> { typedef double2 t; };

template <typename T, int R>
__device__ __forceinline__ void vld(const T *p, T out[R]) {
  typedef typename VecT<T, R>::t V;
  const V x = __ldg(reinterpret_cast<const V *>(p));
  const T *q = reinterpret_cast<const T *>(&x);
#pragma unroll
  for (int k = 0; k < R; ++k) out[k] = q[k];
}

template <typename T, int R>
__device__ __forceinline__ void vst(T *p, const T in[R]) {
  typedef typename VecT<T, R>::t V;
  V x;
  T *q = reinterpret_cast<T *>(&x);
#pragma unroll
  for (int k = 0; k < R; ++k) q[k] = in[k];
  *reinterpret_cast<V *>(p) = x;
}

// acc[r] += w d[r] and d[r] -= c[r] over a lane's R columns; two FP32 columns
// go through one packed instruction (FFMA2 / FADD2 of sm_100+), with the same
// rounding as the scalar FMA and add
template <typename T, int R>
__device__ __forceinline__ void axpy_w(T (&acc)[R], T w, const T (&d)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] += w * d[r];
}
template <>
__device__ __forceinline__ void axpy_w<float, 2>(float (&acc)[2], float w, const float (&d)[2]) {
  const float2 o = __ffma2_rn(make_float2(w, w), make_float2(d[0], d[1]), make_float2(acc[0], acc[1]));
  acc[0] = o.x;
  acc[1] = o.y;
}
template <typename T, int R>
__device__ __forceinline__ void sub_v(T (&d)[R], const T (&c)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) d[r] -= c[r];
}
template <>
__device__ __forceinline__ void sub_v<float, 2>(float (&d)[2], const float (&c)[2]) {
  const float2 o = __fadd2_rn(make_float2(d[0], d[1]), make_float2(-c[0], -c[1]));
  d[0] = o.x;
  d[1] = o.y;
}

// One warp per cell; each lane takes R adjacent columns (32 R per group).  For
// a group the lane loads the cell's node values (NX x positions per pass, XH
// passes) into registers and applies each row of the cell: the y-z weights
// along each x position (P[cx] = sum_{cy,cz} w_y w_z u), then the x weights.
// Partial sums of the passes wait in shared memory.
//
// DIFF (the FP32 form): the node values enter as differences to the cell's
// base-node value u_c and each row adds u_c - u_i, which equals
// sum_n w_n (u_n - u_i) since sum_n w_n = 1; rounding then stays relative to
// local differences.
template <typename T, bool DIFF, int DIM, int NP, int XH, int R>
__global__ void __launch_bounds__(WARPS * 32, 2)
    gather_cells_kernel(ApplyArgs<T> A, const int32_t *__restrict__ cstart, const uint32_t *__restrict__ ckey,
                        const int32_t *__restrict__ crows, int64_t ncells, T cs, const T *__restrict__ u,
                        T *__restrict__ a, int nrhs, int64_t ld_) {
  constexpr int NZ = (DIM == 3) ? NP : 1;
  constexpr int NL = NP * NZ;  // stencil lines along x
  constexpr int NN = NP * NL;  // stencil nodes
  constexpr int NX = NP / XH;  // x positions per pass
  static_assert(NX * XH == NP, "passes must split the stencil's x positions");
  typedef typename VecT<T, R>::t V;
  __shared__ __align__(16) T s_wyz[WARPS][CHUNK][NL];
  __shared__ __align__(16) T s_wx[WARPS][CHUNK][4];
  __shared__ int32_t s_row[WARPS][CHUNK];
  __shared__ __align__(16) int32_t s_idx[WARPS][NN];
  __shared__ V s_acc[(XH > 1) ? WARPS : 1][CHUNK][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ngroups = (nrhs + 32 * R - 1) / (32 * R);
  for (int64_t cid = warp; cid < ncells; cid += nwarps) {
    const uint32_t key = __ldg(ckey + cid);
    // node (x, line) at s_idx[line * NP + x], line = cz * NP + cy
    for (int e = lane; e < NN; e += 32) {
      const int x = e % NP, ln = e / NP;
      s_idx[wib][e] = entry_node(A.v, key, x + 4 * (ln % NP) + 16 * (ln / NP));
    }
    __syncwarp();
    const int32_t base = s_idx[wib][0];
    const int32_t r0 = __ldg(cstart + cid), r1 = __ldg(cstart + cid + 1);
    for (int32_t c0 = r0; c0 < r1; c0 += CHUNK) {
      const int k = min(CHUNK, r1 - c0);
      if (lane < k) {
        const int32_t row = __ldg(crows + c0 + lane);
        s_row[wib][lane] = row;
        T wx[4], wy[4], wz[4];
        cpm_lagrange<NP, T>(__ldg(A.t + 3 * (int64_t)row), wx);
        cpm_lagrange<NP, T>(__ldg(A.t + 3 * (int64_t)row + 1), wy);
        if (DIM == 3) cpm_lagrange<NP, T>(__ldg(A.t + 3 * (int64_t)row + 2), wz);
        else { wz[0] = T(1); wz[1] = wz[2] = wz[3] = T(0); }
#pragma unroll
        for (int q = 0; q < NP; ++q) s_wx[wib][lane][q] = wx[q];
#pragma unroll
        for (int q = 0; q < NL; ++q) s_wyz[wib][lane][q] = wy[q % NP] * wz[q / NP];
      }
      __syncwarp();
      for (int grp = 0; grp < ngroups; ++grp) {
        const int col = (grp * 32 + lane) * R;
        const bool on = col < nrhs;
        T uc[R];
#pragma unroll
        for (int q = 0; q < R; ++q) uc[q] = T(0);
        if (DIFF && on) vld<T, R>(u + (int64_t)base * ld_ + col, uc);
#pragma unroll 1
        for (int xp = 0; xp < XH; ++xp) {
          T d[NL][NX][R];
#pragma unroll
          for (int ln = 0; ln < NL; ++ln) {
#pragma unroll
            for (int q = 0; q < NX; ++q) {
              const int32_t idx = s_idx[wib][ln * NP + xp * NX + q];
              if (on) {
                vld<T, R>(u + (int64_t)idx * ld_ + col, d[ln][q]);
                if (DIFF) sub_v<T, R>(d[ln][q], uc);
              } else {
#pragma unroll
                for (int r = 0; r < R; ++r) d[ln][q][r] = T(0);
              }
            }
          }
#pragma unroll 1
          for (int j = 0; j < k; ++j) {
            T P[NX][R];
#pragma unroll
            for (int q = 0; q < NX; ++q)
#pragma unroll
              for (int r = 0; r < R; ++r) P[q][r] = T(0);
#pragma unroll
            for (int ln = 0; ln < NL; ++ln) {
              const T w = s_wyz[wib][j][ln];
#pragma unroll
              for (int q = 0; q < NX; ++q) axpy_w<T, R>(P[q], w, d[ln][q]);
            }
            T part[R];
#pragma unroll
            for (int r = 0; r < R; ++r) part[r] = T(0);
#pragma unroll
            for (int q = 0; q < NX; ++q) axpy_w<T, R>(part, s_wx[wib][j][xp * NX + q], P[q]);
            if (XH > 1 && xp > 0) {
              const V pv = s_acc[(XH > 1) ? wib : 0][j][lane];
              const T *pp = reinterpret_cast<const T *>(&pv);
#pragma unroll
              for (int r = 0; r < R; ++r) part[r] += pp[r];
            }
            if (XH > 1 && xp < XH - 1) {
              V pv;
              T *pp = reinterpret_cast<T *>(&pv);
#pragma unroll
              for (int r = 0; r < R; ++r) pp[r] = part[r];
              s_acc[(XH > 1) ? wib : 0][j][lane] = pv;
            } else if (on) {
              const int64_t row = s_row[wib][j];
              if (DIFF) {
                T ui[R];
                vld<T, R>(u + row * ld_ + col, ui);
#pragma unroll
                for (int r = 0; r < R; ++r) part[r] += uc[r] - ui[r];
              }
#pragma unroll
              for (int r = 0; r < R; ++r) part[r] *= cs;
              vst<T, R>(a + row * ld_ + col, part);
            }
          }
        }
      }
      __syncwarp();
    }
  }
}

// a_i += sum over the row's flipped entries of w (u_twin - u_node): one warp
// per special row with flips, lanes over R adjacent columns
template <typename T, int R>
__global__ void __launch_bounds__(256) correct_kernel(const int32_t *__restrict__ crow,
                                                      const int32_t *__restrict__ cstart,
                                                      const int32_t *__restrict__ cnode,
                                                      const int32_t *__restrict__ ccol, const T *__restrict__ cw,
                                                      int64_t ncorr, T cs, const T *__restrict__ u,
                                                      T *__restrict__ a, int nrhs, int64_t ld_) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ngroups = (nrhs + 32 * R - 1) / (32 * R);
  for (int64_t q = warp; q < ncorr; q += nwarps) {
    const int64_t row = __ldg(crow + q);
    const int32_t e0 = __ldg(cstart + q), e1 = __ldg(cstart + q + 1);
    for (int grp = 0; grp < ngroups; ++grp) {
      const int col = (grp * 32 + lane) * R;
      if (col >= nrhs) continue;
      T acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = T(0);
      for (int32_t e = e0; e < e1; ++e) {
        const T w = __ldg(cw + e);
        T ut[R], un[R];
        vld<T, R>(u + (int64_t)__ldg(ccol + e) * ld_ + col, ut);
        vld<T, R>(u + (int64_t)__ldg(cnode + e) * ld_ + col, un);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += w * (ut[r] - cs * un[r]);
      }
      T av[R];
      vld<T, R>(a + row * ld_ + col, av);
#pragma unroll
      for (int r = 0; r < R; ++r) av[r] += acc[r];
      vst<T, R>(a + row * ld_ + col, av);
    }
  }
}

// per cell the start of each of its stencil lines along x (slot cz * 4 + cy of
// 16; np1^2 used in 3D, np1 in 2D): s0 the DOF of the line's first node; s1 the
// DOF of its first node past the brick's x face where the line crosses it (-1
// otherwise)
__global__ void cell_lines_kernel(BandView v, const uint32_t *cell_key, int64_t ncells, int2 *lines) {
  const int np1 = v.np1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncells * 16;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cid = t >> 4;
    const int ln = (int)(t & 15);
    const int cy = ln & 3, cz = ln >> 2;
    int2 out = make_int2(-1, -1);
    if (cy < np1 && (v.dim == 3 ? cz < np1 : cz == 0)) {
      const uint32_t key = cell_key[cid];
      const int32_t b = (int32_t)(key >> 9);
      const int l = (int)(key & 511u);
      const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
      out.x = cpm_node_index(v, b, lx, ly + cy, lz + cz);
      if (lx + np1 - 1 >= 8) out.y = cpm_node_index(v, b, 8, ly + cy, lz + cz);
    }
    lines[t] = out;
  }
}

__global__ void row_cell_kernel(const int32_t *cell_start, int64_t ncells, int32_t *row_cell) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x)
    for (int32_t q = cell_start[c]; q < cell_start[c + 1]; ++q) row_cell[q] = (int32_t)c;
}

// single right-hand side: one thread per PDE row, rows taken in cell order so
// that the rows of a cell (same 64 nodes) run in neighbouring threads and share
// the cell's line table and node values in cache
template <typename T, bool DIFF, int DIM, int NP>
__global__ void __launch_bounds__(256) gather1_kernel(ApplyArgs<T> A, const int32_t *__restrict__ crows,
                                                      const int32_t *__restrict__ row_cell,
                                                      const uint32_t *__restrict__ ckey,
                                                      const int2 *__restrict__ lines, int64_t NS, T cs,
                                                      const T *__restrict__ u, T *__restrict__ a) {
  constexpr int NZ = (DIM == 3) ? NP : 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < NS; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = __ldg(crows + q);
    const int32_t cid = __ldg(row_cell + q);
    const int lx = (int)(__ldg(ckey + cid) & 7u);
    const int split = (lx + NP - 1 < 8) ? NP : 8 - lx;
    const int2 *ln = lines + (int64_t)cid * 16;
    T wx[4], wy[4], wz[4];
    cpm_lagrange<NP, T>(__ldg(A.t + 3 * row), wx);
    cpm_lagrange<NP, T>(__ldg(A.t + 3 * row + 1), wy);
    if (DIM == 3) cpm_lagrange<NP, T>(__ldg(A.t + 3 * row + 2), wz);
    else { wz[0] = T(1); wz[1] = wz[2] = wz[3] = T(0); }
    const T uc = DIFF ? __ldg(u + __ldg(&ln[0].x)) : T(0);
    T acc = T(0);
#pragma unroll
    for (int cz = 0; cz < NZ; ++cz) {
      T pz = T(0);
#pragma unroll
      for (int cy = 0; cy < NP; ++cy) {
        const int2 se = __ldg(ln + cz * 4 + cy);
        T line = T(0);
#pragma unroll
        for (int cx = 0; cx < NP; ++cx) {
          const int32_t idx = (cx < split) ? (se.x + cx) : (se.y + (cx - split));
          line += wx[cx] * (__ldg(u + idx) - uc);
        }
        pz += wy[cy] * line;
      }
      acc += wz[cz] * pz;
    }
    if (DIFF) acc += uc - __ldg(u + row);
    a[row] = cs * acc;
  }
}

// single right-hand side, one thread per cell: the thread loads the cell's
// NP^dim node values once (as differences to the base node's value) and applies
// the separable weights of each of the cell's rows to them, so the node loads
// and index arithmetic are shared by the ~5 rows of a cell instead of repeated
// per row.  FP32 x pairs go through packed FMAs.
template <typename T, int DIM, int NP>
__global__ void __launch_bounds__(128) gather1c_kernel(ApplyArgs<T> A, const int32_t *__restrict__ cstart,
                                                       const uint32_t *__restrict__ ckey,
                                                       const int32_t *__restrict__ crows,
                                                       const int2 *__restrict__ lines, int64_t ncells, T cs,
                                                       const T *__restrict__ u, T *__restrict__ a) {
  constexpr int NZ = (DIM == 3) ? NP : 1;
  constexpr bool PAIR = (sizeof(T) == 4);
  for (int64_t cid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cid < ncells;
       cid += (int64_t)gridDim.x * blockDim.x) {
    const int lx = (int)(__ldg(ckey + cid) & 7u);
    const int split = (lx + NP - 1 < 8) ? NP : 8 - lx;
    const int2 *ln = lines + cid * 16;
    const T uc = __ldg(u + __ldg(&ln[0].x));
    T d[NZ][NP][NP];  // [cz][cy][cx]
#pragma unroll
    for (int cz = 0; cz < NZ; ++cz)
#pragma unroll
      for (int cy = 0; cy < NP; ++cy) {
        const int2 se = __ldg(ln + cz * 4 + cy);
#pragma unroll
        for (int cx = 0; cx < NP; ++cx) {
          const int32_t idx = (cx < split) ? (se.x + cx) : (se.y + (cx - split));
          d[cz][cy][cx] = __ldg(u + idx) - uc;
        }
      }
    const int32_t q1 = __ldg(cstart + cid + 1);
    for (int32_t q = __ldg(cstart + cid); q < q1; ++q) {
      const int64_t row = __ldg(crows + q);
      T wx[4], wy[4], wz[4];
      cpm_lagrange<NP, T>(__ldg(A.t + 3 * row), wx);
      cpm_lagrange<NP, T>(__ldg(A.t + 3 * row + 1), wy);
      if (DIM == 3) cpm_lagrange<NP, T>(__ldg(A.t + 3 * row + 2), wz);
      else { wz[0] = T(1); wz[1] = wz[2] = wz[3] = T(0); }
      T P[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int cz = 0; cz < NZ; ++cz)
#pragma unroll
        for (int cy = 0; cy < NP; ++cy) {
          const T w = wy[cy] * wz[cz];
          if constexpr (PAIR) {
            const float2 p01 = __ffma2_rn(make_float2(w, w), make_float2(d[cz][cy][0], d[cz][cy][1]),
                                          make_float2(P[0], P[1]));
            P[0] = p01.x; P[1] = p01.y;
            if constexpr (NP == 4) {
              const float2 p23 = __ffma2_rn(make_float2(w, w), make_float2(d[cz][cy][2], d[cz][cy][3]),
                                            make_float2(P[2], P[3]));
              P[2] = p23.x; P[3] = p23.y;
            } else {
              P[2] += w * d[cz][cy][2];
            }
          } else {
#pragma unroll
            for (int cx = 0; cx < NP; ++cx) P[cx] += w * d[cz][cy][cx];
          }
        }
      T acc = T(0);
#pragma unroll
      for (int cx = 0; cx < NP; ++cx) acc += wx[cx] * P[cx];
      acc += uc - __ldg(u + row);
      a[row] = cs * acc;
    }
  }
}

// single right-hand side correction: one thread per row with flipped entries
template <typename T>
__global__ void __launch_bounds__(256) correct1_kernel(const int32_t *__restrict__ crow,
                                                       const int32_t *__restrict__ cstart,
                                                       const int32_t *__restrict__ cnode,
                                                       const int32_t *__restrict__ ccol, const T *__restrict__ cw,
                                                       int64_t ncorr, T cs, const T *__restrict__ u,
                                                       T *__restrict__ a) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ncorr; q += (int64_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    const int32_t e1 = __ldg(cstart + q + 1);
    for (int32_t e = __ldg(cstart + q); e < e1; ++e)
      acc += __ldg(cw + e) * (__ldg(u + __ldg(ccol + e)) - cs * __ldg(u + __ldg(cnode + e)));
    a[__ldg(crow + q)] += acc;
  }
}

}  // namespace

void cpm_free_cells(cpm_ctx *c) {
  cpm_free_fused1(c);
  cudaFree(c->d_cell_start); cudaFree(c->d_cell_rows); cudaFree(c->d_cell_key); cudaFree(c->d_nbr8);
  cudaFree(c->d_corr_row); cudaFree(c->d_corr_start); cudaFree(c->d_corr_node); cudaFree(c->d_corr_col);
  cudaFree(c->d_corr_w64); cudaFree(c->d_corr_w32); cudaFree(c->d_cell_lines); cudaFree(c->d_row_cell);
  c->d_cell_lines = nullptr; c->d_row_cell = nullptr;
  c->d_cell_start = nullptr; c->d_cell_rows = nullptr; c->d_cell_key = nullptr; c->d_nbr8 = nullptr;
  c->d_corr_row = nullptr; c->d_corr_start = nullptr; c->d_corr_node = nullptr; c->d_corr_col = nullptr;
  c->d_corr_w64 = nullptr; c->d_corr_w32 = nullptr;
  c->ncells = 0; c->nbulk = 0; c->ncorr = 0; c->ncorr_ent = 0;
}

cpm_status cpm_build_cells(cpm_ctx *c) {
  cudaStream_t st = c->stream;
  cpm_free_cells(c);
  const int64_t nkeys = c->nb * 512;
  const int64_t nsp = std::max<int64_t>(c->nspec, 1);
  int32_t *count = nullptr, *offs = nullptr, *flag = nullptr, *cellpos = nullptr, *d_tot = nullptr;
  int32_t *ccnt = nullptr, *coffs = nullptr, *cflag = nullptr, *cpos = nullptr;
  int32_t h_tot = 0, h_cells = 0, h_ent = 0, h_rows = 0;
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
  TRY(cudaMalloc(&c->d_cell_rows, sizeof(int32_t) * std::max<int64_t>(c->nbulk, 1)));
  TRY(cudaMalloc(&c->d_cell_start, sizeof(int32_t) * (c->ncells + 1)));
  TRY(cudaMalloc(&c->d_cell_key, sizeof(uint32_t) * std::max<int64_t>(c->ncells, 1)));
  // scatter with a cursor copy of the offsets, then order each bucket
  TRY(cudaMemcpyAsync(flag, offs, sizeof(int32_t) * nkeys, cudaMemcpyDeviceToDevice, st));
  cell_scatter_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(c->d_rbase, c->NS, flag, c->d_cell_rows);
  cell_finish_kernel<<<cpm_grid(nkeys, 256), 256, 0, st>>>(count, offs, cellpos, nkeys, c->d_cell_rows,
                                                           c->d_cell_start, c->d_cell_key);
  set_i32_kernel<<<1, 1, 0, st>>>(c->d_cell_start + c->ncells, h_tot);
  TRY(cudaMalloc(&c->d_cell_lines, sizeof(int2) * 16 * std::max<int64_t>(c->ncells, 1)));
  TRY(cudaMalloc(&c->d_row_cell, sizeof(int32_t) * std::max<int64_t>(c->NS, 1)));
  if (c->ncells > 0) {
    cell_lines_kernel<<<cpm_grid(c->ncells * 16, 256), 256, 0, st>>>(c->view(), c->d_cell_key, c->ncells,
                                                                    reinterpret_cast<int2 *>(c->d_cell_lines));
    row_cell_kernel<<<cpm_grid(c->ncells, 256), 256, 0, st>>>(c->d_cell_start, c->ncells, c->d_row_cell);
  }
  TRY(cudaMalloc(&c->d_nbr8, sizeof(int32_t) * 8 * std::max<int64_t>(c->NS, 1)));
  nbr8_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(c->view(), c->d_rself, c->d_rbase, c->d_spec_of, c->d_spec_fcol,
                                                    c->d_nbr8);
  TRY(cudaGetLastError());
  // flipped interpolation entries of the special rows
  TRY(cudaMalloc(&ccnt, sizeof(int32_t) * nsp));
  TRY(cudaMalloc(&coffs, sizeof(int32_t) * nsp));
  TRY(cudaMalloc(&cflag, sizeof(int32_t) * nsp));
  TRY(cudaMalloc(&cpos, sizeof(int32_t) * nsp));
  if (c->nspec > 0) {
    corr_count_kernel<<<cpm_grid(c->nspec, 128), 128, 0, st>>>(c->view(), c->d_spec_row, c->nspec, c->d_rbase,
                                                               c->d_spec_ecol, ccnt);
    TRY(cpm_exclusive_scan(ccnt, coffs, c->nspec, d_tot, st));
    TRY(cudaMemcpyAsync(&h_ent, d_tot, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    flag_nonzero_kernel<<<cpm_grid(c->nspec, 256), 256, 0, st>>>(ccnt, c->nspec, cflag);
    TRY(cpm_exclusive_scan(cflag, cpos, c->nspec, d_tot, st));
    TRY(cudaMemcpyAsync(&h_rows, d_tot, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
  }
  c->ncorr = h_rows;
  c->ncorr_ent = h_ent;
  TRY(cudaMalloc(&c->d_corr_row, sizeof(int32_t) * std::max<int64_t>(c->ncorr, 1)));
  TRY(cudaMalloc(&c->d_corr_start, sizeof(int32_t) * (c->ncorr + 1)));
  TRY(cudaMalloc(&c->d_corr_node, sizeof(int32_t) * std::max<int64_t>(c->ncorr_ent, 1)));
  TRY(cudaMalloc(&c->d_corr_col, sizeof(int32_t) * std::max<int64_t>(c->ncorr_ent, 1)));
  TRY(cudaMalloc(&c->d_corr_w64, sizeof(double) * std::max<int64_t>(c->ncorr_ent, 1)));
  TRY(cudaMalloc(&c->d_corr_w32, sizeof(float) * std::max<int64_t>(c->ncorr_ent, 1)));
  set_i32_kernel<<<1, 1, 0, st>>>(c->d_corr_start + c->ncorr, h_ent);
  if (c->ncorr > 0)
    corr_fill_kernel<<<cpm_grid(c->nspec, 128), 128, 0, st>>>(c->view(), c->d_spec_row, c->nspec, c->d_rbase,
                                                              c->d_spec_ecol, c->d_spec_ew, ccnt, coffs, cpos,
                                                              c->d_corr_row, c->d_corr_start, c->d_corr_node,
                                                              c->d_corr_col, c->d_corr_w64, c->d_corr_w32);
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(st));
  rc = cpm_build_fused1(c);
done:
#undef TRY
  cudaFree(count); cudaFree(offs); cudaFree(flag); cudaFree(cellpos); cudaFree(d_tot);
  cudaFree(ccnt); cudaFree(coffs); cudaFree(cflag); cudaFree(cpos);
  if (rc != CPM_OK) cpm_free_cells(c);
  return rc;
}

// x passes of the cell gather that keep the node values of one pass in
// registers: a divisor of NP; FP64 pairs of columns are not held four x wide
template <typename T, int NP, int R>
__host__ __device__ constexpr bool xh_ok(int xh) {
  return (NP % xh == 0) && !(sizeof(T) == 8 && R == 2 && NP / xh > 2) && !(sizeof(T) == 8 && NP / xh > 2);
}

template <typename T, int DIM, int NP, int R, int XH>
static void launch_cells_xh(const cpm_ctx *c, const ApplyArgs<T> &A, T cs, const T *u, T *a, int nrhs, int64_t ld,
                            cudaStream_t st, unsigned g) {
  if constexpr (xh_ok<T, NP, R>(XH))
    gather_cells_kernel<T, true, DIM, NP, XH, R><<<g, WARPS * 32, 0, st>>>(
        A, c->d_cell_start, c->d_cell_key, c->d_cell_rows, c->ncells, cs, u, a, nrhs, ld);
}

// the default number of x passes (node values of one pass near 64 registers)
template <typename T, int NP, int R>
constexpr int default_xh() {
  return (NP == 3) ? ((sizeof(T) == 8 && R == 2) ? 3 : 1) : ((sizeof(T) == 8) ? ((R == 2) ? 4 : 2) : 2);
}

int cpm_cells_default_xh(int np1, bool fp64, int rpl) {
  if (np1 == 3) return fp64 ? (rpl == 2 ? default_xh<double, 3, 2>() : default_xh<double, 3, 1>())
                            : (rpl == 2 ? default_xh<float, 3, 2>() : default_xh<float, 3, 1>());
  return fp64 ? (rpl == 2 ? default_xh<double, 4, 2>() : default_xh<double, 4, 1>())
              : (rpl == 2 ? default_xh<float, 4, 2>() : default_xh<float, 4, 1>());
}

template <typename T, int DIM, int NP, int R>
static void launch_cells_k(const cpm_ctx *c, const ApplyArgs<T> &A, T cs, const T *u, T *a, int nrhs, int64_t ld,
                           cudaStream_t st) {
  int xh = c->tune.cells_xh[sizeof(T) == 8 ? 1 : 0][R - 1];
  if (xh <= 0 || xh > 4 || !xh_ok<T, NP, R>(xh)) xh = default_xh<T, NP, R>();
  const int per_sm = c->tune.cells_blocks_per_sm > 0 ? c->tune.cells_blocks_per_sm : 16;
  unsigned g = (unsigned)std::min<int64_t>((c->ncells + WARPS - 1) / WARPS, (int64_t)c->nsm * per_sm);
  if (g < 1) g = 1;
  switch (xh) {
    case 1: launch_cells_xh<T, DIM, NP, R, 1>(c, A, cs, u, a, nrhs, ld, st, g); break;
    case 2: launch_cells_xh<T, DIM, NP, R, 2>(c, A, cs, u, a, nrhs, ld, st, g); break;
    case 3: launch_cells_xh<T, DIM, NP, R, 3>(c, A, cs, u, a, nrhs, ld, st, g); break;
    default: launch_cells_xh<T, DIM, NP, R, 4>(c, A, cs, u, a, nrhs, ld, st, g); break;
  }
}

template <typename T, int NP, int R>
static void launch_cells_np(const cpm_ctx *c, const ApplyArgs<T> &A, T cs, const T *u, T *a, int nrhs, int64_t ld,
                            cudaStream_t st) {
  if (c->dim == 3) launch_cells_k<T, 3, NP, R>(c, A, cs, u, a, nrhs, ld, st);
  else launch_cells_k<T, 2, NP, R>(c, A, cs, u, a, nrhs, ld, st);
}

// the cell gather always takes the difference form (the batched products are
// only used in it)
template <typename T, int R>
static void launch_cells_r(const cpm_ctx *c, const ApplyArgs<T> &A, T cs, const T *u, T *a, int nrhs, int64_t ld,
                           cudaStream_t st, bool /*diff*/) {
  if (c->p == 2) launch_cells_np<T, 3, R>(c, A, cs, u, a, nrhs, ld, st);
  else launch_cells_np<T, 4, R>(c, A, cs, u, a, nrhs, ld, st);
  if (c->ncorr > 0) {
    const T *cw;
    if constexpr (sizeof(T) == 8) cw = reinterpret_cast<const T *>(c->d_corr_w64);
    else cw = reinterpret_cast<const T *>(c->d_corr_w32);
    unsigned gc = (unsigned)std::min<int64_t>((c->ncorr + 7) / 8, (int64_t)c->nsm * 16);
    correct_kernel<T, R><<<gc, 256, 0, st>>>(c->d_corr_row, c->d_corr_start, c->d_corr_node, c->d_corr_col, cw,
                                             c->ncorr, cs, u, a, nrhs, ld);
  }
}

template <typename T>
int cpm_launch_gather_cells(const cpm_ctx *c, const ApplyArgs<T> &A, T cs, const T *u, T *a, int nrhs, int64_t ld,
                            cudaStream_t st, bool diff, int rpl) {
  if (c->ncells == 0) return 0;
  if (rpl == 2) launch_cells_r<T, 2>(c, A, cs, u, a, nrhs, ld, st, diff);
  else launch_cells_r<T, 1>(c, A, cs, u, a, nrhs, ld, st, diff);
  return (c->ncorr > 0) ? 2 : 1;
}
template int cpm_launch_gather_cells<float>(const cpm_ctx *, const ApplyArgs<float> &, float, const float *, float *,
                                            int, int64_t, cudaStream_t, bool, int);
template int cpm_launch_gather_cells<double>(const cpm_ctx *, const ApplyArgs<double> &, double, const double *,
                                             double *, int, int64_t, cudaStream_t, bool, int);

template <typename T>
int cpm_launch_gather1(const cpm_ctx *c, const ApplyArgs<T> &A, T cs, const T *u, T *a, cudaStream_t st, bool diff) {
  if (c->ncells == 0) return 0;
  const unsigned g = cpm_grid(c->NS, 256);
  const int2 *lines = reinterpret_cast<const int2 *>(c->d_cell_lines);
  if (diff && c->tune.single_mode != 1) {
    // one thread per cell (the difference form only)
    const unsigned gc = cpm_grid(c->ncells, 128);
#define CPM_G1C(D, NP)                                                                                           \
  gather1c_kernel<T, D, NP><<<gc, 128, 0, st>>>(A, c->d_cell_start, c->d_cell_key, c->d_cell_rows, lines, c->ncells, \
                                                cs, u, a)
    if (c->dim == 3) {
      if (c->p == 2) CPM_G1C(3, 3); else CPM_G1C(3, 4);
    } else {
      if (c->p == 2) CPM_G1C(2, 3); else CPM_G1C(2, 4);
    }
#undef CPM_G1C
  } else {
#define CPM_G1(D, NP)                                                                                       \
  do {                                                                                                      \
    if (diff)                                                                                               \
      gather1_kernel<T, true, D, NP><<<g, 256, 0, st>>>(A, c->d_cell_rows, c->d_row_cell, c->d_cell_key, lines, \
                                                        c->NS, cs, u, a);                                   \
    else                                                                                                    \
      gather1_kernel<T, false, D, NP><<<g, 256, 0, st>>>(A, c->d_cell_rows, c->d_row_cell, c->d_cell_key,     \
                                                         lines, c->NS, cs, u, a);                           \
  } while (0)
  if (c->dim == 3) {
    if (c->p == 2) CPM_G1(3, 3); else CPM_G1(3, 4);
  } else {
    if (c->p == 2) CPM_G1(2, 3); else CPM_G1(2, 4);
  }
#undef CPM_G1
  }
  if (c->ncorr > 0) {
    const T *cw;
    if constexpr (sizeof(T) == 8) cw = reinterpret_cast<const T *>(c->d_corr_w64);
    else cw = reinterpret_cast<const T *>(c->d_corr_w32);
    correct1_kernel<T><<<cpm_grid(c->ncorr, 256), 256, 0, st>>>(c->d_corr_row, c->d_corr_start, c->d_corr_node,
                                                                c->d_corr_col, cw, c->ncorr, cs, u, a);
    return 2;
  }
  return 1;
}
template int cpm_launch_gather1<float>(const cpm_ctx *, const ApplyArgs<float> &, float, const float *, float *,
                                       cudaStream_t, bool);
template int cpm_launch_gather1<double>(const cpm_ctx *, const ApplyArgs<double> &, double, const double *, double *,
                                        cudaStream_t, bool);
