// fused1.cu -- the single right-hand side product v = A u in one persistent
// kernel, without the E u intermediate leaving the L2 cache.
//
// A u needs E u at the six FD neighbours of every PDE row (Eq. 8 with the
// discrete Laplacian of Sec. 5), and E u of a row is best computed per stencil
// cell (the ~5 rows sharing one 4x4x4 node set share its loads).  The two
// passes are interleaved over z-slabs of bricks (bricks are stored in (z, y, x)
// order, so a slab is a contiguous range of bricks, rows and cells): "gather"
// items compute E u of the rows of 128 cells of one slab (a lane per cell),
// "combine" items apply the FD stencil to the rows of two bricks; every warp
// claims its own items.  A row's stencil cell lies in
// its own brick or an adjacent one and its FD neighbours too, so the combine of
// slab z reads E u written by the gathers of slabs z-2 .. z+2 only.  Items are
// claimed in the order
//     G(0) ... G(L-1) G(L) C(0) G(L+1) C(1) ... G(S-1) C(S-L-1) C(S-L) ... C(S-1) B
// (L = F1_LAG >= 2) through one atomic ticket; a combine item waits (bounded)
// until the gather items of its window are done.  Every item it waits for has a smaller ticket,
// so it is held by a running block that waits on nothing: the waits always end.
// E u of a slab is consumed a few slabs after it is written, while it is still
// in L2, so HBM sees u once, the per-row fractions, the cell lists and v.  The
// B items (BC rows) depend on nothing.
//
// The arithmetic is that of the two-pass difference form (cells.cu gather,
// apply.cu combine), so the products agree to rounding; the stencil's x-line
// starts are computed from the brick occupancy masks instead of being read
// from a per-cell table.
#include <algorithm>
#include <vector>

#include "apply.cuh"
#include "cpm_internal.cuh"

namespace {

constexpr int F1T = 256;      // threads per block (8 warps, each claiming its own items)
constexpr int F1_GCELLS = 128;  // cells per gather item (4 per lane)
constexpr int F1_CBRICKS = 2;   // bricks per combine item
constexpr int F1_BCROWS = 128;  // BC rows per item
// slabs by which the combine items trail the gathers: the combine of slab z
// needs the gathers up to slab z + 2; issuing it after those of slab z + 8
// leaves them several waves to finish, so the combines find them done instead
// of waiting on the gathers just claimed
constexpr int F1_LAG = 8;
enum { F1_GATHER = 0, F1_COMBINE = 1, F1_BC = 2 };

template <typename T>
struct F1Args {
  ApplyArgs<T> A;
  const int2 *items;           // (kind << 28 | slab, first cell / brick / BC row)
  const int32_t *gtot;         // [S] gather items per slab
  const int32_t *cend;         // [S] end of each slab's cells
  const int32_t *bend;         // [S] end of each slab's bricks
  unsigned *sync;              // [S] gather items done, [S] ticket, [S+1] exits
  const int32_t *cstart;       // [ncells+1]
  const uint32_t *ckey;        // [ncells]
  const int32_t *rows;         // [NS] cell rows, bit 31: the row has flipped E entries
  const int32_t *corr_of_row;  // [NS]
  const int32_t *corr_start, *corr_node, *corr_col;
  const T *corr_w;
  const uint64_t *bspec;       // [nb*8] special rows
  unsigned *err;
  int64_t nitems;
  int S;
  T m, n, rowscale, cs;
  const T *u;
  T *a, *v;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned r;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
  return r;
}

// E u - u (difference form) of the rows of cell cid, as the per-cell gather of
// cells.cu computes it, plus the row's flipped entries
template <typename T, int DIM, int NP>
__device__ __forceinline__ void gather_cell(const F1Args<T> &F, int64_t cid) {
  constexpr int NZ = (DIM == 3) ? NP : 1;
  constexpr bool PAIR = (sizeof(T) == 4);
  const BandView &v = F.A.v;
  const uint32_t key = __ldg(F.ckey + cid);
  const int32_t b = (int32_t)(key >> 9);
  const int l = (int)(key & 511u);
  const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  const int split = (lx + NP - 1 < 8) ? NP : 8 - lx;
  int32_t s0[NZ][NP], s1[NZ][NP];
  bool ok = true;
#pragma unroll
  for (int cz = 0; cz < NZ; ++cz)
#pragma unroll
    for (int cy = 0; cy < NP; ++cy) ok &= cpm_line_start<NP>(v, b, lx, ly, lz, cy, cz, s0[cz][cy], s1[cz][cy]);
  if (!ok) {
    atomicOr(F.err, CPM_DEVERR_MISSING_NODE);
    return;
  }
  const T uc = __ldg(F.u + s0[0][0]);
  T d[NZ][NP][NP];
#pragma unroll
  for (int cz = 0; cz < NZ; ++cz)
#pragma unroll
    for (int cy = 0; cy < NP; ++cy)
#pragma unroll
      for (int cx = 0; cx < NP; ++cx) {
        const int32_t idx = (cx < split) ? (s0[cz][cy] + cx) : (s1[cz][cy] + (cx - split));
        d[cz][cy][cx] = __ldg(F.u + idx) - uc;
      }
  const int32_t q1 = __ldg(F.cstart + cid + 1);
  for (int32_t q = __ldg(F.cstart + cid); q < q1; ++q) {
    const int32_t rf = __ldg(F.rows + q);
    const int64_t row = rf & 0x7fffffff;
    T wx[4], wy[4], wz[4];
    cpm_lagrange<NP, T>(__ldg(F.A.t + 3 * row), wx);
    cpm_lagrange<NP, T>(__ldg(F.A.t + 3 * row + 1), wy);
    if (DIM == 3) cpm_lagrange<NP, T>(__ldg(F.A.t + 3 * row + 2), wz);
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
    acc += uc - __ldg(F.u + row);
    T av = F.cs * acc;
    if (rf < 0) {
      // the row's E entries that the crossing test flipped to BC DOFs
      const int32_t k = __ldg(F.corr_of_row + row);
      T cacc = T(0);
      const int32_t e1 = __ldg(F.corr_start + k + 1);
      for (int32_t e = __ldg(F.corr_start + k); e < e1; ++e)
        cacc += __ldg(F.corr_w + e) * (__ldg(F.u + __ldg(F.corr_col + e)) - F.cs * __ldg(F.u + __ldg(F.corr_node + e)));
      av += cacc;
    }
    F.a[row] = av;
  }
}

// v at the PDE rows of brick b (one warp, 16 node slots per lane), E u read
// through L2
template <typename T, int DIM>
__device__ __forceinline__ void combine_brick(const F1Args<T> &F, int32_t b, int lane) {
  const BandView &v = F.A.v;
  const int64_t NS = v.NS;
  const T inv_h2 = T(v.inv_h * v.inv_h);
  constexpr int nfd = 2 * DIM;
  const int nslot = (DIM == 3) ? 512 : 64;
  for (int l = lane; l < nslot; l += 32) {
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    const uint64_t word = __ldg(reinterpret_cast<const unsigned long long *>(v.bmask) + (int64_t)b * 8 + lz);
    const int bit = ly * 8 + lx;
    if (!((word >> bit) & 1ull)) continue;
    const int64_t i = __ldg(v.bstart + b) + __ldg(v.brank + (int64_t)b * 8 + lz) + __popcll(word & ((1ull << bit) - 1ull));
    const T ui = F.cs * __ldg(F.u + i);
    T s = T(0);
    int present = 0;
    if ((__ldg(reinterpret_cast<const unsigned long long *>(F.bspec) + (int64_t)b * 8 + lz) >> bit) & 1ull) {
      // a row near a curve: its FD columns, flipped ones pointing at BC DOFs
      const int64_t sp = __ldg(F.A.spec_of + i);
      for (int k = 0; k < 6; ++k) {
        const int32_t c = __ldg(F.A.fcol + sp * 6 + k);
        if (c < 0) continue;
        ++present;
        const T uc = __ldg(F.u + c) * ((c < NS) ? F.cs : T(1));
        s += (c < NS) ? (__ldcg(F.a + c) + (uc - ui)) : (uc - ui);
      }
    } else {
      int32_t nbr[6];
      nbr[0] = cpm_node_index(v, b, lx - 1, ly, lz);
      nbr[1] = cpm_node_index(v, b, lx + 1, ly, lz);
      nbr[2] = cpm_node_index(v, b, lx, ly - 1, lz);
      nbr[3] = cpm_node_index(v, b, lx, ly + 1, lz);
      nbr[4] = (DIM == 3) ? cpm_node_index(v, b, lx, ly, lz - 1) : -1;
      nbr[5] = (DIM == 3) ? cpm_node_index(v, b, lx, ly, lz + 1) : -1;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int32_t j = nbr[k];
        if (j < 0) continue;
        ++present;
        s += __ldcg(F.a + j) + (F.cs * __ldg(F.u + j) - ui);
      }
    }
    const T val = F.m * ui + (F.n * inv_h2) * (s - T(nfd - present) * ui);
    F.v[i] = F.rowscale * val;
  }
}

// one BC row
template <typename T>
__device__ __forceinline__ void bc_row(const F1Args<T> &F, int64_t al) {
  const int64_t NS = F.A.v.NS;
  const int cnt = __ldg(F.A.bc_cnt + al);
  T s = T(0);
  for (int e = 0; e < cnt; ++e) {
    const int32_t c = __ldg(F.A.bc_col + al * CPM_BC_STRIDE + e);
    s += __ldg(F.A.bc_val + al * CPM_BC_STRIDE + e) * (__ldg(F.u + c) * ((c < NS) ? F.cs : T(1)));
  }
  F.v[NS + al] = s;
}

// blocks per SM: FP64 node values take twice the registers
template <typename T>
constexpr int f1_blocks() { return sizeof(T) == 8 ? 1 : 2; }

template <typename T, int DIM, int NP>
__global__ void __launch_bounds__(F1T, f1_blocks<T>()) fused1_kernel(F1Args<T> F) {
  const int lane = threadIdx.x & 31;
  unsigned *ticket = F.sync + F.S, *exits = F.sync + F.S + 1;
  while (true) {
    // each warp claims its own items: no block barrier ties a warp to the
    // slowest cell of another
    int64_t item = 0;
    if (lane == 0) item = atomicAdd(ticket, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= F.nitems) break;
    const int2 it = __ldg(F.items + item);
    const int kind = it.x >> 28, slab = it.x & 0x0fffffff;
    if (kind == F1_GATHER) {
      const int64_t end = min((int64_t)it.y + F1_GCELLS, (int64_t)__ldg(F.cend + slab));
      for (int64_t cid = (int64_t)it.y + lane; cid < end; cid += 32) gather_cell<T, DIM, NP>(F, cid);
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(F.sync + slab, 1u);
    } else if (kind == F1_COMBINE) {
      if (lane == 0) {
        // the gathers of slabs slab-2 .. slab+2 (all claimed before this item)
        for (int z = max(0, slab - 2); z <= min(F.S - 1, slab + 2); ++z) {
          const unsigned target = (unsigned)__ldg(F.gtot + z);
          int polls = 0;
          while (ld_acquire(F.sync + z) < target) {
            if (++polls > (1 << 20)) {
              atomicOr(F.err, CPM_DEVERR_WAIT);
              break;
            }
            __nanosleep(200);
          }
        }
      }
      __syncwarp();
      const int32_t bend = min(it.y + F1_CBRICKS, __ldg(F.bend + slab));
      for (int32_t b = it.y; b < bend; ++b) combine_brick<T, DIM>(F, b, lane);
    } else {
      const int64_t end = min((int64_t)it.y + F1_BCROWS, F.A.v.NC);
      for (int64_t al = (int64_t)it.y + lane; al < end; al += 32) bc_row<T>(F, al);
    }
  }
  // the last warp out resets the counters for the next product
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(exits, 1u) == gridDim.x * (F1T / 32) - 1) {
      for (int z = 0; z < F.S; ++z) F.sync[z] = 0u;
      *ticket = 0u;
      *exits = 0u;
      __threadfence();
    }
  }
}

__global__ void corr_of_row_kernel(const int32_t *corr_row, int64_t ncorr, int32_t *corr_of_row) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ncorr; q += (int64_t)gridDim.x * blockDim.x)
    corr_of_row[corr_row[q]] = (int32_t)q;
}

__global__ void flag_rows_kernel(const int32_t *cell_rows, int64_t n, const int32_t *corr_of_row, int32_t *rows) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = cell_rows[q];
    rows[q] = (corr_of_row[r] >= 0) ? (int32_t)((uint32_t)r | 0x80000000u) : r;
  }
}

__global__ void bspec_kernel(const int32_t *spec_row, int64_t nspec, const uint32_t *rself,
                             unsigned long long *bspec) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nspec; s += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t rs = rself[spec_row[s]];
    const uint32_t b = rs >> 9, l = rs & 511u;
    atomicOr(bspec + (int64_t)b * 8 + (l >> 6), 1ull << (l & 63u));
  }
}

}  // namespace

void cpm_free_fused1(cpm_ctx *c) {
  cudaFree(c->d_f1_items); cudaFree(c->d_f1_gtot); cudaFree(c->d_f1_cend); cudaFree(c->d_f1_bend);
  cudaFree(c->d_f1_sync);
  cudaFree(c->d_f1_rows); cudaFree(c->d_corr_of_row); cudaFree(c->d_bspec);
  c->d_f1_items = nullptr; c->d_f1_gtot = nullptr; c->d_f1_cend = nullptr; c->d_f1_bend = nullptr;
  c->d_f1_sync = nullptr;
  c->d_f1_rows = nullptr; c->d_corr_of_row = nullptr; c->d_bspec = nullptr;
  c->f1_nitems = 0; c->f1_S = 0;
}

// the item list of the fused product: slabs from the brick keys, each slab's
// cells from the cell keys (both sorted), then the interleaved order above
cpm_status cpm_build_fused1(cpm_ctx *c) {
  cpm_free_fused1(c);
  if (c->ncells == 0 || c->nb == 0) return CPM_OK;
  cudaStream_t st = c->stream;
  std::vector<int64_t> bkey(c->nb);
  std::vector<uint32_t> ckey(c->ncells);
  CPM_CUDA_TRY(cudaMemcpy(bkey.data(), c->d_bkey, sizeof(int64_t) * c->nb, cudaMemcpyDeviceToHost));
  CPM_CUDA_TRY(cudaMemcpy(ckey.data(), c->d_cell_key, sizeof(uint32_t) * c->ncells, cudaMemcpyDeviceToHost));
  // slab boundaries in brick order
  std::vector<int64_t> bs{0};
  for (int64_t b = 1; b < c->nb; ++b)
    if ((bkey[b] >> 42) != (bkey[b - 1] >> 42)) bs.push_back(b);
  bs.push_back(c->nb);
  const int S = (int)bs.size() - 1;
  // cells per slab (cells are ordered by base brick): the first cell of each
  // slab's first brick
  std::vector<int64_t> cs(S + 1);
  for (int z = 0; z <= S; ++z)
    cs[z] = std::lower_bound(ckey.begin(), ckey.end(), bs[z],
                             [](uint32_t k, int64_t b) { return (int64_t)(k >> 9) < b; }) - ckey.begin();
  std::vector<int2> items;
  std::vector<int32_t> gtot(S, 0), cend(S), bend(S);
  for (int z = 0; z < S; ++z) {
    cend[z] = (int32_t)cs[z + 1];
    bend[z] = (int32_t)bs[z + 1];
  }
  for (int s = 0; s < S + F1_LAG; ++s) {
    if (s < S)
      for (int64_t f = cs[s]; f < cs[s + 1]; f += F1_GCELLS) {
        items.push_back(make_int2((F1_GATHER << 28) | s, (int)f));
        ++gtot[s];
      }
    const int z = s - F1_LAG;
    if (z >= 0)
      for (int64_t b = bs[z]; b < bs[z + 1]; b += F1_CBRICKS)
        items.push_back(make_int2((F1_COMBINE << 28) | z, (int)b));
  }
  for (int64_t al = 0; al < c->NC; al += F1_BCROWS) items.push_back(make_int2(F1_BC << 28, (int)al));
  cpm_status rc = CPM_OK;
#define TRY(x)                                             \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_) { rc = cpm_internal_cuda_err(e_); goto fail; } \
  } while (0)
  TRY(cudaMalloc(&c->d_f1_items, sizeof(int2) * items.size()));
  TRY(cudaMalloc(&c->d_f1_gtot, sizeof(int32_t) * S));
  TRY(cudaMalloc(&c->d_f1_cend, sizeof(int32_t) * S));
  TRY(cudaMalloc(&c->d_f1_bend, sizeof(int32_t) * S));
  TRY(cudaMalloc(&c->d_f1_sync, sizeof(unsigned) * (S + 2)));
  TRY(cudaMalloc(&c->d_f1_rows, sizeof(int32_t) * std::max<int64_t>(c->NS, 1)));
  TRY(cudaMalloc(&c->d_corr_of_row, sizeof(int32_t) * std::max<int64_t>(c->NS, 1)));
  TRY(cudaMalloc(&c->d_bspec, sizeof(uint64_t) * 8 * c->nb));
  TRY(cudaMemcpy(c->d_f1_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(c->d_f1_gtot, gtot.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(c->d_f1_cend, cend.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(c->d_f1_bend, bend.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice));
  TRY(cudaMemsetAsync(c->d_f1_sync, 0, sizeof(unsigned) * (S + 2), st));
  TRY(cudaMemsetAsync(c->d_corr_of_row, 0xff, sizeof(int32_t) * std::max<int64_t>(c->NS, 1), st));
  TRY(cudaMemsetAsync(c->d_bspec, 0, sizeof(uint64_t) * 8 * c->nb, st));
  if (c->ncorr > 0)
    corr_of_row_kernel<<<cpm_grid(c->ncorr, 256), 256, 0, st>>>(c->d_corr_row, c->ncorr, c->d_corr_of_row);
  flag_rows_kernel<<<cpm_grid(c->nbulk, 256), 256, 0, st>>>(c->d_cell_rows, c->nbulk, c->d_corr_of_row, c->d_f1_rows);
  if (c->nspec > 0)
    bspec_kernel<<<cpm_grid(c->nspec, 256), 256, 0, st>>>(c->d_spec_row, c->nspec, c->d_rself,
                                                         reinterpret_cast<unsigned long long *>(c->d_bspec));
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(st));
#undef TRY
  c->f1_nitems = (int64_t)items.size();
  c->f1_S = S;
  return CPM_OK;
fail:
  cpm_free_fused1(c);
  return rc;
}

template <typename T>
int cpm_launch_fused1(const cpm_ctx *c, const ApplyArgs<T> &A, T m, T n, T rowscale, T cs, const T *u, T *a, T *v,
                      cudaStream_t st) {
  if (c->f1_nitems == 0) return 0;
  F1Args<T> F;
  F.A = A;
  F.items = c->d_f1_items; F.gtot = c->d_f1_gtot; F.cend = c->d_f1_cend; F.bend = c->d_f1_bend;
  F.sync = c->d_f1_sync;
  F.cstart = c->d_cell_start; F.ckey = c->d_cell_key; F.rows = c->d_f1_rows; F.corr_of_row = c->d_corr_of_row;
  F.corr_start = c->d_corr_start; F.corr_node = c->d_corr_node; F.corr_col = c->d_corr_col;
  if constexpr (sizeof(T) == 8) F.corr_w = reinterpret_cast<const T *>(c->d_corr_w64);
  else F.corr_w = reinterpret_cast<const T *>(c->d_corr_w32);
  F.bspec = c->d_bspec; F.err = c->d_err; F.nitems = c->f1_nitems; F.S = c->f1_S;
  F.m = m; F.n = n; F.rowscale = rowscale; F.cs = cs; F.u = u; F.a = a; F.v = v;
  const unsigned g = (unsigned)std::min<int64_t>(c->f1_nitems, (int64_t)c->nsm * f1_blocks<T>());
  if (c->dim == 3) {
    if (c->p == 2) fused1_kernel<T, 3, 3><<<g, F1T, 0, st>>>(F);
    else fused1_kernel<T, 3, 4><<<g, F1T, 0, st>>>(F);
  } else {
    if (c->p == 2) fused1_kernel<T, 2, 3><<<g, F1T, 0, st>>>(F);
    else fused1_kernel<T, 2, 4><<<g, F1T, 0, st>>>(F);
  }
  return 1;
}
template int cpm_launch_fused1<float>(const cpm_ctx *, const ApplyArgs<float> &, float, float, float, float,
                                      const float *, float *, float *, cudaStream_t);
template int cpm_launch_fused1<double>(const cpm_ctx *, const ApplyArgs<double> &, double, double, double, double,
                                       const double *, double *, double *, cudaStream_t);
