// band.cu -- construction of the computational band Omega(S) on the device.
//
// Sec. 5.1 / Alg. 1 grow the band by a breadth-first search from one node near
// S, evaluating cp_S only near S; the paper stores it in a two-level sparse
// grid (coarse blocks selecting fine blocks, Sec. 2.3).  Here the search runs
// at the granularity of 8^3 bricks: each frontier brick evaluates all of its
// nodes in one CTA (one thread per node, FP64 closest points), records the
// member mask |x - cp_S(x)| <= r (Eq. 3), and inserts the face-neighbour bricks
// that a member node touches into a device hash table (CAS on 64-bit keys).
// Newly inserted bricks form the next frontier.  Member nodes are then numbered
// in canonical order (bricks by (bz, by, bx), nodes by (lz, ly, lx)).
//
// Difference from node-level BFS: a visited brick keeps all of its members,
// not only those connected to the seed; for a band that is one connected tube
// (every workload here) the two sets coincide.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "cpm_internal.cuh"
#include "util.cuh"

namespace {

__global__ void seed_kernel(unsigned long long *hkeys, int64_t hcap, uint64_t key, int32_t *front, unsigned *err) {
  bool fresh;
  int64_t p = cpm_hash_insert(hkeys, hcap, key, &fresh);
  if (p < 0) atomicOr(err, CPM_DEVERR_HASH);
  else front[0] = (int32_t)p;
}

// one CTA of 512 threads per frontier brick
__global__ void __launch_bounds__(512) eval_bricks_kernel(ShapeDev shape, int dim, double h, double rband,
                                                          unsigned long long *hkeys, int64_t hcap,
                                                          unsigned long long *hmask, const int32_t *front,
                                                          int nfront, int32_t *next, int *next_n,
                                                          unsigned long long *n_inserted, unsigned *err) {
  __shared__ unsigned long long words[8];
  __shared__ int faces;
  for (int fb = blockIdx.x; fb < nfront; fb += gridDim.x) {
    int32_t slot = front[fb];
    int bx, by, bz;
    cpm_brick_unkey((int64_t)hkeys[slot], bx, by, bz);
    if (threadIdx.x < 8) words[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) faces = 0;
    __syncthreads();
    int l = threadIdx.x, lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    bool member = false;
    if (dim == 3 || lz == 0) {
      double x[3], cp[3];
      cpm_node_x(dim, h, bx * 8 + lx, by * 8 + ly, bz * 8 + lz, x);
      if (cpm_cp_S(shape, x, cp)) {
        // the analytic shapes always have a closest point; the level-set
        // Newton iteration (App. A) can fail to converge only far from the
        // surface (deep inside, near the bumps' medial axes), at nodes that
        // bricks reach but the band does not: they are taken as outside, and
        // every stencil node of every band row is checked present afterwards.
        // A failure where the first-order distance estimate |phi| / |grad phi|
        // puts the node inside the band is a genuine failure near S.
        if (shape.kind != CPM_SHAPE_BUMPY) {
          atomicOr(err, CPM_DEVERR_CP);
        } else {
          double phi, g[3];
          cpm_bumpy::bumpy_eval(shape, x, &phi, g, nullptr);
          const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
          if (!(gn > 0.0) || fabs(phi) <= rband * gn) atomicOr(err, CPM_DEVERR_CP);
        }
      } else {
        double d[3] = {rn_sub(x[0], cp[0]), rn_sub(x[1], cp[1]), rn_sub(x[2], cp[2])};
        member = rn_norm3(d) <= rband;
      }
    }
    unsigned bal = __ballot_sync(0xffffffffu, member);
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0 && bal)
      atomicOr(&words[w >> 1], (unsigned long long)bal << (32 * (w & 1)));
    if (member) {
      int f = 0;
      if (lx == 0) f |= 1;
      if (lx == 7) f |= 2;
      if (ly == 0) f |= 4;
      if (ly == 7) f |= 8;
      if (dim == 3 && lz == 0) f |= 16;
      if (dim == 3 && lz == 7) f |= 32;
      if (f) atomicOr(&faces, f);
    }
    __syncthreads();
    if (threadIdx.x < 8) hmask[(int64_t)slot * 8 + threadIdx.x] = words[threadIdx.x];
    if (threadIdx.x < 6 && ((faces >> threadIdx.x) & 1)) {
      int a = threadIdx.x >> 1, s = (threadIdx.x & 1) ? 1 : -1;
      int nb3[3] = {bx, by, bz};
      nb3[a] += s;
      bool fresh = false;
      int64_t p = cpm_hash_insert(hkeys, hcap, (uint64_t)cpm_brick_key(nb3[0], nb3[1], nb3[2]), &fresh);
      if (p < 0) {
        atomicOr(err, CPM_DEVERR_HASH);
      } else if (fresh) {
        unsigned long long cnt = atomicAdd(n_inserted, 1ull);
        if (2 * (int64_t)(cnt + 2) > hcap) atomicOr(err, CPM_DEVERR_HASH);
        int q = atomicAdd(next_n, 1);
        next[q] = (int32_t)p;  // next has hcap entries, more than the table can hold
      }
    }
    __syncthreads();
  }
}

__global__ void active_flags_kernel(const unsigned long long *hkeys, const unsigned long long *hmask, int64_t hcap,
                                    int32_t *flag) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < hcap; s += (int64_t)gridDim.x * blockDim.x) {
    int on = 0;
    if (hkeys[s] != CPM_HASH_EMPTY)
      for (int w = 0; w < 8; ++w) on |= (hmask[s * 8 + w] != 0ull);
    flag[s] = on;
  }
}

__global__ void compact_active_kernel(const unsigned long long *hkeys, const int32_t *flag, const int32_t *pos,
                                      int64_t hcap, int64_t *keys, int32_t *slots) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < hcap; s += (int64_t)gridDim.x * blockDim.x)
    if (flag[s]) {
      keys[pos[s]] = (int64_t)hkeys[s];
      slots[pos[s]] = (int32_t)s;
    }
}

__global__ void sorted_bricks_kernel(const int32_t *slots, const unsigned long long *hmask, int64_t nb,
                                     uint64_t *bmask, int32_t *brank, int32_t *bcount, int32_t *slot_to_sorted) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    int32_t s = slots[b];
    int run = 0;
    for (int w = 0; w < 8; ++w) {
      uint64_t m = hmask[(int64_t)s * 8 + w];
      bmask[b * 8 + w] = m;
      brank[b * 8 + w] = run;
      run += __popcll(m);
    }
    bcount[b] = run;
    slot_to_sorted[s] = (int32_t)b;
  }
}

__global__ void brick_nbr_kernel(const int64_t *bkey, int64_t nb, const unsigned long long *hkeys, int64_t hcap,
                                 const int32_t *slot_to_sorted, int32_t *bnbr) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nb * 27; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = q / 27;
    int o = (int)(q % 27);
    int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    int bx, by, bz;
    cpm_brick_unkey(bkey[b], bx, by, bz);
    int64_t p = cpm_hash_find(hkeys, hcap, (uint64_t)cpm_brick_key(bx + dx, by + dy, bz + dz));
    bnbr[q] = (p < 0) ? -1 : slot_to_sorted[p];
  }
}

// one CTA (512 threads) per sorted brick: number members, store ijk and cp_S
__global__ void __launch_bounds__(512) nodes_kernel(ShapeDev shape, int dim, double h, const int64_t *bkey,
                                                    const uint64_t *bmask, const int32_t *brank,
                                                    const int32_t *bstart, int64_t nb, int32_t *ijk, double *cp,
                                                    uint32_t *rself, unsigned *err) {
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    int l = threadIdx.x, lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    uint64_t word = bmask[b * 8 + lz];
    int bit = ly * 8 + lx;
    if (!((word >> bit) & 1ull)) continue;
    uint64_t below = bit ? (word & ((1ull << bit) - 1ull)) : 0ull;
    int64_t idx = (int64_t)bstart[b] + brank[b * 8 + lz] + __popcll(below);
    int bx, by, bz;
    cpm_brick_unkey(bkey[b], bx, by, bz);
    int i = bx * 8 + lx, j = by * 8 + ly, k = bz * 8 + lz;
    ijk[idx * 3] = i; ijk[idx * 3 + 1] = j; ijk[idx * 3 + 2] = k;
    double x[3], c[3];
    cpm_node_x(dim, h, i, j, k, x);
    if (cpm_cp_S(shape, x, c)) atomicOr(err, CPM_DEVERR_CP);
    cp[idx * 3] = c[0]; cp[idx * 3 + 1] = c[1]; cp[idx * 3 + 2] = c[2];
    rself[idx] = ((uint32_t)b << 9) | (uint32_t)l;
  }
}

// per PDE row: interpolation stencil base location and t (FP64 and FP32)
__global__ void row_stencil_kernel(BandView v, const double *cp, const unsigned long long *hkeys, int64_t hcap,
                                   const int32_t *slot_to_sorted, uint32_t *rbase, double *t64, float *t32,
                                   unsigned *err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.NS; i += (int64_t)gridDim.x * blockDim.x) {
    double y[3] = {cp[i * 3], cp[i * 3 + 1], cp[i * 3 + 2]};
    int base[3];
    double t[3];
    cpm_stencil_of(v.dim, v.h, v.np1, y, base, t);
    int bb[3] = {base[0] >> 3, base[1] >> 3, base[2] >> 3};
    int64_t p = cpm_hash_find(hkeys, hcap, (uint64_t)cpm_brick_key(bb[0], bb[1], bb[2]));
    int32_t b = (p < 0) ? -1 : slot_to_sorted[p];
    if (b < 0) {
      atomicOr(err, CPM_DEVERR_MISSING_NODE);
      rbase[i] = 0;
    } else {
      int lx = base[0] & 7, ly = base[1] & 7, lz = base[2] & 7;
      rbase[i] = ((uint32_t)b << 9) | (uint32_t)(lz * 64 + ly * 8 + lx);
      const int np1 = v.np1, nz = (v.dim == 3) ? np1 : 1;
      for (int cz = 0; cz < nz; ++cz)
        for (int cy = 0; cy < np1; ++cy)
          for (int cx = 0; cx < np1; ++cx)
            if (cpm_node_index(v, b, lx + cx, ly + cy, lz + cz) < 0) atomicOr(err, CPM_DEVERR_MISSING_NODE);
    }
    for (int a = 0; a < 3; ++a) {
      t64[i * 3 + a] = t[a];
      t32[i * 3 + a] = (float)t[a];
    }
  }
}

double shape_area(const cpm_shape_desc *s) {
  const double pi = 3.14159265358979323846;
  switch (s->kind) {
    case CPM_SHAPE_CIRCLE: return 2 * pi * s->R;
    case CPM_SHAPE_SPHERE: return 4 * pi * s->R * s->R;
    case CPM_SHAPE_TORUS: return 4 * pi * pi * s->R * s->rt;
    default: return 4 * pi * (1 + std::fabs(s->amp)) * (1 + std::fabs(s->amp)) * 1.5;
  }
}

}  // namespace

cpm_status cpm_internal_cuda_err(cudaError_t e) {
  (void)cudaGetLastError();
  return (e == cudaErrorMemoryAllocation) ? CPM_ERR_OOM : CPM_ERR_CUDA;
}

int cpm_device_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { (void)cudaGetLastError(); return 152; }
  if (cached[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      (void)cudaGetLastError();
      n = 152;
    }
    cached[dev] = n;
  }
  return cached[dev];
}

cpm_status cpm_ensure(WorkBuf &b, size_t bytes) {
  if (b.bytes >= bytes) return CPM_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  CPM_CUDA_TRY(cudaMalloc(&b.p, bytes));
  b.bytes = bytes;
  return CPM_OK;
}

// Eq. (3) with q = 1
static double eq3_radius(int dim, int p, double h) {
  double half = ((double)p + 1.0) / 2.0;
  return h * std::sqrt((double)(dim - 1) * (half * half) + (1.0 + half) * (1.0 + half));
}

// one attempt with a given hash capacity; on CPM_ERR_CAPACITY the caller retries
static cpm_status build_once(cpm_ctx *c, int64_t hcap) {
  cudaStream_t st = c->stream;
  unsigned long long *hkeys = nullptr, *hmask = nullptr, *n_ins = nullptr;
  int32_t *front = nullptr, *next = nullptr, *flag = nullptr, *pos = nullptr, *slots = nullptr,
          *slot_to_sorted = nullptr, *bcount = nullptr, *d_total = nullptr;
  int *d_next_n = nullptr;
  int64_t *keys = nullptr;
  cpm_status rc = CPM_OK;
  int h_next_n = 0, h_total = 0;
  unsigned h_err = 0;
  BandView v;
#define TRY(x)                                   \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_) { rc = cpm_internal_cuda_err(e_); goto done; } \
  } while (0)
  TRY(cudaMalloc(&hkeys, sizeof(unsigned long long) * hcap));
  TRY(cudaMalloc(&hmask, sizeof(unsigned long long) * hcap * 8));
  TRY(cudaMalloc(&front, sizeof(int32_t) * hcap));
  TRY(cudaMalloc(&next, sizeof(int32_t) * hcap));
  TRY(cudaMalloc(&d_next_n, sizeof(int)));
  TRY(cudaMalloc(&n_ins, sizeof(unsigned long long)));
  TRY(cudaMemsetAsync(hkeys, 0xFF, sizeof(unsigned long long) * hcap, st));
  TRY(cudaMemsetAsync(hmask, 0, sizeof(unsigned long long) * hcap * 8, st));
  TRY(cudaMemsetAsync(n_ins, 0, sizeof(unsigned long long), st));
  TRY(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), st));
  {
    int seed[3];
    for (int a = 0; a < 3; ++a) seed[a] = (a < c->dim) ? (int)std::lround(c->shape_seed[a] / c->h) : 0;
    uint64_t key = (uint64_t)cpm_brick_key(seed[0] >> 3, seed[1] >> 3, seed[2] >> 3);
    seed_kernel<<<1, 1, 0, st>>>(hkeys, hcap, key, front, c->d_err);
    int nfront = 1;
    int iters = 0;
    const int max_iters = 1 << 20;
    while (nfront > 0) {
      if (++iters > max_iters) { rc = CPM_ERR_TIMEOUT; goto done; }
      TRY(cudaMemsetAsync(d_next_n, 0, sizeof(int), st));
      int grid = std::min(nfront, c->nsm * 8);
      eval_bricks_kernel<<<grid, 512, 0, st>>>(c->shape, c->dim, c->h, c->rband, hkeys, hcap, hmask, front, nfront,
                                               next, d_next_n, n_ins, c->d_err);
      TRY(cudaGetLastError());
      TRY(cudaMemcpyAsync(&h_next_n, d_next_n, sizeof(int), cudaMemcpyDeviceToHost, st));
      TRY(cudaMemcpyAsync(&h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      TRY(cudaStreamSynchronize(st));
      if (h_err & CPM_DEVERR_HASH) { rc = CPM_ERR_CAPACITY; goto done; }
      if (h_err & CPM_DEVERR_CP) { rc = CPM_ERR_CP_FAILED; goto done; }
      std::swap(front, next);
      nfront = h_next_n;
    }
  }
  // compact the active bricks and sort them by key
  TRY(cudaMalloc(&flag, sizeof(int32_t) * hcap));
  TRY(cudaMalloc(&pos, sizeof(int32_t) * hcap));
  TRY(cudaMalloc(&d_total, sizeof(int32_t)));
  active_flags_kernel<<<cpm_grid(hcap, 256), 256, 0, st>>>(hkeys, hmask, hcap, flag);
  TRY(cpm_exclusive_scan(flag, pos, hcap, d_total, st));
  TRY(cudaMemcpyAsync(&h_total, d_total, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  c->nb = h_total;
  if (c->nb <= 0) { rc = CPM_ERR_ARG; goto done; }
  TRY(cudaMalloc(&keys, sizeof(int64_t) * c->nb));
  TRY(cudaMalloc(&slots, sizeof(int32_t) * c->nb));
  compact_active_kernel<<<cpm_grid(hcap, 256), 256, 0, st>>>(hkeys, flag, pos, hcap, keys, slots);
  TRY(cpm_sort_pairs(keys, slots, c->nb, st));
  c->d_bkey = keys;
  keys = nullptr;
  TRY(cudaMalloc(&c->d_bmask, sizeof(uint64_t) * c->nb * 8));
  TRY(cudaMalloc(&c->d_brank, sizeof(int32_t) * c->nb * 8));
  TRY(cudaMalloc(&c->d_bstart, sizeof(int32_t) * (c->nb + 1)));
  TRY(cudaMalloc(&c->d_bnbr, sizeof(int32_t) * c->nb * 27));
  TRY(cudaMalloc(&bcount, sizeof(int32_t) * (c->nb + 1)));
  TRY(cudaMalloc(&slot_to_sorted, sizeof(int32_t) * hcap));
  TRY(cudaMemsetAsync(slot_to_sorted, 0xFF, sizeof(int32_t) * hcap, st));
  sorted_bricks_kernel<<<cpm_grid(c->nb, 256), 256, 0, st>>>(slots, hmask, c->nb, c->d_bmask, c->d_brank, bcount,
                                                             slot_to_sorted);
  TRY(cpm_exclusive_scan(bcount, c->d_bstart, c->nb, d_total, st));
  TRY(cudaMemcpyAsync(c->d_bstart + c->nb, d_total, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  TRY(cudaMemcpyAsync(&h_total, d_total, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  brick_nbr_kernel<<<cpm_grid(c->nb * 27, 256), 256, 0, st>>>(c->d_bkey, c->nb, hkeys, hcap, slot_to_sorted,
                                                              c->d_bnbr);
  TRY(cudaStreamSynchronize(st));
  c->NS = h_total;
  TRY(cudaMalloc(&c->d_ijk, sizeof(int32_t) * c->NS * 3));
  TRY(cudaMalloc(&c->d_cp, sizeof(double) * c->NS * 3));
  TRY(cudaMalloc(&c->d_rself, sizeof(uint32_t) * c->NS));
  TRY(cudaMalloc(&c->d_rbase, sizeof(uint32_t) * c->NS));
  TRY(cudaMalloc(&c->d_t64, sizeof(double) * c->NS * 3));
  TRY(cudaMalloc(&c->d_t32, sizeof(float) * c->NS * 3));
  nodes_kernel<<<(unsigned)std::min<int64_t>(c->nb, (int64_t)c->nsm * 16), 512, 0, st>>>(
      c->shape, c->dim, c->h, c->d_bkey, c->d_bmask, c->d_brank, c->d_bstart, c->nb, c->d_ijk, c->d_cp, c->d_rself,
      c->d_err);
  v = c->view();
  row_stencil_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(v, c->d_cp, hkeys, hcap, slot_to_sorted, c->d_rbase,
                                                           c->d_t64, c->d_t32, c->d_err);
  TRY(cudaGetLastError());
  TRY(cudaMemcpyAsync(&h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  if (h_err & CPM_DEVERR_CP) rc = CPM_ERR_CP_FAILED;
  else if (h_err & CPM_DEVERR_MISSING_NODE) rc = CPM_ERR_STATE;
done:
#undef TRY
  cudaStreamSynchronize(st);
  if (rc == CPM_OK) {
    c->d_hkeys = hkeys;  // kept for set-up lookups of far nodes
    c->d_slot_to_sorted = slot_to_sorted;
    c->hcap = hcap;
  } else {
    cudaFree(hkeys);
    cudaFree(slot_to_sorted);
  }
  cudaFree(hmask); cudaFree(front); cudaFree(next); cudaFree(d_next_n); cudaFree(n_ins);
  cudaFree(flag); cudaFree(pos); cudaFree(slots); cudaFree(bcount); cudaFree(d_total);
  cudaFree(keys);
  return rc;
}

static void free_band(cpm_ctx *c) {
  cudaFree(c->d_bkey); cudaFree(c->d_bmask); cudaFree(c->d_brank); cudaFree(c->d_bstart); cudaFree(c->d_bnbr);
  cudaFree(c->d_ijk); cudaFree(c->d_cp); cudaFree(c->d_rself); cudaFree(c->d_rbase); cudaFree(c->d_t64);
  cudaFree(c->d_t32); cudaFree(c->d_hkeys); cudaFree(c->d_slot_to_sorted);
  c->d_hkeys = nullptr; c->d_slot_to_sorted = nullptr; c->hcap = 0;
  c->d_bkey = nullptr; c->d_bmask = nullptr; c->d_brank = nullptr; c->d_bstart = nullptr; c->d_bnbr = nullptr;
  c->d_ijk = nullptr; c->d_cp = nullptr; c->d_rself = nullptr; c->d_rbase = nullptr; c->d_t64 = nullptr;
  c->d_t32 = nullptr;
  c->nb = 0; c->NS = 0;
}

cpm_status cpm_internal_band_build(cpm_ctx *c, const cpm_shape_desc *s, double h, int p, double r_band) {
  c->dim = s->dim;
  c->h = h;
  c->p = p;
  c->rband = (r_band > 0) ? r_band : eq3_radius(s->dim, p, h);
  for (int a = 0; a < 3; ++a) c->shape_seed[a] = s->seed[a];
  c->shape.kind = s->kind; c->shape.dim = s->dim; c->shape.K = s->K;
  c->shape.R = s->R; c->shape.rt = s->rt; c->shape.amp = s->amp; c->shape.width = s->width;
  c->shape.newton_maxit = 200;
  // test hook: a forced small iteration cap makes the projection fail next to S
  if (const char *e = std::getenv("CPM_NEWTON_MAXIT")) {
    const int v = std::atoi(e);
    if (v >= 1) c->shape.newton_maxit = v;
  }
  if (s->K > 0) {
    CPM_CUDA_TRY(cudaMalloc(&c->d_shape_a, sizeof(double) * s->K));
    CPM_CUDA_TRY(cudaMalloc(&c->d_shape_c, sizeof(double) * 3 * s->K));
    CPM_CUDA_TRY(cudaMemcpy(c->d_shape_a, s->a, sizeof(double) * s->K, cudaMemcpyHostToDevice));
    CPM_CUDA_TRY(cudaMemcpy(c->d_shape_c, s->c, sizeof(double) * 3 * s->K, cudaMemcpyHostToDevice));
  }
  c->shape.a = c->d_shape_a;
  c->shape.c = c->d_shape_c;
  // brick-count estimate: band volume / brick volume, generous occupancy margin
  double nodes = shape_area(s) * 2.0 * c->rband / std::pow(h, (double)s->dim);
  double bricks = nodes / (s->dim == 3 ? 512.0 : 64.0) * 6.0 + 1024.0;
  int64_t hcap = 1 << 12;
  while ((double)hcap < 4.0 * bricks) hcap <<= 1;
  // test hook: a forced small initial capacity exercises the overflow retry
  if (const char *e = std::getenv("CPM_HASH_CAP_INIT")) {
    const long long v = std::atoll(e);
    if (v >= 16) {
      hcap = 16;
      while (hcap < v) hcap <<= 1;
    }
  }
  cpm_status rc = CPM_ERR_CAPACITY;
  for (int attempt = 0; attempt < 4 && rc == CPM_ERR_CAPACITY; ++attempt) {
    free_band(c);
    rc = build_once(c, hcap);
    hcap <<= 2;
  }
  if (rc != CPM_OK) free_band(c);
  return rc;
}

void cpm_internal_free_band(cpm_ctx *c) { free_band(c); }
