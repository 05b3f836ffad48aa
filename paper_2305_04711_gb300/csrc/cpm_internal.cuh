// cpm_internal.cuh -- device-side data layout and helpers shared by the
// CUDA translation units of the sm_103a CPM library.
//
// Layout in HBM (all owned by one cpm_ctx):
//   bricks   : nb active 8^3 bricks sorted by (bz, by, bx); per brick the
//              member mask as 8 x uint64 (one per z layer, bit = ly*8+lx),
//              the exclusive member count before each layer, the first DOF
//              index of the brick, and the 27 neighbour bricks (-1 = absent).
//   nodes    : per PDE DOF its grid index (int3), cp_S (double3), its own
//              packed location (brick << 9 | local) and the packed location of
//              its interpolation stencil's base node (bit 31 marks a "special"
//              row near an interior boundary, whose stencils are stored
//              explicitly with the crossing-test flips applied).
//   operator : per PDE row the fractional stencil position t = cp/h - base in
//              FP64 and FP32; explicit stencils for special rows; Dirichlet BC
//              rows in a fixed-stride table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/cpm.h"

#define CPM_BRICK 8
#define CPM_NBR27 27
#define CPM_SPECIAL_BIT 0x80000000u
#define CPM_BC_STRIDE 65

// device-side error flags (bit set by kernels, read by the host)
#define CPM_DEVERR_MISSING_NODE 1u   // an interpolation or FD node was absent
#define CPM_DEVERR_CP 2u             // a Newton closest point did not converge
#define CPM_DEVERR_OVERLAP 4u        // a node lies within 2 r of two curves
#define CPM_DEVERR_HASH 8u           // brick hash table full
#define CPM_DEVERR_WAIT 16u          // a bounded wait of the fused product gave up

struct CurveDev {
  int kind, bc, two_sided, n_samples;
  int bc_minus;        // BC type on the minus side (resolved: never 0)
  int projected;       // projected crossing test (Sec. 4.7)
  double p[3], nu[3], ref[3], rad;
  int64_t sample_off;  // offset of this curve's samples in the concatenated layout
};

struct ShapeDev {
  int kind, dim, K;
  int newton_maxit;  // iteration cap of each stage of the level-set projection (200)
  double R, rt, amp, width;
  const double *a;  // device [K]
  const double *c;  // device [3K]
};

// read-only view passed by value to kernels
struct BandView {
  int dim;
  int np1;  // interpolation stencil nodes per axis: p + 1 (4 cubic, 3 quadratic)
  double h, inv_h, rband;
  int64_t nb, NS, NC;
  const uint64_t *bmask;  // [nb*8]
  const int32_t *brank;   // [nb*8]
  const int32_t *bstart;  // [nb+1]
  const int32_t *bnbr;    // [nb*27]
  // brick hash kept after the build for set-up lookups of far nodes
  const unsigned long long *hkeys;  // [hcap]
  const int32_t *slot_to_sorted;    // [hcap]
  int64_t hcap;
};

struct WorkBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct SolveWork;

// launch shapes chosen by the autotuner (tune.cu); 0 means the default
struct Tune {
  int cells_xh[2][2] = {{0, 0}, {0, 0}};  // [FP32 / FP64][columns per lane - 1]: x passes of the cell gather
  int cells_blocks_per_sm = 0;            // grid cap of the cell gather (blocks of 8 warps per SM)
  int combine_warps_per_sm = 0;           // grid cap of the warp-per-row combine
  int vec_blocks_per_sm = 0;              // blocks per SM of the Krylov vector kernels (1, 2 or 4)
  int single_mode = 0;                    // single right-hand side: 0 per-cell / 1 per-row gather + combine, 2 fused
  bool tuned = false;
};

// event-pair timing of operator products and a kernel-launch counter
struct Profiler {
  bool on = false;
  int64_t launches = 0;
  int64_t applies = 0;
  int64_t row_rhs = 0;
  std::vector<cudaEvent_t> ev;  // pairs (start, stop), reused
  size_t used = 0;
};

struct cpm_ctx {
  cudaStream_t stream = nullptr;
  int nsm = 152;                    // streaming multiprocessors of the device (queried at build)
  // the solves run on an internal stream, joined to the caller's by events, so
  // that their iteration groups can be captured and replayed as CUDA graphs
  cudaStream_t istream = nullptr;
  cudaEvent_t ev_join[2] = {nullptr, nullptr};
  // geometry
  ShapeDev shape{};
  double *d_shape_a = nullptr, *d_shape_c = nullptr;
  int dim = 3;
  int p = 3;                        // interpolation degree: 3 (cubic) or 2 (quadratic)
  double h = 0, rband = 0;
  double shape_seed[3] = {0, 0, 0};
  // bricks
  int64_t nb = 0;
  int64_t *d_bkey = nullptr;    // [nb] packed brick coordinates, canonical order
  uint64_t *d_bmask = nullptr;  // [nb*8]
  int32_t *d_brank = nullptr;   // [nb*8]
  int32_t *d_bstart = nullptr;  // [nb+1]
  int32_t *d_bnbr = nullptr;    // [nb*27]
  unsigned long long *d_hkeys = nullptr;  // brick hash (set-up lookups)
  int32_t *d_slot_to_sorted = nullptr;
  int64_t hcap = 0;
  // nodes
  int64_t NS = 0;
  int32_t *d_ijk = nullptr;     // [NS*3]
  double *d_cp = nullptr;       // [NS*3]
  uint32_t *d_rself = nullptr;  // [NS] brick << 9 | local
  uint32_t *d_rbase = nullptr;  // [NS] stencil base location, special bit
  double *d_t64 = nullptr;      // [NS*3]
  float *d_t32 = nullptr;       // [NS*3]
  // boundary
  bool boundary_set = false;
  int ncurves = 0;
  CurveDev *h_curves = nullptr;
  CurveDev *d_curves = nullptr;
  int64_t NC = 0;
  int64_t nsamples_total = 0;
  int32_t *d_bc_of = nullptr;     // [NS] BC DOF index (>= NS) at this node or -1
  int8_t *d_near = nullptr;       // [NS] curve whose 2r zone holds the node, or -1
  int32_t *d_twin = nullptr;      // [NC]
  int32_t *d_bc_curve = nullptr;  // [NC]
  double *d_cpc = nullptr;        // [NC*3]
  int32_t *d_side = nullptr;      // [NC]
  int32_t *d_bc_type = nullptr;   // [NC] BC type of the row (the side opposite cp_S(x_alpha))
  double *d_param = nullptr;      // [NC]
  int32_t *d_bc_cnt = nullptr;    // [NC]
  int32_t *d_curve_first = nullptr;  // [ncurves+1] first BC DOF of each curve
  int32_t *d_bc_col = nullptr;    // [NC*65]
  double *d_bc_val = nullptr;     // [NC*65]
  float *d_bc_val32 = nullptr;    // [NC*65]
  // special rows (rows within 2 r of a curve)
  int64_t nspec = 0;
  int32_t *d_spec_row = nullptr;   // [nspec]
  int32_t *d_spec_of = nullptr;    // [NS] special index or -1
  int32_t *d_spec_ecol = nullptr;  // [nspec*64]
  double *d_spec_ew = nullptr;     // [nspec*64]
  float *d_spec_ew32 = nullptr;    // [nspec*64]
  int32_t *d_spec_fcol = nullptr;  // [nspec*6]
  // PDE rows bucketed by their stencil base node ("cells"), for the batched products
  int64_t ncells = 0, nbulk = 0;
  int32_t *d_cell_start = nullptr;  // [ncells+1]
  int32_t *d_cell_rows = nullptr;   // [nbulk] (nbulk = NS)
  uint32_t *d_cell_key = nullptr;   // [ncells] packed base location (brick << 9 | local)
  int32_t *d_nbr8 = nullptr;        // [NS][8] FD neighbour columns (6 used; flipped near curves)
  int32_t *d_cell_lines = nullptr;  // [ncells][16] int2 line starts of each cell's stencil
  int32_t *d_row_cell = nullptr;    // [NS] cell of each position of cell_rows
  // flipped interpolation entries of the special rows: row i's E entry at node
  // corr_node holds column corr_col instead (a BC DOF), weight corr_w
  int64_t ncorr = 0, ncorr_ent = 0;
  int32_t *d_corr_row = nullptr;    // [ncorr]
  int32_t *d_corr_start = nullptr;  // [ncorr+1]
  int32_t *d_corr_node = nullptr;   // [ncorr_ent]
  int32_t *d_corr_col = nullptr;    // [ncorr_ent]
  double *d_corr_w64 = nullptr;     // [ncorr_ent]
  float *d_corr_w32 = nullptr;      // [ncorr_ent]
  // single right-hand side fused product (fused1.cu): work items over z-slabs
  int64_t f1_nitems = 0;
  int f1_S = 0;
  int2 *d_f1_items = nullptr;        // [f1_nitems] (kind << 28 | slab, first cell / brick / BC row)
  int32_t *d_f1_gtot = nullptr;      // [S] gather items per slab
  int32_t *d_f1_cend = nullptr;      // [S] end of each slab's cells
  int32_t *d_f1_bend = nullptr;      // [S] end of each slab's bricks
  unsigned *d_f1_sync = nullptr;     // [S + 2] gather items done per slab, ticket, exits
  int32_t *d_f1_rows = nullptr;      // [NS] cell rows, bit 31 set where the row has flipped E entries
  int32_t *d_corr_of_row = nullptr;  // [NS] index into the corr lists or -1
  uint64_t *d_bspec = nullptr;       // [nb*8] rows near a curve, per brick
  // transposed structure (adjoint)
  bool transpose_ready = false;
  int64_t nT = 0;                   // entries of the per-column remainder lists
  int32_t *d_cellid = nullptr;      // [nb*512] cell index of a packed base location, -1 if none
  double *d_tblk = nullptr;         // [ncells][64] per-cell blocks of E^T b (one right-hand side; FP32 uses the front half)
  double *d_w1d64 = nullptr;        // [NS][12] per-axis Lagrange factors (transposed gather)
  float *d_w1d32 = nullptr;         // [NS][12]
  int32_t *d_T_ptr = nullptr;       // [N+1] CSR over columns
  int32_t *d_T_row = nullptr;       // [nT] source DOF
  int32_t *d_T_kind = nullptr;      // [nT] 0: flipped FD entry, 1: flipped E entry, 2: BC-row entry
  double *d_T_val = nullptr;        // [nT]
  float *d_T_val32 = nullptr;       // [nT]
  // scratch, reserved in cpm_set_boundary / cpm_reserve (the products and
  // solves themselves allocate nothing)
  WorkBuf a_scratch;                // E u intermediate (also the heat steps' extensions)
  WorkBuf b_scratch;                // transposed FD intermediate
  int64_t res_ld = 0;               // leading dimension the workspaces are reserved for
  int res_flags = 0;                // solve forms reserved (CPM_RESERVE_* bits)
  unsigned *d_err = nullptr;        // device error flags
  unsigned long long *d_counter = nullptr;  // diagnostics counters [4]
  int64_t noflip_twin = 0;
  Profiler prof;
  Tune tune;
  SolveWork *solve = nullptr;        // workspace of the solves (all forms share it)
  BandView view() const {
    BandView v;
    v.dim = dim; v.np1 = p + 1; v.h = h; v.inv_h = 1.0 / h; v.rband = rband;
    v.nb = nb; v.NS = NS; v.NC = NC;
    v.bmask = d_bmask; v.brank = d_brank; v.bstart = d_bstart; v.bnbr = d_bnbr;
    v.hkeys = d_hkeys; v.slot_to_sorted = d_slot_to_sorted; v.hcap = hcap;
    return v;
  }
};

// ---------------------------------------------------------------------------
// host status helpers
#define CPM_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return cpm_internal_cuda_err(e_); \
  } while (0)

cpm_status cpm_internal_cuda_err(cudaError_t e);
// profiler hooks (no-ops unless enabled)
inline void cpm_count_launches(cpm_ctx *c, int k) { c->prof.launches += k; }
void cpm_prof_begin(cpm_ctx *c, cudaStream_t st);
void cpm_prof_end(cpm_ctx *c, cudaStream_t st, int64_t row_rhs);
cpm_status cpm_ensure(WorkBuf &b, size_t bytes);
void cpm_free_boundary(cpm_ctx *c);
cpm_status cpm_build_transpose(cpm_ctx *c);
cpm_status cpm_build_cells(cpm_ctx *c);
void cpm_free_cells(cpm_ctx *c);

// element loop over the [N][nrhs] block of a [N][ld] array without a division
// per element: a block of B threads takes B / nrhs rows at a time, thread t
// column t % nrhs (nrhs <= B)
#define CPM_ROWS_COLS_LOOP(N, nrhs, i, c)                                                     \
  const int c = (int)(threadIdx.x % (unsigned)(nrhs));                                         \
  const int rows_per_ = (int)(blockDim.x / (unsigned)(nrhs));                                  \
  if ((int)(threadIdx.x / (unsigned)(nrhs)) >= rows_per_) return;                              \
  for (int64_t i = blockIdx.x * (int64_t)rows_per_ + threadIdx.x / (unsigned)(nrhs); i < (N); \
       i += (int64_t)gridDim.x * rows_per_)

// SM count of the current device (queried once per device)
int cpm_device_sms();

static inline unsigned cpm_grid(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  const int64_t cap = (int64_t)cpm_device_sms() * 64;  // grid-stride loops beyond this
  if (g > cap) g = cap;
  return (unsigned)g;
}

// ---------------------------------------------------------------------------
// device helpers

// integer floor division by 8 and the remainder in [0, 8)
__host__ __device__ inline int cpm_fdiv8(int v) { return v >> 3; }  // arithmetic shift
__host__ __device__ inline int cpm_fmod8(int v) { return v & 7; }

// packed brick key: 21 bits per coordinate with offset 2^20
__host__ __device__ inline int64_t cpm_brick_key(int bx, int by, int bz) {
  const int64_t o = 1LL << 20;
  return (((int64_t)bz + o) << 42) | (((int64_t)by + o) << 21) | ((int64_t)bx + o);
}
__host__ __device__ inline void cpm_brick_unkey(int64_t k, int &bx, int &by, int &bz) {
  const int64_t o = 1LL << 20, m = (1LL << 21) - 1;
  bz = (int)(((k >> 42) & m) - o);
  by = (int)(((k >> 21) & m) - o);
  bx = (int)((k & m) - o);
}

// DOF index of the node at local coordinates (lx, ly, lz) relative to brick b
// (coordinates may leave [0,8) by up to one brick); -1 if not in the band.
__device__ __forceinline__ int32_t cpm_node_index(const BandView &v, int32_t b, int lx, int ly, int lz) {
  int dx = lx >> 3, dy = ly >> 3, dz = lz >> 3;
  if (dx | dy | dz) {
    b = __ldg(v.bnbr + (int64_t)b * 27 + 13 + dx + 3 * dy + 9 * dz);
    if (b < 0) return -1;
  }
  lx &= 7; ly &= 7; lz &= 7;
  int bit = ly * 8 + lx;
  uint64_t word = __ldg(reinterpret_cast<const unsigned long long *>(v.bmask) + (int64_t)b * 8 + lz);
  if (!((word >> bit) & 1ull)) return -1;
  uint64_t below = (bit == 0) ? 0ull : (word & ((1ull << bit) - 1ull));
  return __ldg(v.bstart + b) + __ldg(v.brank + (int64_t)b * 8 + lz) + __popcll(below);
}

// start of the stencil line (cy, cz) of the cell with base (lx, ly, lz) in
// brick b: s0 the DOF of its first node; s1 that of its first node past the
// brick's x face when the line crosses it.  Nodes of one x-run inside a brick
// are consecutive DOFs (every stencil node is in the band); a line whose first
// node is absent or whose run would pass the last PDE DOF is reported.
template <int NP>
__device__ __forceinline__ bool cpm_line_start(const BandView &v, int32_t b, int lx, int ly, int lz, int cy, int cz,
                                           int32_t &s0, int32_t &s1) {
  const int y = ly + cy, z = lz + cz;
  const int oy = y >> 3, oz = z >> 3, yl = y & 7, zl = z & 7;
  int32_t b0 = b;
  if (oy | oz) b0 = __ldg(v.bnbr + (int64_t)b * 27 + 13 + 3 * oy + 9 * oz);
  if (b0 < 0) return false;
  const uint64_t w0 = __ldg(reinterpret_cast<const unsigned long long *>(v.bmask) + (int64_t)b0 * 8 + zl);
  const int bit = yl * 8 + lx;
  if (!((w0 >> bit) & 1ull)) return false;
  s0 = __ldg(v.bstart + b0) + __ldg(v.brank + (int64_t)b0 * 8 + zl) + __popcll(w0 & ((1ull << bit) - 1ull));
  s1 = s0;
  const int split = (lx + NP - 1 < 8) ? NP : 8 - lx;
  if (s0 + split > v.NS) return false;
  if (split < NP) {
    const int32_t b1 = __ldg(v.bnbr + (int64_t)b0 * 27 + 14);
    if (b1 < 0) return false;
    const uint64_t w1 = __ldg(reinterpret_cast<const unsigned long long *>(v.bmask) + (int64_t)b1 * 8 + zl);
    if (!((w1 >> (yl * 8)) & 1ull)) return false;
    s1 = __ldg(v.bstart + b1) + __ldg(v.brank + (int64_t)b1 * 8 + zl) + __popcll(w1 & ((1ull << (yl * 8)) - 1ull));
    if (s1 + (NP - split) > v.NS) return false;
  }
  return true;
}

// DOF index of grid node (i, j, k) anywhere in the band, through the brick hash
// (set-up only); -1 if absent.
__device__ inline int32_t cpm_lookup_global(const BandView &v, int i, int j, int k) {
  const uint64_t key = (uint64_t)cpm_brick_key(i >> 3, j >> 3, k >> 3);
  uint64_t x = key;
  x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL; x ^= x >> 33;
  const uint64_t mask = (uint64_t)v.hcap - 1;
  uint64_t p = x & mask;
  for (int64_t probe = 0; probe < v.hcap; ++probe) {
    unsigned long long kk = v.hkeys[p];
    if (kk == key) {
      int32_t b = v.slot_to_sorted[p];
      if (b < 0) return -1;
      return cpm_node_index(v, b, i & 7, j & 7, k & 7);
    }
    if (kk == 0xFFFFFFFFFFFFFFFFull) return -1;
    p = (p + 1) & mask;
  }
  return -1;
}

// --- FP64 geometry with explicit rounding (no FMA contraction) -------------
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double rn_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double rn_dot3(const double *a, const double *b) {
  return rn_add(rn_add(rn_mul(a[0], b[0]), rn_mul(a[1], b[1])), rn_mul(a[2], b[2]));
}
__device__ __forceinline__ double rn_norm3(const double *a) { return rn_sqrt(rn_dot3(a, a)); }

// grid node coordinates x = h * (i, j, k)
__device__ __forceinline__ void cpm_node_x(int dim, double h, int i, int j, int k, double x[3]) {
  x[0] = rn_mul((double)i, h);
  x[1] = rn_mul((double)j, h);
  x[2] = (dim == 3) ? rn_mul((double)k, h) : 0.0;
}

// Newton projection onto the bumpy-sphere level set
#include "bumpy.cuh"

// cp_S for the analytic shapes (closed forms; medial-axis points take a fixed
// direction, which keeps the distance exact); returns nonzero on failure.
__device__ __forceinline__ int cpm_cp_S(const ShapeDev &s, const double *x, double *cp) {
  if (s.kind == CPM_SHAPE_CIRCLE) {
    double n = rn_sqrt(rn_add(rn_mul(x[0], x[0]), rn_mul(x[1], x[1])));
    if (n == 0.0) { cp[0] = s.R; cp[1] = 0.0; cp[2] = 0.0; return 0; }
    cp[0] = rn_mul(s.R, rn_div(x[0], n)); cp[1] = rn_mul(s.R, rn_div(x[1], n)); cp[2] = 0.0;
    return 0;
  }
  if (s.kind == CPM_SHAPE_SPHERE) {
    double n = rn_sqrt(rn_add(rn_add(rn_mul(x[0], x[0]), rn_mul(x[1], x[1])), rn_mul(x[2], x[2])));
    if (n == 0.0) { cp[0] = s.R; cp[1] = 0.0; cp[2] = 0.0; return 0; }
    cp[0] = rn_mul(s.R, rn_div(x[0], n)); cp[1] = rn_mul(s.R, rn_div(x[1], n)); cp[2] = rn_mul(s.R, rn_div(x[2], n));
    return 0;
  }
  if (s.kind == CPM_SHAPE_TORUS) {
    double rho = rn_sqrt(rn_add(rn_mul(x[0], x[0]), rn_mul(x[1], x[1])));
    double ux = 1.0, uy = 0.0;
    if (rho != 0.0) { ux = rn_div(x[0], rho); uy = rn_div(x[1], rho); }
    double cx = rn_mul(s.R, ux), cy = rn_mul(s.R, uy);
    double dx = rn_sub(x[0], cx), dy = rn_sub(x[1], cy), dz = x[2];
    double m = rn_sqrt(rn_add(rn_add(rn_mul(dx, dx), rn_mul(dy, dy)), rn_mul(dz, dz)));
    if (m == 0.0) { cp[0] = cx; cp[1] = cy; cp[2] = s.rt; return 0; }
    cp[0] = rn_add(cx, rn_mul(s.rt, rn_div(dx, m)));
    cp[1] = rn_add(cy, rn_mul(s.rt, rn_div(dy, m)));
    cp[2] = rn_mul(s.rt, rn_div(dz, m));
    return 0;
  }
  if (s.kind == CPM_SHAPE_BUMPY) return cpm_cp_bumpy(s, x, cp);
  return 1;
}

// cp to an interior boundary: a point, or a circle (centre p, normal nu, radius)
__device__ __forceinline__ void cpm_cp_C(const CurveDev &cv, const double *x, double *out) {
  if (cv.kind == CPM_CURVE_POINT) { out[0] = cv.p[0]; out[1] = cv.p[1]; out[2] = cv.p[2]; return; }
  double w[3] = {rn_sub(x[0], cv.p[0]), rn_sub(x[1], cv.p[1]), rn_sub(x[2], cv.p[2])};
  double s = rn_dot3(w, cv.nu);
  double q[3] = {rn_sub(w[0], rn_mul(s, cv.nu[0])), rn_sub(w[1], rn_mul(s, cv.nu[1])), rn_sub(w[2], rn_mul(s, cv.nu[2]))};
  double nq = rn_norm3(q);
  if (nq == 0.0) { q[0] = cv.ref[0]; q[1] = cv.ref[1]; q[2] = cv.ref[2]; nq = 1.0; }
  out[0] = rn_add(cv.p[0], rn_mul(cv.rad, rn_div(q[0], nq)));
  out[1] = rn_add(cv.p[1], rn_mul(cv.rad, rn_div(q[1], nq)));
  out[2] = rn_add(cv.p[2], rn_mul(cv.rad, rn_div(q[2], nq)));
}

// stencil of a query point y: the np1 = p + 1 nodes per axis nearest to y.
// Cubic: base floor(y/h) - 1 (y between stencil nodes 1 and 2); quadratic:
// base floor(y/h + 1/2) - 1 (node 1 nearest, every node within 1.5 h, the
// half-width Eq. (3) assumes).  t = y/h - base per axis.
__device__ __forceinline__ void cpm_stencil_of(int dim, double h, int np1, const double *y, int base[3],
                                               double t[3]) {
  for (int a = 0; a < 3; ++a) {
    if (a >= dim) { base[a] = 0; t[a] = 0.0; continue; }
    double s = rn_div(y[a], h);
    base[a] = (np1 == 3) ? (int)floor(rn_add(s, 0.5)) - 1 : (int)floor(s) - 1;
    t[a] = rn_sub(s, (double)base[a]);
  }
}

// entry e of a stencil in the fixed 4 x 4 x 4 layout (x fastest) lies inside
// the np1^dim stencil
__host__ __device__ inline bool cpm_in_stencil(int e, int np1, int dim) {
  return (e & 3) < np1 && ((e >> 2) & 3) < np1 && (dim == 3 ? (e >> 4) < np1 : (e >> 4) == 0);
}

// c_alpha of the BC-row right-hand side: 1 (DIR1), 2 (DIR2), 0 (zero-Neumann)
__host__ __device__ inline double cpm_bc_data_scale(int type) {
  return (type == CPM_BC_DIR1) ? 1.0 : (type == CPM_BC_DIR2) ? 2.0 : 0.0;
}

// 1D cubic Lagrange weights on nodes 0..3 (product form)
template <typename T>
__device__ __forceinline__ void cpm_lagrange4(T t, T w[4]) {
  T a = t, b = t - T(1), c = t - T(2), d = t - T(3);
  w[0] = -(b * c * d) * T(1.0 / 6.0);
  w[1] = (a * c * d) * T(0.5);
  w[2] = -(a * b * d) * T(0.5);
  w[3] = (a * b * c) * T(1.0 / 6.0);
}

// 1D quadratic Lagrange weights on nodes 0..2 (product form)
template <typename T>
__device__ __forceinline__ void cpm_lagrange3(T t, T w[3]) {
  T a = t, b = t - T(1), c = t - T(2);
  w[0] = (b * c) * T(0.5);
  w[1] = -(a * c);
  w[2] = (a * b) * T(0.5);
}

template <int NP, typename T>
__device__ __forceinline__ void cpm_lagrange(T t, T *w) {
  if constexpr (NP == 4) cpm_lagrange4<T>(t, w);
  else cpm_lagrange3<T>(t, w);
}

// run-time degree: weights in w[0..np1), zeros after
template <typename T>
__device__ __forceinline__ void cpm_lagrange_rt(int np1, T t, T w[4]) {
  if (np1 == 4) cpm_lagrange4<T>(t, w);
  else { cpm_lagrange3<T>(t, w); w[3] = T(0); }
}
