// boundary.cu -- interior boundaries on the device (Sec. 4).
//
//  * Omega(C) (Sec. 4.1): band nodes within r of a curve get a BC DOF, numbered
//    after the PDE DOFs in (curve, canonical) order.
//  * Localisation (Sec. 4.6): rows within 2 r of a curve are "special": their
//    interpolation (Eq. 1) and FD (Eq. 2) stencils are stored explicitly with
//    the crossing test applied (Eqs. 8-10): node j is replaced by its BC twin
//    when d*_i . cp_{S-C}(x_j) < 0, d*_i = cp_{S-C}(x_i).  A node within 2 r of
//    two curves is rejected (CPM_ERR_OVERLAP), so each special row and each BC
//    DOF belongs to one curve; a twin is only taken from the row's own curve.
//  * On-C tie (Sec. 4.2): |cp_{S-C}(x)| < 0.1 h^2 means cp_S(x) lies on C and may
//    take either side; the node takes the side of the first node of its own
//    interpolation stencil (x fastest, then y, then z) whose vector is longer.
//  * BC rows (Sec. 4.3), with the type of the side the BC DOF stands in for
//    (the side opposite cp_S(x_alpha); mixed types per side, Sec. 4.2):
//      DIR1 u_alpha = g;  DIR2 u_alpha + sum_beta wbar_beta u_sigma(beta) = 2 g;
//      NEU1 u_alpha - sum_beta w_beta u_sigma(beta) = 0 with the stencil at
//      cp_C(x_alpha);  NEU2 as NEU1 with the stencil at the mirror point
//      cpbar_C(x) = cp_S(2 cp_C(x) - x), which DIR2 uses too.  A stencil's
//      default column is the BC twin, replaced by the PDE DOF when
//      d*_alpha . cp_{S-C}(x_beta) < 0 (Eq. 11).
//
// Geometry uses explicit round-to-nearest FP64 operations so that every flip
// decision is reproducible bit for bit.
#include <cmath>
#include <cstring>
#include <vector>

#include "cpm_internal.cuh"
#include "util.cuh"

namespace {

struct BView {
  BandView v;
  ShapeDev shape;
  const int32_t *ijk;
  const double *cp;
  const uint32_t *rself;
  const CurveDev *curves;
  int ncurves;
};

__device__ __forceinline__ void node_coords(const BView &b, int32_t j, double x[3]) {
  cpm_node_x(b.v.dim, b.v.h, b.ijk[3 * j], b.ijk[3 * j + 1], b.ijk[3 * j + 2], x);
}

// DOF index of grid node (gi, gj, gk): through the brick of node j when the
// node lies within one brick of it, otherwise through the brick hash.
__device__ __forceinline__ int32_t lookup_near(const BView &b, int32_t j, int gi, int gj, int gk) {
  uint32_t rs = b.rself[j];
  int32_t bj = (int32_t)(rs >> 9);
  int l = (int)(rs & 511u);
  int ox = b.ijk[3 * j] - (l & 7), oy = b.ijk[3 * j + 1] - ((l >> 3) & 7), oz = b.ijk[3 * j + 2] - (l >> 6);
  int lx = gi - ox, ly = gj - oy, lz = gk - oz;
  if (lx < -8 || lx > 15 || ly < -8 || ly > 15 || lz < -8 || lz > 15) return cpm_lookup_global(b.v, gi, gj, gk);
  return cpm_node_index(b.v, bj, lx, ly, lz);
}

// unit normal of S at a point y on S: the radial direction of the circle and
// the sphere, the direction from the torus's ring, the level-set gradient of
// the bumpy sphere (App. A)
__device__ void shape_normal(const ShapeDev &sh, const double *y, double n[3]) {
  double d[3] = {y[0], y[1], y[2]};
  if (sh.kind == CPM_SHAPE_BUMPY) {
    double phi;
    cpm_bumpy::bumpy_eval(sh, y, &phi, d, nullptr);
  } else if (sh.kind == CPM_SHAPE_CIRCLE) {
    d[2] = 0.0;
  } else if (sh.kind == CPM_SHAPE_TORUS) {
    const double rho = rn_sqrt(rn_add(rn_mul(y[0], y[0]), rn_mul(y[1], y[1])));
    d[0] = rn_sub(y[0], rn_mul(sh.R, rn_div(y[0], rho)));
    d[1] = rn_sub(y[1], rn_mul(sh.R, rn_div(y[1], rho)));
  }
  const double m = rn_norm3(d);
  n[0] = rn_div(d[0], m); n[1] = rn_div(d[1], m); n[2] = rn_div(d[2], m);
}

// cp_{S-C}(x_j); with the projected test (Sec. 4.7) its components along n_S
// and the circle's tangent nu x (cp_C - p), both at cp_C(x_j), removed in that
// order (a point: n_S only)
__device__ __forceinline__ void zraw(const BView &b, const CurveDev &cv, int32_t j, double z[3]) {
  double x[3], cc[3];
  node_coords(b, j, x);
  cpm_cp_C(cv, x, cc);
  z[0] = rn_sub(b.cp[3 * j], cc[0]);
  z[1] = rn_sub(b.cp[3 * j + 1], cc[1]);
  z[2] = rn_sub(b.cp[3 * j + 2], cc[2]);
  if (!cv.projected) return;
  double n[3];
  shape_normal(b.shape, cc, n);
  const double a = rn_dot3(z, n);
  for (int e = 0; e < 3; ++e) z[e] = rn_sub(z[e], rn_mul(a, n[e]));
  if (cv.kind == CPM_CURVE_CIRCLE) {
    const double w[3] = {rn_sub(cc[0], cv.p[0]), rn_sub(cc[1], cv.p[1]), rn_sub(cc[2], cv.p[2])};
    double t[3] = {rn_sub(rn_mul(cv.nu[1], w[2]), rn_mul(cv.nu[2], w[1])),
                   rn_sub(rn_mul(cv.nu[2], w[0]), rn_mul(cv.nu[0], w[2])),
                   rn_sub(rn_mul(cv.nu[0], w[1]), rn_mul(cv.nu[1], w[0]))};
    const double m = rn_norm3(t);
    for (int e = 0; e < 3; ++e) t[e] = rn_div(t[e], m);
    const double bt = rn_dot3(z, t);
    for (int e = 0; e < 3; ++e) z[e] = rn_sub(z[e], rn_mul(bt, t[e]));
  }
}

// tie-resolved cp_{S-C}(x_j) for one curve (see the file comment)
__device__ void zhat(const BView &b, const CurveDev &cv, int32_t j, double z[3]) {
  double tiny = rn_mul(rn_mul(0.1, b.v.h), b.v.h);
  zraw(b, cv, j, z);
  if (rn_norm3(z) >= tiny) return;
  double y[3] = {b.cp[3 * j], b.cp[3 * j + 1], b.cp[3 * j + 2]};
  int base[3];
  double t[3];
  cpm_stencil_of(b.v.dim, b.v.h, b.v.np1, y, base, t);
  const int np1 = b.v.np1, nz = (b.v.dim == 3) ? np1 : 1;
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < np1; ++cy)
      for (int cx = 0; cx < np1; ++cx) {
        int32_t q = lookup_near(b, j, base[0] + cx, base[1] + cy, (b.v.dim == 3) ? base[2] + cz : 0);
        if (q < 0) continue;
        double w[3];
        zraw(b, cv, q, w);
        if (rn_norm3(w) >= tiny) { z[0] = w[0]; z[1] = w[1]; z[2] = w[2]; return; }
      }
  z[0] = z[1] = z[2] = 0.0;
}

// distance of every node to every curve: zone (< 2r) and Omega(C) (<= r)
__global__ void near_kernel(BView b, int8_t *near, int8_t *inC, int32_t *count_per_curve, unsigned *err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b.v.NS; i += (int64_t)gridDim.x * blockDim.x) {
    double x[3];
    node_coords(b, (int32_t)i, x);
    int nzone = 0;
    int8_t nr = -1, ic = -1;
    double two_r = rn_mul(2.0, b.v.rband);
    for (int k = 0; k < b.ncurves; ++k) {
      double cc[3];
      cpm_cp_C(b.curves[k], x, cc);
      double d[3] = {rn_sub(x[0], cc[0]), rn_sub(x[1], cc[1]), rn_sub(x[2], cc[2])};
      double dC = rn_norm3(d);
      if (dC < two_r) { nzone++; nr = (int8_t)k; }
      if (dC <= b.v.rband) ic = (int8_t)k;
    }
    if (nzone > 1) atomicOr(err, CPM_DEVERR_OVERLAP);
    near[i] = nr;
    inC[i] = ic;
    if (ic >= 0) atomicAdd(count_per_curve + ic, 1);
  }
}

__global__ void flag_eq_kernel(const int8_t *arr, int64_t n, int8_t val, int32_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (arr[i] == val) ? 1 : 0;
}

__global__ void flag_ge0_kernel(const int8_t *arr, int64_t n, int32_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (arr[i] >= 0) ? 1 : 0;
}

__global__ void assign_bc_kernel(const int8_t *inC, int8_t k, const int32_t *pos, int64_t NS, int64_t off,
                                 int32_t *bc_of, int32_t *twin, int32_t *bc_curve) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NS; i += (int64_t)gridDim.x * blockDim.x)
    if (inC[i] == k) {
      int64_t a = off + pos[i];
      bc_of[i] = (int32_t)(NS + a);
      twin[a] = (int32_t)i;
      bc_curve[a] = k;
    }
}

__global__ void assign_spec_kernel(const int8_t *near, const int32_t *pos, int64_t NS, int32_t *spec_row,
                                   int32_t *spec_of, uint32_t *rbase) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NS; i += (int64_t)gridDim.x * blockDim.x) {
    if (near[i] >= 0) {
      spec_row[pos[i]] = (int32_t)i;
      spec_of[i] = pos[i];
      rbase[i] |= CPM_SPECIAL_BIT;
    } else {
      spec_of[i] = -1;
      rbase[i] &= ~CPM_SPECIAL_BIT;
    }
  }
}

// per BC DOF: cp_C, side of cp_S (sign of zhat . nu; none for a point in 3D),
// angle, and the row's BC type (that of the opposite side)
__global__ void bc_info_kernel(BView b, const int32_t *twin, const int32_t *bc_curve, int64_t NC, double *cpc,
                               int32_t *side, double *param, int32_t *type) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < NC; a += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = twin[a];
    const CurveDev &cv = b.curves[bc_curve[a]];
    double x[3], cc[3], z[3];
    node_coords(b, j, x);
    cpm_cp_C(cv, x, cc);
    cpc[3 * a] = cc[0]; cpc[3 * a + 1] = cc[1]; cpc[3 * a + 2] = cc[2];
    zhat(b, cv, j, z);
    double s = rn_dot3(z, cv.nu);
    side[a] = (cv.kind == CPM_CURVE_POINT && b.v.dim == 3) ? 0 : ((s > 0.0) - (s < 0.0));
    type[a] = (side[a] > 0) ? cv.bc_minus : cv.bc;
    double ang = 0.0;
    if (cv.kind == CPM_CURVE_CIRCLE) {
      double q[3] = {cc[0] - cv.p[0], cc[1] - cv.p[1], cc[2] - cv.p[2]};
      double e2[3] = {cv.nu[1] * cv.ref[2] - cv.nu[2] * cv.ref[1], cv.nu[2] * cv.ref[0] - cv.nu[0] * cv.ref[2],
                      cv.nu[0] * cv.ref[1] - cv.nu[1] * cv.ref[0]};
      ang = atan2(q[0] * e2[0] + q[1] * e2[1] + q[2] * e2[2], q[0] * cv.ref[0] + q[1] * cv.ref[1] + q[2] * cv.ref[2]);
      const double two_pi = 6.283185307179586476925286766559;
      ang = fmod(ang, two_pi);
      if (ang < 0) ang += two_pi;
      if (ang >= two_pi) ang -= two_pi;
    }
    param[a] = ang;
  }
}

// column of stencil node j for a special PDE row (Eq. 10)
__device__ __forceinline__ int32_t pde_col(const BView &b, const CurveDev &cv, int k, const double *dstar, int32_t j,
                                           const int32_t *bc_of, const int32_t *bc_curve,
                                           unsigned long long *noflip) {
  double z[3];
  zhat(b, cv, j, z);
  if (rn_dot3(dstar, z) < 0.0) {
    int32_t a = bc_of[j];
    if (a >= 0 && bc_curve[a - b.v.NS] == k) return a;
    atomicAdd(noflip, 1ull);
  }
  return j;
}

// explicit stencils of the special rows (one thread per row)
__global__ void spec_stencil_kernel(BView b, const int32_t *spec_row, int64_t nspec, const int8_t *near,
                                    const int32_t *bc_of, const int32_t *bc_curve, int32_t *ecol, double *ew,
                                    float *ew32, int32_t *fcol, unsigned long long *noflip, unsigned *err) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nspec; s += (int64_t)gridDim.x * blockDim.x) {
    int32_t i = spec_row[s];
    int k = near[i];
    const CurveDev &cv = b.curves[k];
    double dstar[3];
    zhat(b, cv, i, dstar);
    double y[3] = {b.cp[3 * i], b.cp[3 * i + 1], b.cp[3 * i + 2]};
    int base[3];
    double t[3], w[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {1, 0, 0, 0}};
    const int np1 = b.v.np1;
    cpm_stencil_of(b.v.dim, b.v.h, np1, y, base, t);
    for (int a = 0; a < b.v.dim; ++a) cpm_lagrange_rt<double>(np1, t[a], w[a]);
    // explicit stencil in the fixed 4 x 4 x 4 layout; entries outside the
    // np1^dim stencil are absent (-1)
    int e = 0;
    for (int cz = 0; cz < 4; ++cz)
      for (int cy = 0; cy < 4; ++cy)
        for (int cx = 0; cx < 4; ++cx, ++e) {
          if (!cpm_in_stencil(e, np1, b.v.dim)) {
            ecol[s * 64 + e] = -1; ew[s * 64 + e] = 0.0; ew32[s * 64 + e] = 0.0f;
            continue;
          }
          int32_t j = lookup_near(b, i, base[0] + cx, base[1] + cy, (b.v.dim == 3) ? base[2] + cz : 0);
          if (j < 0) { atomicOr(err, CPM_DEVERR_MISSING_NODE); j = i; }
          double wt = w[0][cx] * w[1][cy] * w[2][cz];
          ecol[s * 64 + e] = pde_col(b, cv, k, dstar, j, bc_of, bc_curve, noflip);
          ew[s * 64 + e] = wt;
          ew32[s * 64 + e] = (float)wt;
        }
    int gi = b.ijk[3 * i], gj = b.ijk[3 * i + 1], gk = b.ijk[3 * i + 2];
    for (int a = 0; a < 3; ++a)
      for (int sg = 0; sg < 2; ++sg) {
        int slot = 2 * a + sg;
        if (a >= b.v.dim) { fcol[s * 6 + slot] = -1; continue; }
        int d[3] = {0, 0, 0};
        d[a] = sg ? 1 : -1;
        int32_t j = lookup_near(b, i, gi + d[0], gj + d[1], gk + d[2]);
        fcol[s * 6 + slot] = (j < 0) ? -1 : pde_col(b, cv, k, dstar, j, bc_of, bc_curve, noflip);
      }
  }
}

// BC rows
__global__ void bc_rows_kernel(BView b, const int32_t *twin, const int32_t *bc_curve, const int32_t *type,
                               const double *cpc, int64_t NC, const int32_t *bc_of, int32_t *cnt, int32_t *col,
                               double *val, float *val32, unsigned *err) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < NC; a += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = twin[a];
    int k = bc_curve[a];
    const CurveDev &cv = b.curves[k];
    int64_t o = a * CPM_BC_STRIDE;
    col[o] = (int32_t)(b.v.NS + a);
    val[o] = 1.0;
    val32[o] = 1.0f;
    const int ty = type[a];
    if (ty == CPM_BC_DIR1) { cnt[a] = 1; continue; }
    double dstar[3], x[3], yv[3], cpb[3];
    zhat(b, cv, j, dstar);
    if (ty == CPM_BC_NEU1) {
      // first-order Neumann: the query point is cp_C(x_alpha) itself
      for (int e = 0; e < 3; ++e) cpb[e] = cpc[3 * a + e];
    } else {
      node_coords(b, j, x);
      for (int e = 0; e < 3; ++e) yv[e] = rn_sub(rn_mul(2.0, cpc[3 * a + e]), x[e]);
      if (cpm_cp_S(b.shape, yv, cpb)) { atomicOr(err, CPM_DEVERR_CP); cnt[a] = 1; continue; }
    }
    const double sgn = (ty == CPM_BC_DIR2) ? 1.0 : -1.0;
    int base[3];
    double t[3], w[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {1, 0, 0, 0}};
    const int np1 = b.v.np1;
    cpm_stencil_of(b.v.dim, b.v.h, np1, cpb, base, t);
    for (int e = 0; e < b.v.dim; ++e) cpm_lagrange_rt<double>(np1, t[e], w[e]);
    int nz = (b.v.dim == 3) ? np1 : 1, n = 1;
    for (int cz = 0; cz < nz; ++cz)
      for (int cy = 0; cy < np1; ++cy)
        for (int cx = 0; cx < np1; ++cx) {
          int32_t q = lookup_near(b, j, base[0] + cx, base[1] + cy, (b.v.dim == 3) ? base[2] + cz : 0);
          if (q < 0) { atomicOr(err, CPM_DEVERR_MISSING_NODE); continue; }
          double z[3];
          zhat(b, cv, q, z);
          int32_t c = q;
          if (!(rn_dot3(dstar, z) < 0.0)) {
            int32_t t2 = bc_of[q];
            if (t2 >= 0 && bc_curve[t2 - b.v.NS] == k) c = t2;
          }
          double wt = sgn * (w[0][cx] * w[1][cy] * w[2][cz]);
          col[o + n] = c;
          val[o + n] = wt;
          val32[o + n] = (float)wt;
          ++n;
        }
    cnt[a] = n;
  }
}

}  // namespace

void cpm_free_boundary(cpm_ctx *c) {
  cudaFree(c->d_curves); cudaFree(c->d_bc_of); cudaFree(c->d_near); cudaFree(c->d_twin); cudaFree(c->d_bc_curve);
  cudaFree(c->d_cpc); cudaFree(c->d_side); cudaFree(c->d_param); cudaFree(c->d_bc_cnt); cudaFree(c->d_bc_col);
  cudaFree(c->d_bc_type);
  c->d_bc_type = nullptr;
  cudaFree(c->d_bc_val); cudaFree(c->d_bc_val32); cudaFree(c->d_spec_row); cudaFree(c->d_spec_of);
  cudaFree(c->d_curve_first);
  c->d_curve_first = nullptr;
  cudaFree(c->d_spec_ecol); cudaFree(c->d_spec_ew); cudaFree(c->d_spec_ew32); cudaFree(c->d_spec_fcol);
  cpm_free_cells(c);
  cudaFree(c->d_T_ptr); cudaFree(c->d_T_row); cudaFree(c->d_cellid); cudaFree(c->d_w1d64); cudaFree(c->d_w1d32);
  cudaFree(c->d_tblk);
  c->d_tblk = nullptr;
  cudaFree(c->d_T_kind); cudaFree(c->d_T_val); cudaFree(c->d_T_val32);
  delete[] c->h_curves;
  c->h_curves = nullptr;
  c->d_curves = nullptr; c->d_bc_of = nullptr; c->d_near = nullptr; c->d_twin = nullptr; c->d_bc_curve = nullptr;
  c->d_cpc = nullptr; c->d_side = nullptr; c->d_param = nullptr; c->d_bc_cnt = nullptr; c->d_bc_col = nullptr;
  c->d_bc_val = nullptr; c->d_bc_val32 = nullptr; c->d_spec_row = nullptr; c->d_spec_of = nullptr;
  c->d_spec_ecol = nullptr; c->d_spec_ew = nullptr; c->d_spec_ew32 = nullptr; c->d_spec_fcol = nullptr;
  c->d_T_ptr = nullptr; c->d_T_row = nullptr; c->d_cellid = nullptr; c->nT = 0; c->d_w1d64 = nullptr; c->d_w1d32 = nullptr;
  c->d_T_kind = nullptr; c->d_T_val = nullptr; c->d_T_val32 = nullptr;
  c->transpose_ready = false;
  c->boundary_set = false;
  c->NC = 0; c->nspec = 0; c->ncurves = 0; c->nsamples_total = 0; c->nT = 0;
}

cpm_status cpm_internal_set_boundary(cpm_ctx *c, const cpm_curve_desc *curves, int n) {
  cudaStream_t st = c->stream;
  cpm_free_boundary(c);
  c->ncurves = n;
  c->h_curves = new CurveDev[n > 0 ? n : 1];
  int64_t off = 0;
  for (int k = 0; k < n; ++k) {
    CurveDev &d = c->h_curves[k];
    const cpm_curve_desc &s = curves[k];
    d.kind = s.kind; d.bc = s.bc; d.two_sided = s.two_sided; d.n_samples = s.n_samples;
    d.bc_minus = s.bc_minus ? s.bc_minus : s.bc;
    d.projected = s.projected ? 1 : 0;
    for (int e = 0; e < 3; ++e) { d.p[e] = s.p[e]; d.nu[e] = s.nu[e]; d.ref[e] = s.ref[e]; }
    d.rad = s.rad;
    d.sample_off = off;
    off += (int64_t)s.n_samples * (s.two_sided ? 2 : 1);
  }
  c->nsamples_total = off;
  int8_t *inC = nullptr;
  int32_t *flag = nullptr, *pos = nullptr, *cnt = nullptr, *d_total = nullptr;
  cpm_status rc = CPM_OK;
  unsigned h_err = 0;
  unsigned long long h_noflip = 0;
  int32_t h_total = 0;
  std::vector<int32_t> counts(n > 0 ? n : 1, 0);
  BView b;
#define TRY(x)                                             \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_) { rc = cpm_internal_cuda_err(e_); goto done; } \
  } while (0)
  TRY(cudaMalloc(&c->d_curves, sizeof(CurveDev) * (n > 0 ? n : 1)));
  if (n > 0) TRY(cudaMemcpyAsync(c->d_curves, c->h_curves, sizeof(CurveDev) * n, cudaMemcpyHostToDevice, st));
  TRY(cudaMalloc(&c->d_near, c->NS));
  TRY(cudaMalloc(&inC, c->NS));
  TRY(cudaMalloc(&c->d_bc_of, sizeof(int32_t) * c->NS));
  TRY(cudaMalloc(&c->d_spec_of, sizeof(int32_t) * c->NS));
  TRY(cudaMalloc(&flag, sizeof(int32_t) * c->NS));
  TRY(cudaMalloc(&pos, sizeof(int32_t) * c->NS));
  TRY(cudaMalloc(&cnt, sizeof(int32_t) * (n > 0 ? n : 1)));
  TRY(cudaMalloc(&d_total, sizeof(int32_t)));
  TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n > 0 ? n : 1), st));
  TRY(cudaMemsetAsync(c->d_bc_of, 0xFF, sizeof(int32_t) * c->NS, st));
  TRY(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), st));
  TRY(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long) * 4, st));
  b.v = c->view();
  b.shape = c->shape;
  b.ijk = c->d_ijk;
  b.cp = c->d_cp;
  b.rself = c->d_rself;
  b.curves = c->d_curves;
  b.ncurves = n;
  near_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(b, c->d_near, inC, cnt, c->d_err);
  if (n > 0) TRY(cudaMemcpyAsync(counts.data(), cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  if (h_err & CPM_DEVERR_OVERLAP) { rc = CPM_ERR_OVERLAP; goto done; }
  c->NC = 0;
  for (int k = 0; k < n; ++k) c->NC += counts[k];
  b.v.NC = c->NC;
  {
    // first BC DOF of each curve (BC DOFs are numbered curve by curve)
    std::vector<int32_t> first(n + 1, 0);
    for (int k = 0; k < n; ++k) first[k + 1] = first[k] + counts[k];
    TRY(cudaMalloc(&c->d_curve_first, sizeof(int32_t) * (n + 1)));
    TRY(cudaMemcpyAsync(c->d_curve_first, first.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
    TRY(cudaStreamSynchronize(st));
  }
  {
    int64_t nc1 = c->NC > 0 ? c->NC : 1;
    TRY(cudaMalloc(&c->d_twin, sizeof(int32_t) * nc1));
    TRY(cudaMalloc(&c->d_bc_curve, sizeof(int32_t) * nc1));
    TRY(cudaMalloc(&c->d_cpc, sizeof(double) * 3 * nc1));
    TRY(cudaMalloc(&c->d_side, sizeof(int32_t) * nc1));
    TRY(cudaMalloc(&c->d_bc_type, sizeof(int32_t) * nc1));
    TRY(cudaMalloc(&c->d_param, sizeof(double) * nc1));
    TRY(cudaMalloc(&c->d_bc_cnt, sizeof(int32_t) * nc1));
    TRY(cudaMalloc(&c->d_bc_col, sizeof(int32_t) * CPM_BC_STRIDE * nc1));
    TRY(cudaMalloc(&c->d_bc_val, sizeof(double) * CPM_BC_STRIDE * nc1));
    TRY(cudaMalloc(&c->d_bc_val32, sizeof(float) * CPM_BC_STRIDE * nc1));
    int64_t boff = 0;
    for (int k = 0; k < n; ++k) {
      flag_eq_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(inC, c->NS, (int8_t)k, flag);
      TRY(cpm_exclusive_scan(flag, pos, c->NS, nullptr, st));
      assign_bc_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(inC, (int8_t)k, pos, c->NS, boff, c->d_bc_of, c->d_twin,
                                                           c->d_bc_curve);
      boff += counts[k];
    }
    // special rows: all rows within 2 r of a curve
    flag_ge0_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(c->d_near, c->NS, flag);
    TRY(cpm_exclusive_scan(flag, pos, c->NS, d_total, st));
    TRY(cudaMemcpyAsync(&h_total, d_total, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    c->nspec = h_total;
    int64_t ns1 = c->nspec > 0 ? c->nspec : 1;
    TRY(cudaMalloc(&c->d_spec_row, sizeof(int32_t) * ns1));
    TRY(cudaMalloc(&c->d_spec_ecol, sizeof(int32_t) * 64 * ns1));
    TRY(cudaMalloc(&c->d_spec_ew, sizeof(double) * 64 * ns1));
    TRY(cudaMalloc(&c->d_spec_ew32, sizeof(float) * 64 * ns1));
    TRY(cudaMalloc(&c->d_spec_fcol, sizeof(int32_t) * 6 * ns1));
    assign_spec_kernel<<<cpm_grid(c->NS, 256), 256, 0, st>>>(c->d_near, pos, c->NS, c->d_spec_row, c->d_spec_of,
                                                             c->d_rbase);
    if (c->NC > 0)
      bc_info_kernel<<<cpm_grid(c->NC, 128), 128, 0, st>>>(b, c->d_twin, c->d_bc_curve, c->NC, c->d_cpc, c->d_side,
                                                           c->d_param, c->d_bc_type);
    if (c->nspec > 0)
      spec_stencil_kernel<<<cpm_grid(c->nspec, 64), 64, 0, st>>>(b, c->d_spec_row, c->nspec, c->d_near, c->d_bc_of,
                                                                 c->d_bc_curve, c->d_spec_ecol, c->d_spec_ew,
                                                                 c->d_spec_ew32, c->d_spec_fcol, c->d_counter,
                                                                 c->d_err);
    if (c->NC > 0)
      bc_rows_kernel<<<cpm_grid(c->NC, 64), 64, 0, st>>>(b, c->d_twin, c->d_bc_curve, c->d_bc_type, c->d_cpc, c->NC,
                                                         c->d_bc_of,
                                                         c->d_bc_cnt, c->d_bc_col, c->d_bc_val, c->d_bc_val32,
                                                         c->d_err);
    TRY(cudaGetLastError());
    TRY(cudaMemcpyAsync(&h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(&h_noflip, c->d_counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    c->noflip_twin = (int64_t)h_noflip;
    if (h_err & CPM_DEVERR_CP) { rc = CPM_ERR_CP_FAILED; goto done; }
    if (h_err & CPM_DEVERR_MISSING_NODE) { rc = CPM_ERR_STATE; goto done; }
  }
done:
#undef TRY
  cudaStreamSynchronize(st);
  cudaFree(inC); cudaFree(flag); cudaFree(pos); cudaFree(cnt); cudaFree(d_total);
  if (rc != CPM_OK) {
    cpm_free_boundary(c);
    return rc;
  }
  rc = cpm_build_cells(c);
  if (rc != CPM_OK) {
    cpm_free_boundary(c);
    return rc;
  }
  rc = cpm_build_transpose(c);
  if (rc != CPM_OK) {
    cpm_free_boundary(c);
    return rc;
  }
  c->boundary_set = true;
  return CPM_OK;
}
