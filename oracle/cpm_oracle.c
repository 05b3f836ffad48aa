/*
 * cpm_oracle.c -- plain, slow FP64 CPU reference of the closest point method
 * (CPM) with interior boundary conditions (IBCs).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only tests/, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code with the CUDA library.
 *
 * Every function restates one passage of King, Su, Aanjaneya, Ruuth, Batty,
 * "A Closest Point Method for PDEs on Manifolds with Interior Boundary
 * Conditions for Geometry Processing" (ACM TOG 2024):
 *   - closest points: Sec. 3.1 and App. A (analytic shapes, level-set Newton)
 *   - tube radius, Eq. (3) "bandwidth"; band Omega(S) and BFS, Alg. 1, Sec. 5.1
 *   - barycentric Lagrange interpolation (E), Eq. (1); FD Laplacian (L), Eq. (2)
 *   - BC DOFs Omega(C), Sec. 4.1; crossing test Eqs. (8)-(9), Sec. 4.2
 *   - stencil modification Eqs. (10)-(11), Sec. 4.3; Dirichlet and zero-Neumann
 *     IBC rows of first and second order, with a BC type per side, Sec. 4.3
 *   - interpolation degree p = 3 (cubic) or p = 2 (quadratic, Sec. 7), Eq. (3)
 *   - localisation 2 r_Omega, Sec. 4.6
 *   - M = diag(L) + (L - diag L) E, Sec. 5.3; A = mI + nM and the four-step
 *     partially matrix-free product, Sec. 5.4; diagonal-preconditioned BiCGSTAB
 *
 * Readings of points the paper leaves open (the BC-row algebra, DOF order,
 * tie handling, missing FD neighbours) are listed in the project's design notes;
 * the ones that shape code here are repeated next to that code.
 *
 * Precision: FP64 throughout, compiled with -ffp-contract=off so that every
 * product and sum is rounded separately in the order written.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_CP 3
#define ORC_ERR_OVERLAP 4
#define ORC_ERR_STATE 5
#define ORC_ERR_BREAKDOWN 6
#define ORC_ERR_NOT_CONVERGED 7

enum { SH_CIRCLE = 1, SH_SPHERE = 2, SH_TORUS = 3, SH_BUMPY = 4 };
enum { CV_POINT = 1, CV_CIRCLE = 2 };
enum { BC_DIR1 = 1, BC_DIR2 = 2, BC_NEU1 = 3, BC_NEU2 = 4 };

typedef struct {
  int kind;      /* SH_* */
  int dim;       /* 2 (circle) or 3 */
  double R;      /* circle/sphere radius; torus major radius */
  double rt;     /* torus minor radius */
  int K;         /* bumpy sphere: number of bumps */
  double amp;    /* bumpy sphere: rho(w) = 1 + amp * sum_k a_k exp(-|w - c_k|^2 / width) */
  double width;
  const double *a; /* [K] */
  const double *c; /* [3K], unit vectors */
  double seed[3];  /* a surface point used to seed the BFS */
} orc_shape;

typedef struct {
  int kind;          /* CV_POINT or CV_CIRCLE */
  int bc;            /* BC_DIR1 or BC_DIR2 */
  double p[3];       /* point, or circle centre */
  double nu[3];      /* circle: unit normal of its plane; point in 2D: unit tangent of S
                        at the point (orients the two sides); point in 3D: unused */
  double rad;        /* circle radius */
  double ref[3];     /* circle: unit reference direction in its plane (angle 0) */
  int two_sided;     /* 0: one value set for both sides; 1: separate sets per side */
  int bc_minus;      /* BC type on the minus side (0: the same as bc, which is the plus side's) */
  int projected;     /* 1: projected crossing test of Sec. 4.7 (components along n_S and t_C removed) */
} orc_curve;

/* ------------------------------------------------------------------ */
/* small vector helpers (no contraction; written out in a fixed order) */
static double dot3(const double *a, const double *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------ */
/* Closest point to S (Sec. 3.1; App. A).  Returns 0 on success.      */

/* bumpy sphere level set phi(x) = |x| - rho(x/|x|) with gradient and Hessian
 * (App. A: analytic expressions for grad phi and D^2 phi).  With s = |x|,
 * u = x/s, P = I - u u^T, g = grad_u rho, H = Hess_u rho, q = P g:
 *   grad phi = u - q / s
 *   D^2 phi  = P/s - [P H P - u q^T - q u^T - (u.g) P] / s^2            */
static void bumpy_phi(const orc_shape *sh, const double *x, double *phi, double grad[3], double hess[9]) {
  double s = norm3(x);
  double u[3] = {x[0] / s, x[1] / s, x[2] / s};
  double rho = 1.0, g[3] = {0, 0, 0}, H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < sh->K; ++k) {
    const double *ck = sh->c + 3 * k;
    double d[3] = {u[0] - ck[0], u[1] - ck[1], u[2] - ck[2]};
    double e = exp(-dot3(d, d) / sh->width);
    double coef = sh->amp * sh->a[k] * e;
    rho += coef;
    for (int i = 0; i < 3; ++i) g[i] += coef * (-2.0 * d[i] / sh->width);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        H[3 * i + j] += coef * ((4.0 / (sh->width * sh->width)) * d[i] * d[j] - (i == j ? 2.0 / sh->width : 0.0));
  }
  *phi = s - rho;
  double P[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[3 * i + j] = (i == j ? 1.0 : 0.0) - u[i] * u[j];
  double q[3];
  for (int i = 0; i < 3; ++i) q[i] = (P[3 * i + 0] * g[0] + P[3 * i + 1] * g[1]) + P[3 * i + 2] * g[2];
  for (int i = 0; i < 3; ++i) grad[i] = u[i] - q[i] / s;
  if (!hess) return;
  double ug = dot3(u, g);
  double PH[9], PHP[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) PH[3 * i + j] = (P[3 * i + 0] * H[0 + j] + P[3 * i + 1] * H[3 + j]) + P[3 * i + 2] * H[6 + j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) PHP[3 * i + j] = (PH[3 * i + 0] * P[0 + j] + PH[3 * i + 1] * P[3 + j]) + PH[3 * i + 2] * P[6 + j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      hess[3 * i + j] = P[3 * i + j] / s - (PHP[3 * i + j] - u[i] * q[j] - q[i] * u[j] - ug * P[3 * i + j]) / (s * s);
}

/* solve a 4x4 system by Gaussian elimination with partial pivoting */
static int solve4(double A[16], double b[4], double x[4]) {
  int piv[4] = {0, 1, 2, 3};
  for (int c = 0; c < 4; ++c) {
    int best = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(A[4 * piv[r] + c]) > fabs(A[4 * piv[best] + c])) best = r;
    int t = piv[c]; piv[c] = piv[best]; piv[best] = t;
    double d = A[4 * piv[c] + c];
    if (d == 0.0) return 1;
    for (int r = c + 1; r < 4; ++r) {
      double f = A[4 * piv[r] + c] / d;
      for (int k = c; k < 4; ++k) A[4 * piv[r] + k] -= f * A[4 * piv[c] + k];
      b[piv[r]] -= f * b[piv[c]];
    }
  }
  for (int c = 3; c >= 0; --c) {
    double s = b[piv[c]];
    for (int k = c + 1; k < 4; ++k) s -= A[4 * piv[c] + k] * x[k];
    x[c] = s / A[4 * piv[c] + c];
  }
  return 0;
}

/* App. A: a gradient-projection start cp <- cp - phi grad/|grad|^2 until the step
 * is below 1e-10, then Newton on f(cp, lam) = 1/2|cp - x|^2 + lam phi(cp) until
 * |dy| < 1e-10, with lam_0 = (x - cp*).grad/|grad|^2.  Iteration caps: 200. */
static int cp_bumpy(const orc_shape *sh, const double *x, double *cp) {
  double y[3] = {x[0], x[1], x[2]}, phi, gr[3], H[9];
  int it;
  for (it = 0; it < 200; ++it) {
    bumpy_phi(sh, y, &phi, gr, NULL);
    double g2 = dot3(gr, gr);
    double st[3] = {phi * gr[0] / g2, phi * gr[1] / g2, phi * gr[2] / g2};
    for (int i = 0; i < 3; ++i) y[i] -= st[i];
    if (norm3(st) < 1e-10) break;
  }
  if (it == 200) return ORC_ERR_CP;
  bumpy_phi(sh, y, &phi, gr, NULL);
  double d0[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double lam = dot3(d0, gr) / dot3(gr, gr);
  for (it = 0; it < 200; ++it) {
    bumpy_phi(sh, y, &phi, gr, H);
    double J[16], F[4], dy[4];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) J[4 * i + j] = (i == j ? 1.0 : 0.0) + lam * H[3 * i + j];
      J[4 * i + 3] = gr[i];
      J[12 + i] = gr[i];
      F[i] = (y[i] - x[i]) + lam * gr[i];
    }
    J[15] = 0.0;
    F[3] = phi;
    if (solve4(J, F, dy)) return ORC_ERR_CP;
    for (int i = 0; i < 3; ++i) y[i] -= dy[i];
    lam -= dy[3];
    double ny = sqrt(((dy[0] * dy[0] + dy[1] * dy[1]) + dy[2] * dy[2]) + dy[3] * dy[3]);
    if (ny < 1e-10) break;
  }
  if (it == 200) return ORC_ERR_CP;
  cp[0] = y[0]; cp[1] = y[1]; cp[2] = y[2];
  return 0;
}

/* cp_S for the analytic shapes, written as the closed forms of Sec. 3.1 / App. A.
 * Circle/sphere: cp = R (x/|x|).  Torus (axis z): c = R (x,y,0)/|(x,y)|, then
 * cp = c + rt (x - c)/|x - c|.  x is 2D for the circle (x[2] ignored, cp[2]=0).
 * On the medial axis (x = 0; the torus axis; the torus's centre circle) every
 * choice is equally close; a fixed one is taken (direction +x, resp. +z), which
 * keeps the distance, the only thing the band needs there, exact. */
static int cp_S(const orc_shape *sh, const double *x, double *cp) {
  if (sh->kind == SH_CIRCLE) {
    double n = sqrt(x[0] * x[0] + x[1] * x[1]);
    if (n == 0.0) { cp[0] = sh->R; cp[1] = 0.0; cp[2] = 0.0; return 0; }
    cp[0] = sh->R * (x[0] / n); cp[1] = sh->R * (x[1] / n); cp[2] = 0.0;
    return 0;
  }
  if (sh->kind == SH_SPHERE) {
    double n = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    if (n == 0.0) { cp[0] = sh->R; cp[1] = 0.0; cp[2] = 0.0; return 0; }
    cp[0] = sh->R * (x[0] / n); cp[1] = sh->R * (x[1] / n); cp[2] = sh->R * (x[2] / n);
    return 0;
  }
  if (sh->kind == SH_TORUS) {
    double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
    double ux = 1.0, uy = 0.0;
    if (rho != 0.0) { ux = x[0] / rho; uy = x[1] / rho; }
    double cx = sh->R * ux, cy = sh->R * uy;
    double dx = x[0] - cx, dy = x[1] - cy, dz = x[2];
    double m = sqrt((dx * dx + dy * dy) + dz * dz);
    if (m == 0.0) { cp[0] = cx; cp[1] = cy; cp[2] = sh->rt; return 0; }
    cp[0] = cx + sh->rt * (dx / m); cp[1] = cy + sh->rt * (dy / m); cp[2] = sh->rt * (dz / m);
    return 0;
  }
  if (sh->kind == SH_BUMPY) return cp_bumpy(sh, x, cp);
  return ORC_ERR_ARG;
}

/* cp to an interior boundary C: a point, or a circle (centre p, unit normal nu,
 * radius rad): cp = p + rad * unit((x - p) - ((x - p).nu) nu). */
static void cp_C(const orc_curve *cv, const double *x, double *out) {
  if (cv->kind == CV_POINT) { out[0] = cv->p[0]; out[1] = cv->p[1]; out[2] = cv->p[2]; return; }
  double w[3] = {x[0] - cv->p[0], x[1] - cv->p[1], x[2] - cv->p[2]};
  double s = dot3(w, cv->nu);
  double q[3] = {w[0] - s * cv->nu[0], w[1] - s * cv->nu[1], w[2] - s * cv->nu[2]};
  double nq = norm3(q);
  if (nq == 0.0) { q[0] = cv->ref[0]; q[1] = cv->ref[1]; q[2] = cv->ref[2]; nq = 1.0; }
  out[0] = cv->p[0] + cv->rad * (q[0] / nq);
  out[1] = cv->p[1] + cv->rad * (q[1] / nq);
  out[2] = cv->p[2] + cv->rad * (q[2] / nq);
}

/* ------------------------------------------------------------------ */
/* Integer grid nodes, a hash set/map over them, and the canonical order */

#define KOFF (1LL << 20)
static int64_t node_key(int i, int j, int k) {
  return (((int64_t)i + KOFF) << 42) | (((int64_t)j + KOFF) << 21) | ((int64_t)k + KOFF);
}
static int floordiv8(int v) { return (v >= 0) ? v / 8 : -((-v + 7) / 8); }
/* canonical DOF order: 8^3 bricks ordered by (bz, by, bx), nodes inside a brick
 * by (lz, ly, lx) -- a reading, since the paper fixes no order */
static int64_t canon_key(const int *ijk) {
  int b[3], l[3];
  for (int a = 0; a < 3; ++a) { b[a] = floordiv8(ijk[a]); l[a] = ijk[a] - 8 * b[a]; }
  const int64_t o = 1LL << 17;
  return (((int64_t)b[2] + o) << 45) | (((int64_t)b[1] + o) << 27) | (((int64_t)b[0] + o) << 9) |
         (int64_t)(l[2] * 64 + l[1] * 8 + l[0]);
}

typedef struct { int64_t *keys; int64_t *vals; int64_t cap; int64_t n; } hmap;
static uint64_t hmix(uint64_t k) {
  k ^= k >> 33; k *= 0xff51afd7ed558ccdULL; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ULL; k ^= k >> 33;
  return k;
}
static int hm_init(hmap *m, int64_t cap) {
  int64_t c = 1024;
  while (c < 2 * cap) c <<= 1;
  m->cap = c; m->n = 0;
  m->keys = (int64_t *)malloc(sizeof(int64_t) * c);
  m->vals = (int64_t *)malloc(sizeof(int64_t) * c);
  if (!m->keys || !m->vals) return ORC_ERR_OOM;
  for (int64_t i = 0; i < c; ++i) m->keys[i] = -1;
  return 0;
}
static void hm_free(hmap *m) { free(m->keys); free(m->vals); m->keys = m->vals = NULL; }
static int hm_grow(hmap *m);
static int64_t *hm_slot(hmap *m, int64_t key, int insert) {
  uint64_t mask = (uint64_t)m->cap - 1, p = hmix((uint64_t)key) & mask;
  for (;;) {
    if (m->keys[p] == key) return &m->vals[p];
    if (m->keys[p] == -1) {
      if (!insert) return NULL;
      if (2 * (m->n + 1) > m->cap) { if (hm_grow(m)) return NULL; return hm_slot(m, key, insert); }
      m->keys[p] = key; m->vals[p] = -1; m->n++;
      return &m->vals[p];
    }
    p = (p + 1) & mask;
  }
}
static int hm_grow(hmap *m) {
  hmap g;
  if (hm_init(&g, m->cap)) return ORC_ERR_OOM;
  for (int64_t i = 0; i < m->cap; ++i)
    if (m->keys[i] != -1) *hm_slot(&g, m->keys[i], 1) = m->vals[i];
  hm_free(m);
  *m = g;
  return 0;
}
static int64_t hm_get(const hmap *m, int64_t key) {
  uint64_t mask = (uint64_t)m->cap - 1, p = hmix((uint64_t)key) & mask;
  for (;;) {
    if (m->keys[p] == key) return m->vals[p];
    if (m->keys[p] == -1) return -1;
    p = (p + 1) & mask;
  }
}

/* ------------------------------------------------------------------ */
/* Context                                                              */

typedef struct {
  int64_t *ptr; int64_t *col; double *val; int64_t nrows, nnz, cap;
} csr;

typedef struct orc_ctx {
  orc_shape sh;
  double *sh_a, *sh_c;
  int dim;
  int p;         /* interpolation degree (3 or 2); p + 1 stencil nodes per axis */
  double h, rband;
  int64_t NS, NC;
  int32_t *ijk;  /* [NS*3] */
  double *cp;    /* [NS*3] */
  hmap index;    /* node key -> PDE index */
  /* boundary */
  int ncurves;
  orc_curve *curves;
  int64_t *bc_of;     /* [NS]: BC DOF alpha at this node (any curve) or -1 */
  int32_t *near_c;    /* [NS]: curve whose 2 r_Omega zone holds the node, or -1 */
  int64_t *twin;      /* [NC]: PDE index of each BC DOF */
  int32_t *bc_curve;  /* [NC] */
  double *cpc;        /* [NC*3]: cp_C(x_alpha) */
  int32_t *bc_side;   /* [NC]: +1/-1/0: side of S_perp holding cp_S(x_alpha) */
  int32_t *bc_type;   /* [NC]: BC type of the row: that of the side opposite cp_S(x_alpha) */
  int64_t n_noflip_twin; /* diagnostics: flip requested but no twin existed */
  /* operator */
  csr E;      /* N_S rows (PDE DOFs) x N columns: interpolation with flips */
  csr Loff;   /* N_S rows x N columns: off-diagonal FD weights with flips */
  csr B;      /* N_C rows x N columns: BC rows (DIR1 identity, DIR2 identity + mirror stencil) */
  int assembled;
} orc_ctx;

static void csr_free(csr *m) { free(m->ptr); free(m->col); free(m->val); memset(m, 0, sizeof(*m)); }
static int csr_begin(csr *m, int64_t nrows, int64_t cap) {
  csr_free(m);
  m->nrows = nrows; m->nnz = 0; m->cap = cap > 16 ? cap : 16;
  m->ptr = (int64_t *)calloc(nrows + 1, sizeof(int64_t));
  m->col = (int64_t *)malloc(sizeof(int64_t) * m->cap);
  m->val = (double *)malloc(sizeof(double) * m->cap);
  return (m->ptr && m->col && m->val) ? 0 : ORC_ERR_OOM;
}
static int csr_push(csr *m, int64_t c, double v) {
  if (m->nnz == m->cap) {
    m->cap *= 2;
    m->col = (int64_t *)realloc(m->col, sizeof(int64_t) * m->cap);
    m->val = (double *)realloc(m->val, sizeof(double) * m->cap);
    if (!m->col || !m->val) return ORC_ERR_OOM;
  }
  m->col[m->nnz] = c; m->val[m->nnz] = v; m->nnz++;
  return 0;
}

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  free(c->sh_a); free(c->sh_c); free(c->ijk); free(c->cp); hm_free(&c->index);
  free(c->curves); free(c->bc_of); free(c->near_c); free(c->twin); free(c->bc_curve);
  free(c->cpc); free(c->bc_side); free(c->bc_type);
  csr_free(&c->E); csr_free(&c->Loff); csr_free(&c->B);
  free(c);
}

/* Eq. (3): r = dx sqrt((d-1)((p+1)/2)^2 + (q+(p+1)/2)^2) with q = 1 */
double orc_tube_radius(int dim, int p, double h) {
  double half = ((double)p + 1.0) / 2.0;
  return h * sqrt((double)(dim - 1) * (half * half) + (1.0 + half) * (1.0 + half));
}

static void node_x(const orc_ctx *c, const int *ijk, double *x) {
  x[0] = (double)ijk[0] * c->h;
  x[1] = (double)ijk[1] * c->h;
  x[2] = (c->dim == 3) ? (double)ijk[2] * c->h : 0.0;
}

/* membership test of Eq. (3)'s band: |x - cp_S(x)| <= r */
static int band_member(const orc_ctx *c, const int *ijk, double *cp, int *err) {
  double x[3];
  node_x(c, ijk, x);
  int e = cp_S(&c->sh, x, cp);
  if (e) { *err = e; return 0; }
  double d[3] = {x[0] - cp[0], x[1] - cp[1], x[2] - cp[2]};
  return norm3(d) <= c->rband;
}

static int cmp_canon(const void *a, const void *b) {
  int64_t ka = ((const int64_t *)a)[0], kb = ((const int64_t *)b)[0];
  return (ka < kb) ? -1 : (ka > kb);
}

/* Alg. 1: BFS from a node near S over the 2d axis neighbours, keeping nodes
 * with |x - cp_S(x)| <= r; then sort into the canonical order. */
int orc_build(const orc_shape *sh, double h, int p, double rband, orc_ctx **out) {
  if (!sh || !out || h <= 0 || (p != 2 && p != 3)) return ORC_ERR_ARG;
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  if (!c) return ORC_ERR_OOM;
  c->sh = *sh;
  if (sh->K > 0) {
    c->sh_a = (double *)malloc(sizeof(double) * sh->K);
    c->sh_c = (double *)malloc(sizeof(double) * 3 * sh->K);
    memcpy(c->sh_a, sh->a, sizeof(double) * sh->K);
    memcpy(c->sh_c, sh->c, sizeof(double) * 3 * sh->K);
    c->sh.a = c->sh_a; c->sh.c = c->sh_c;
  }
  c->dim = sh->dim; c->h = h; c->p = p;
  c->rband = rband > 0 ? rband : orc_tube_radius(sh->dim, p, h);
  int seed[3] = {(int)lround(sh->seed[0] / h), (int)lround(sh->seed[1] / h), sh->dim == 3 ? (int)lround(sh->seed[2] / h) : 0};
  hmap visited;
  if (hm_init(&visited, 1 << 16)) { orc_destroy(c); return ORC_ERR_OOM; }
  int64_t qcap = 1 << 16, qhead = 0, qtail = 0;
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * 3 * qcap);
  double *qcp = (double *)malloc(sizeof(double) * 3 * qcap);
  int err = 0;
  double cp0[3];
  if (!band_member(c, seed, cp0, &err)) { free(q); free(qcp); hm_free(&visited); orc_destroy(c); return err ? err : ORC_ERR_ARG; }
  *hm_slot(&visited, node_key(seed[0], seed[1], seed[2]), 1) = 1;
  memcpy(q, seed, sizeof(int) * 3); memcpy(qcp, cp0, sizeof(cp0)); qtail = 1;
  while (qhead < qtail) {
    int cur[3] = {q[3 * qhead], q[3 * qhead + 1], q[3 * qhead + 2]};
    for (int a = 0; a < c->dim; ++a)
      for (int s = -1; s <= 1; s += 2) {
        int nb[3] = {cur[0], cur[1], cur[2]};
        nb[a] += s;
        int64_t *v = hm_slot(&visited, node_key(nb[0], nb[1], nb[2]), 1);
        if (!v) { err = ORC_ERR_OOM; goto done; }
        if (*v != -1) continue;
        *v = 0;
        double cp[3];
        if (band_member(c, nb, cp, &err)) {
          *v = 1;
          if (qtail == qcap) {
            qcap *= 2;
            q = (int32_t *)realloc(q, sizeof(int32_t) * 3 * qcap);
            qcp = (double *)realloc(qcp, sizeof(double) * 3 * qcap);
            if (!q || !qcp) { err = ORC_ERR_OOM; goto done; }
          }
          memcpy(q + 3 * qtail, nb, sizeof(int) * 3);
          memcpy(qcp + 3 * qtail, cp, sizeof(cp));
          qtail++;
        }
        if (err) goto done;
      }
    qhead++;
  }
done:
  hm_free(&visited);
  if (err) { free(q); free(qcp); orc_destroy(c); return err; }
  /* canonical order */
  int64_t n = qtail;
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * 2 * n);
  for (int64_t i = 0; i < n; ++i) { order[2 * i] = canon_key(q + 3 * i); order[2 * i + 1] = i; }
  qsort(order, n, 2 * sizeof(int64_t), cmp_canon);
  c->NS = n;
  c->ijk = (int32_t *)malloc(sizeof(int32_t) * 3 * n);
  c->cp = (double *)malloc(sizeof(double) * 3 * n);
  hm_init(&c->index, n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t s = order[2 * i + 1];
    memcpy(c->ijk + 3 * i, q + 3 * s, sizeof(int32_t) * 3);
    memcpy(c->cp + 3 * i, qcp + 3 * s, sizeof(double) * 3);
    *hm_slot(&c->index, node_key(c->ijk[3 * i], c->ijk[3 * i + 1], c->ijk[3 * i + 2]), 1) = i;
  }
  free(order); free(q); free(qcp);
  *out = c;
  return 0;
}

/* brute-force band over a box of integer indices (a pin for Alg. 1) */
int64_t orc_band_bruteforce(const orc_shape *sh, double h, int p, double rband, const int *lo, const int *hi, int32_t *out, int64_t cap) {
  orc_ctx c;
  memset(&c, 0, sizeof(c));
  c.sh = *sh; c.dim = sh->dim; c.h = h; c.p = p; c.rband = rband > 0 ? rband : orc_tube_radius(sh->dim, p, h);
  int64_t n = 0;
  int klo = sh->dim == 3 ? lo[2] : 0, khi = sh->dim == 3 ? hi[2] : 0;
  for (int k = klo; k <= khi; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int ijk[3] = {i, j, k}, err = 0;
        double cp[3];
        if (band_member(&c, ijk, cp, &err)) {
          if (n < cap) memcpy(out + 3 * n, ijk, sizeof(ijk));
          n++;
        }
      }
  return n;
}

int64_t orc_ns(const orc_ctx *c) { return c->NS; }
int64_t orc_nc(const orc_ctx *c) { return c->NC; }
double orc_rband(const orc_ctx *c) { return c->rband; }
void orc_export_band(const orc_ctx *c, int32_t *ijk, double *cp) {
  if (ijk) memcpy(ijk, c->ijk, sizeof(int32_t) * 3 * c->NS);
  if (cp) memcpy(cp, c->cp, sizeof(double) * 3 * c->NS);
}
int64_t orc_lookup(const orc_ctx *c, int i, int j, int k) { return hm_get(&c->index, node_key(i, j, k)); }

/* single-point closest point (exported for tests) */
int orc_cp(const orc_shape *sh, const double *x, double *cp) { return cp_S(sh, x, cp); }
void orc_bumpy_phi(const orc_shape *sh, const double *x, double *phi, double *grad, double *hess) {
  bumpy_phi(sh, x, phi, grad, hess);
}
void orc_cpc(const orc_curve *cv, const double *x, double *out) { cp_C(cv, x, out); }

/* ------------------------------------------------------------------ */
/* Interpolation weights: barycentric Lagrange form (Sec. 3.2, Berrut & Trefethen)
 * of degree p on the equispaced nodes 0..p in units of dx; weights lambda_j
 * proportional to (-1)^j C(p,j).  Exact hit on a node gives the Kronecker delta. */
void orc_bary_weights(int p, double t, double *w) {
  static const double lam3[4] = {1.0, -3.0, 3.0, -1.0};
  static const double lam2[3] = {1.0, -2.0, 1.0};
  const double *lam = (p == 2) ? lam2 : lam3;
  const int n = p + 1;
  for (int j = 0; j < n; ++j)
    if (t == (double)j) {
      for (int k = 0; k < n; ++k) w[k] = (k == j) ? 1.0 : 0.0;
      return;
    }
  double q[4], s = 0.0;
  for (int j = 0; j < n; ++j) { q[j] = lam[j] / (t - (double)j); s += q[j]; }
  for (int j = 0; j < n; ++j) w[j] = q[j] / s;
}

/* stencil of a query point y: the p + 1 nodes per axis nearest to y.  Cubic:
 * base floor(y/dx) - 1, so that y lies between stencil nodes 1 and 2.
 * Quadratic: base floor(y/dx + 1/2) - 1, so that node 1 is the nearest node
 * and every stencil node lies within 1.5 dx of y, the half-width (p+1)/2 that
 * Eq. (3) assumes.  t = y/dx - base. */
static void stencil_of(const orc_ctx *c, const double *y, int base[3], double t[3]) {
  for (int a = 0; a < 3; ++a) {
    if (a >= c->dim) { base[a] = 0; t[a] = 0.0; continue; }
    double s = y[a] / c->h;
    base[a] = (c->p == 2) ? (int)floor(s + 0.5) - 1 : (int)floor(s) - 1;
    t[a] = s - (double)base[a];
  }
}

/* ------------------------------------------------------------------ */
/* Interior boundaries (Sec. 4)                                          */

/* cp_{S-C}(x) = cp_S(x) - cp_C(x) (Eq. 8).  A vector shorter than 0.1 dx^2 means
 * cp_S(x) lies on C (Sec. 4.2), and the paper lets such a point take either
 * side.  Reading: it takes the side of the first node of its own interpolation
 * stencil (stencil order x fastest, then y, then z) whose cp_{S-C} is not that
 * short, i.e. that node's vector stands in for its own.  (An exactly-zero
 * vector that flipped nothing would leave the rows of nodes on S_perp as plain
 * Laplacian rows across C, and the IBC would not be imposed there.) */
/* Unit normal of S at a point y on S (Sec. 4.7 evaluates it at cp_C(x)):
 * circle and sphere y/|y|; torus (y - ring point)/|...|; bumpy sphere
 * grad phi/|grad phi| (App. A).  Reading: the analytic shapes give the normal in
 * closed form, where the paper (for meshes) takes the eigenvector of the FD
 * Jacobian of cp_S; both are the normal of S at that point. */
static void shape_normal(const orc_shape *sh, const double *y, double n[3]) {
  if (sh->kind == SH_BUMPY) {
    double phi, g[3], hs[9];
    bumpy_phi(sh, y, &phi, g, hs);
    double m = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
    n[0] = g[0] / m; n[1] = g[1] / m; n[2] = g[2] / m;
    return;
  }
  double d[3] = {y[0], y[1], y[2]};
  if (sh->kind == SH_CIRCLE) d[2] = 0.0;
  if (sh->kind == SH_TORUS) {
    double rho = sqrt(y[0] * y[0] + y[1] * y[1]);
    d[0] = y[0] - sh->R * (y[0] / rho);
    d[1] = y[1] - sh->R * (y[1] / rho);
  }
  double m = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
  n[0] = d[0] / m; n[1] = d[1] / m; n[2] = d[2] / m;
}

/* Unit tangent of a circle C at its point cc: nu x (cc - p), normalised */
static void circle_tangent(const orc_curve *cv, const double *cc, double t[3]) {
  double w[3] = {cc[0] - cv->p[0], cc[1] - cv->p[1], cc[2] - cv->p[2]};
  double u[3] = {cv->nu[1] * w[2] - cv->nu[2] * w[1], cv->nu[2] * w[0] - cv->nu[0] * w[2],
                 cv->nu[0] * w[1] - cv->nu[1] * w[0]};
  double m = sqrt((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]);
  t[0] = u[0] / m; t[1] = u[1] / m; t[2] = u[2] / m;
}

/* cp_{S-C}(x) of one node; with the projected test (Sec. 4.7, Eq. for
 * cp-perp) the components along n_S and t_C at cp_C(x) are removed, in that
 * order (a point C has no tangent: n_S only) */
static void cpdiff_raw(const orc_ctx *c, const orc_curve *cv, int64_t node, double z[3]) {
  double x[3], cc[3];
  node_x(c, c->ijk + 3 * node, x);
  cp_C(cv, x, cc);
  const double *cs = c->cp + 3 * node;
  z[0] = cs[0] - cc[0]; z[1] = cs[1] - cc[1]; z[2] = cs[2] - cc[2];
  if (!cv->projected) return;
  double n[3];
  shape_normal(&c->sh, cc, n);
  double a = dot3(z, n);
  z[0] = z[0] - a * n[0]; z[1] = z[1] - a * n[1]; z[2] = z[2] - a * n[2];
  if (cv->kind == CV_CIRCLE) {
    double t[3];
    circle_tangent(cv, cc, t);
    double b = dot3(z, t);
    z[0] = z[0] - b * t[0]; z[1] = z[1] - b * t[1]; z[2] = z[2] - b * t[2];
  }
}
static void cpdiff(const orc_ctx *c, const orc_curve *cv, int64_t node, double z[3]) {
  double tiny = 0.1 * c->h * c->h;
  cpdiff_raw(c, cv, node, z);
  if (norm3(z) >= tiny) return;
  int base[3];
  double t[3];
  stencil_of(c, c->cp + 3 * node, base, t);
  const int np1 = c->p + 1;
  int nz = (c->dim == 3) ? np1 : 1;
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < np1; ++cy)
      for (int cx = 0; cx < np1; ++cx) {
        int64_t j = hm_get(&c->index, node_key(base[0] + cx, base[1] + cy, c->dim == 3 ? base[2] + cz : 0));
        if (j < 0) continue;
        double w[3];
        cpdiff_raw(c, cv, j, w);
        if (norm3(w) >= tiny) { z[0] = w[0]; z[1] = w[1]; z[2] = w[2]; return; }
      }
  z[0] = z[1] = z[2] = 0.0;
}

static double node_dist_to_curve(const orc_ctx *c, const orc_curve *cv, int64_t node) {
  double x[3], cc[3];
  node_x(c, c->ijk + 3 * node, x);
  cp_C(cv, x, cc);
  double d[3] = {x[0] - cc[0], x[1] - cc[1], x[2] - cc[2]};
  return norm3(d);
}

static int cmp_i64pair(const void *a, const void *b) {
  const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
  return (x[1] < y[1]) ? -1 : (x[1] > y[1]);
}

/* Omega(C) (Sec. 4.1): band nodes within r of each curve receive a BC DOF,
 * numbered after the PDE DOFs in (curve, canonical) order.  Rows within
 * 2 r of a curve are tested for crossings (Sec. 4.6).  Reading: a node within
 * 2 r of two curves is rejected as overlapping, so each tested row (and each
 * BC DOF) belongs to exactly one curve; a twin is only taken from the row's
 * own curve. */
int orc_set_curves(orc_ctx *c, const orc_curve *curves, int ncurves) {
  if (!c || ncurves < 0) return ORC_ERR_ARG;
  free(c->curves); free(c->bc_of); free(c->near_c); free(c->twin); free(c->bc_curve); free(c->cpc); free(c->bc_side);
  free(c->bc_type);
  c->bc_type = NULL;
  c->assembled = 0;
  c->ncurves = ncurves;
  c->curves = (orc_curve *)malloc(sizeof(orc_curve) * (ncurves > 0 ? ncurves : 1));
  if (ncurves) memcpy(c->curves, curves, sizeof(orc_curve) * ncurves);
  int64_t NS = c->NS;
  c->bc_of = (int64_t *)malloc(sizeof(int64_t) * NS);
  c->near_c = (int32_t *)malloc(sizeof(int32_t) * NS);
  for (int64_t i = 0; i < NS; ++i) { c->bc_of[i] = -1; c->near_c[i] = -1; }
  double zone = 2.0 * c->rband;
  int64_t nc = 0, cap = 1024;
  int64_t *list = (int64_t *)malloc(sizeof(int64_t) * 2 * cap); /* (curve, pde index) */
  for (int64_t i = 0; i < NS; ++i) {
    int nz = 0;
    for (int k = 0; k < ncurves; ++k) {
      double dC = node_dist_to_curve(c, &c->curves[k], i);
      if (dC < zone) nz++;
      if (nz > 1) { free(list); return ORC_ERR_OVERLAP; }
      if (dC < 2.0 * c->rband) c->near_c[i] = k;
      if (dC <= c->rband) {
        if (nc == cap) { cap *= 2; list = (int64_t *)realloc(list, sizeof(int64_t) * 2 * cap); }
        list[2 * nc] = k; list[2 * nc + 1] = i; nc++;
      }
    }
  }
  /* PDE indices are already canonical, so (curve, pde index) is (curve, canonical) */
  qsort(list, nc, 2 * sizeof(int64_t), cmp_i64pair);
  c->NC = nc;
  c->twin = (int64_t *)malloc(sizeof(int64_t) * (nc ? nc : 1));
  c->bc_curve = (int32_t *)malloc(sizeof(int32_t) * (nc ? nc : 1));
  c->cpc = (double *)malloc(sizeof(double) * 3 * (nc ? nc : 1));
  c->bc_side = (int32_t *)malloc(sizeof(int32_t) * (nc ? nc : 1));
  c->bc_type = (int32_t *)malloc(sizeof(int32_t) * (nc ? nc : 1));
  for (int64_t a = 0; a < nc; ++a) {
    int k = (int)list[2 * a];
    int64_t j = list[2 * a + 1];
    c->twin[a] = j; c->bc_curve[a] = k;
    c->bc_of[j] = NS + a;
    double x[3];
    node_x(c, c->ijk + 3 * j, x);
    cp_C(&c->curves[k], x, c->cpc + 3 * a);
    double z[3];
    cpdiff(c, &c->curves[k], j, z);
    double s = dot3(z, c->curves[k].nu);
    c->bc_side[a] = (c->curves[k].kind == CV_POINT && c->dim == 3) ? 0 : (s > 0) - (s < 0);
    /* a BC DOF stands in for its node as seen from the other side of C, so its
     * equation is the BC of the side opposite cp_S(x_alpha) (Sec. 4.2: mixed
     * types, one per side) */
    int bminus = c->curves[k].bc_minus ? c->curves[k].bc_minus : c->curves[k].bc;
    c->bc_type[a] = (c->bc_side[a] > 0) ? bminus : c->curves[k].bc;
  }
  free(list);
  return 0;
}

void orc_export_bc(const orc_ctx *c, int64_t *twin, int32_t *curve, double *cpc, int32_t *side, int32_t *type) {
  if (twin) memcpy(twin, c->twin, sizeof(int64_t) * c->NC);
  if (curve) memcpy(curve, c->bc_curve, sizeof(int32_t) * c->NC);
  if (cpc) memcpy(cpc, c->cpc, sizeof(double) * 3 * c->NC);
  if (side) memcpy(side, c->bc_side, sizeof(int32_t) * c->NC);
  if (type) memcpy(type, c->bc_type, sizeof(int32_t) * c->NC);
}
/* the (tie-resolved, possibly projected) crossing vector cp_{S-C} of PDE
 * node i for curve k, as the crossing test uses it */
int orc_crossing_vector(const orc_ctx *c, int k, int64_t i, double *z) {
  if (!c || k < 0 || k >= c->ncurves || i < 0 || i >= c->NS) return ORC_ERR_ARG;
  cpdiff(c, &c->curves[k], i, z);
  return 0;
}
void orc_export_near(const orc_ctx *c, int32_t *near_c, int64_t *bc_of) {
  if (near_c) memcpy(near_c, c->near_c, sizeof(int32_t) * c->NS);
  if (bc_of) memcpy(bc_of, c->bc_of, sizeof(int64_t) * c->NS);
}

/* PDE-row stencil modification, Eq. (10): for a row tested against curve k with
 * direction dstar = cp_{S-C}(x_i), node j is replaced by its BC twin when
 * dstar . cp_{S-C}(x_j) < 0.  A requested flip with no twin keeps j (counted). */
static int64_t pde_col(orc_ctx *c, int k, const double *dstar, int64_t j) {
  if (k < 0) return j;
  double z[3];
  cpdiff(c, &c->curves[k], j, z);
  if (dot3(dstar, z) < 0.0) {
    int64_t a = c->bc_of[j];
    if (a >= 0 && c->bc_curve[a - c->NS] == k) return a;
    c->n_noflip_twin++;
  }
  return j;
}

/* BC-row stencil, Eq. (11) read for the Dirichlet mirror stencil: the default
 * column is the BC twin, replaced by the PDE DOF j when dstar . cp_{S-C}(x_j) < 0;
 * a node without a twin uses j. */
static int64_t bc_col(orc_ctx *c, int k, const double *dstar, int64_t j) {
  double z[3];
  cpdiff(c, &c->curves[k], j, z);
  if (dot3(dstar, z) < 0.0) return j;
  int64_t a = c->bc_of[j];
  if (a >= 0 && c->bc_curve[a - c->NS] == k) return a;
  return j;
}

/* Assemble E (Eq. 1 with Eq. 10 flips), the off-diagonal part of L (Eq. 2 with
 * the same flips) and the BC rows (Sec. 4.3).  Reading: BC rows are the BC
 * equations themselves, with the type of the side the BC DOF stands in for:
 *   first-order Dirichlet   u_alpha                    = g
 *   second-order Dirichlet  u_alpha + sum wbar u       = 2 g   (stencil at cpbar_C)
 *   first-order Neumann     u_alpha - sum w u          = 0     (stencil at cp_C)
 *   second-order Neumann    u_alpha - sum wbar u       = 0     (stencil at cpbar_C)
 * with the mirror point cpbar_C = cp_S(2 cp_C - x) of Sec. 4.3.  A missing FD
 * neighbour (band edge) contributes nothing. */
int orc_assemble(orc_ctx *c) {
  if (!c) return ORC_ERR_ARG;
  int64_t NS = c->NS, NC = c->NC;
  int d = c->dim;
  const int np1 = c->p + 1;
  int npts = (d == 3) ? np1 * np1 * np1 : np1 * np1;
  c->n_noflip_twin = 0;
  if (csr_begin(&c->E, NS, NS * npts) || csr_begin(&c->Loff, NS, NS * 2 * d) || csr_begin(&c->B, NC, NC * (npts + 1)))
    return ORC_ERR_OOM;
  double inv_h2 = 1.0 / (c->h * c->h);
  int nz = (d == 3) ? np1 : 1;
  for (int64_t i = 0; i < NS; ++i) {
    int k = c->near_c[i];
    double dstar[3] = {0, 0, 0};
    if (k >= 0) cpdiff(c, &c->curves[k], i, dstar);
    int base[3];
    double t[3], w[3][4] = {{0}};
    stencil_of(c, c->cp + 3 * i, base, t);
    for (int a = 0; a < d; ++a) orc_bary_weights(c->p, t[a], w[a]);
    for (int cz = 0; cz < nz; ++cz)
      for (int cy = 0; cy < np1; ++cy)
        for (int cx = 0; cx < np1; ++cx) {
          int64_t j = hm_get(&c->index, node_key(base[0] + cx, base[1] + cy, d == 3 ? base[2] + cz : 0));
          if (j < 0) return ORC_ERR_STATE; /* an interpolation node outside the band */
          double wt = w[0][cx] * w[1][cy];
          if (d == 3) wt = wt * w[2][cz];
          if (csr_push(&c->E, pde_col(c, k, dstar, j), wt)) return ORC_ERR_OOM;
        }
    c->E.ptr[i + 1] = c->E.nnz;
    const int32_t *p = c->ijk + 3 * i;
    for (int a = 0; a < d; ++a)
      for (int s = -1; s <= 1; s += 2) {
        int nb[3] = {p[0], p[1], p[2]};
        nb[a] += s;
        int64_t j = hm_get(&c->index, node_key(nb[0], nb[1], nb[2]));
        if (j < 0) continue;
        if (csr_push(&c->Loff, pde_col(c, k, dstar, j), inv_h2)) return ORC_ERR_OOM;
      }
    c->Loff.ptr[i + 1] = c->Loff.nnz;
  }
  for (int64_t a = 0; a < NC; ++a) {
    int k = c->bc_curve[a];
    int64_t j = c->twin[a];
    int type = c->bc_type[a];
    if (csr_push(&c->B, NS + a, 1.0)) return ORC_ERR_OOM;
    if (type != BC_DIR1) {
      double dstar[3], x[3], q[3];
      cpdiff(c, &c->curves[k], j, dstar);
      const double *cc = c->cpc + 3 * a;
      if (type == BC_NEU1) {
        /* first-order Neumann: the query point is cp_C(x_alpha) itself */
        q[0] = cc[0]; q[1] = cc[1]; q[2] = cc[2];
      } else {
        /* second order: the mirror point cpbar_C = cp_S(2 cp_C - x) (Sec. 4.3) */
        double y[3];
        node_x(c, c->ijk + 3 * j, x);
        for (int e = 0; e < 3; ++e) y[e] = 2.0 * cc[e] - x[e];
        int err = cp_S(&c->sh, y, q);
        if (err) return err;
      }
      const double sgn = (type == BC_DIR2) ? 1.0 : -1.0;
      int base[3];
      double t[3], w[3][4] = {{0}};
      stencil_of(c, q, base, t);
      for (int e = 0; e < d; ++e) orc_bary_weights(c->p, t[e], w[e]);
      for (int cz = 0; cz < nz; ++cz)
        for (int cy = 0; cy < np1; ++cy)
          for (int cx = 0; cx < np1; ++cx) {
            int64_t qn = hm_get(&c->index, node_key(base[0] + cx, base[1] + cy, d == 3 ? base[2] + cz : 0));
            if (qn < 0) return ORC_ERR_STATE;
            double wt = w[0][cx] * w[1][cy];
            if (d == 3) wt = wt * w[2][cz];
            if (csr_push(&c->B, bc_col(c, k, dstar, qn), sgn * wt)) return ORC_ERR_OOM;
          }
    }
    c->B.ptr[a + 1] = c->B.nnz;
  }
  c->assembled = 1;
  return 0;
}

int64_t orc_noflip_twin(const orc_ctx *c) { return c->n_noflip_twin; }

void orc_csr_dims(const orc_ctx *c, int which, int64_t *nrows, int64_t *nnz) {
  const csr *m = which == 0 ? &c->E : which == 1 ? &c->Loff : &c->B;
  *nrows = m->nrows; *nnz = m->nnz;
}
void orc_csr_export(const orc_ctx *c, int which, int64_t *ptr, int64_t *col, double *val) {
  const csr *m = which == 0 ? &c->E : which == 1 ? &c->Loff : &c->B;
  memcpy(ptr, m->ptr, sizeof(int64_t) * (m->nrows + 1));
  memcpy(col, m->col, sizeof(int64_t) * m->nnz);
  memcpy(val, m->val, sizeof(double) * m->nnz);
}

/* ------------------------------------------------------------------ */
/* The four-step partially matrix-free product of Sec. 5.4 with stored E, L:
 *   a = E u ; b = (L - diag L) a ; a = diag(L) u ; v = m u + n a + n b
 * on the PDE rows (E rows of BC DOFs are the identity); BC rows apply B. */
int orc_apply(const orc_ctx *c, double m, double n, const double *u, double *v, double *work) {
  if (!c->assembled) return ORC_ERR_STATE;
  int64_t NS = c->NS, NC = c->NC, N = NS + NC;
  double *a = work; /* [N] */
  double diagL = -2.0 * (double)c->dim / (c->h * c->h);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < NS; ++i) {
    double s = 0.0;
    for (int64_t e = c->E.ptr[i]; e < c->E.ptr[i + 1]; ++e) s += c->E.val[e] * u[c->E.col[e]];
    a[i] = s;
  }
#pragma omp parallel for schedule(static)
  for (int64_t al = NS; al < N; ++al) a[al] = u[al];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < NS; ++i) {
    double b = 0.0;
    for (int64_t e = c->Loff.ptr[i]; e < c->Loff.ptr[i + 1]; ++e) b += c->Loff.val[e] * a[c->Loff.col[e]];
    double a2 = diagL * u[i];
    v[i] = (m * u[i] + n * a2) + n * b;
  }
#pragma omp parallel for schedule(static)
  for (int64_t al = 0; al < NC; ++al) {
    double s = 0.0;
    for (int64_t e = c->B.ptr[al]; e < c->B.ptr[al + 1]; ++e) s += c->B.val[e] * u[c->B.col[e]];
    v[NS + al] = s;
  }
  return 0;
}

/* E applied alone: the side-correct surface values (E u)_i at cp_S(x_i) */
int orc_extend(const orc_ctx *c, const double *u, double *a) {
  if (!c->assembled) return ORC_ERR_STATE;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->NS; ++i) {
    double s = 0.0;
    for (int64_t e = c->E.ptr[i]; e < c->E.ptr[i + 1]; ++e) s += c->E.val[e] * u[c->E.col[e]];
    a[i] = s;
  }
  return 0;
}

static double vdot(const double *x, const double *y, int64_t n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

/* Preconditioned BiCGSTAB (van der Vorst 1992) with the diagonal of
 * m I + n diag(L) on PDE rows and 1 on BC rows (Sec. 5.4).  Stops when
 * |r|_2 <= tol |f|_2.  A near-zero rho restarts with rhat = r. */
int orc_bicgstab(const orc_ctx *c, double m, double n, const double *f, double *x, double tol, int maxit,
                 int *iters_out, double *relres_out) {
  if (!c->assembled) return ORC_ERR_STATE;
  int64_t NS = c->NS, N = c->NS + c->NC;
  double dinv_pde = 1.0 / (m + n * (-2.0 * (double)c->dim / (c->h * c->h)));
  double *buf = (double *)calloc((size_t)N * 9, sizeof(double));
  if (!buf) return ORC_ERR_OOM;
  double *r = buf, *rh = buf + N, *p = buf + 2 * N, *v = buf + 3 * N, *s = buf + 4 * N, *t = buf + 5 * N,
         *ph = buf + 6 * N, *sh = buf + 7 * N, *work = buf + 8 * N;
  orc_apply(c, m, n, x, r, work);
  for (int64_t i = 0; i < N; ++i) { r[i] = f[i] - r[i]; rh[i] = r[i]; }
  double fn = sqrt(vdot(f, f, N));
  if (fn == 0.0) fn = 1.0;
  double rho_old = 1.0, alpha = 1.0, omega = 1.0, rn = sqrt(vdot(r, r, N));
  int it = 0, status = ORC_ERR_NOT_CONVERGED, restarts = 0;
  if (rn <= tol * fn) status = ORC_OK;
  while (status != ORC_OK && it < maxit) {
    double rho = vdot(rh, r, N);
    if (fabs(rho) < 1e-32 * sqrt(vdot(rh, rh, N)) * rn) {
      /* restart the shadow residual */
      if (++restarts > 50) { status = ORC_ERR_BREAKDOWN; break; }
      for (int64_t i = 0; i < N; ++i) { rh[i] = r[i]; p[i] = 0.0; v[i] = 0.0; }
      rho = vdot(rh, r, N);
      rho_old = alpha = omega = 1.0;
    }
    double beta = (rho / rho_old) * (alpha / omega);
    for (int64_t i = 0; i < N; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    for (int64_t i = 0; i < N; ++i) ph[i] = (i < NS ? dinv_pde : 1.0) * p[i];
    orc_apply(c, m, n, ph, v, work);
    alpha = rho / vdot(rh, v, N);
    for (int64_t i = 0; i < N; ++i) s[i] = r[i] - alpha * v[i];
    for (int64_t i = 0; i < N; ++i) sh[i] = (i < NS ? dinv_pde : 1.0) * s[i];
    orc_apply(c, m, n, sh, t, work);
    double tt = vdot(t, t, N);
    omega = (tt > 0.0) ? vdot(t, s, N) / tt : 0.0;
    for (int64_t i = 0; i < N; ++i) {
      x[i] += alpha * ph[i] + omega * sh[i];
      r[i] = s[i] - omega * t[i];
    }
    rn = sqrt(vdot(r, r, N));
    rho_old = rho;
    it++;
    if (rn <= tol * fn) status = ORC_OK;
    if (omega == 0.0 && status != ORC_OK) { status = ORC_ERR_BREAKDOWN; break; }
  }
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = rn / fn;
  free(buf);
  return status;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
