/*
 * cpm.h -- C ABI of the GB300 (sm_103a) closest point method library with
 * interior boundary conditions.
 *
 * The library implements the discrete CPM of King, Su, Aanjaneya, Ruuth and
 * Batty, "A Closest Point Method for PDEs on Manifolds with Interior Boundary
 * Conditions for Geometry Processing" (ACM TOG 2024): a narrow band of grid
 * nodes around a manifold S (Eq. 3, Alg. 1), duplicated BC degrees of freedom
 * near interior boundaries C (Sec. 4.1), interpolation and finite-difference
 * stencils restricted to the correct side of C by the closest-point crossing
 * test (Eqs. 8-11), and the system
 *
 *     A = m I + n [ diag(L) + (L - diag L) E ]          (Sec. 5.3-5.4)
 *
 * applied matrix-free and solved with preconditioned BiCGSTAB (Sec. 5.4).
 *
 * Conventions shared by every entry point:
 *  - Status: every call returns cpm_status; nothing throws across the ABI.
 *    A failed call leaves the context usable unless it says otherwise.
 *  - Pointers named *_dev are DEVICE pointers owned by the caller (never freed
 *    or retained by the library).  Descriptor structs are host memory and are
 *    copied during the call.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it; calls that must read results back
 *    (band build, set-boundary, solves when stats are requested) synchronise it.
 *  - DOF layout: N = N_S + N_C unknowns; PDE DOFs [0, N_S) are grid nodes of the
 *    band in canonical order (8^3 bricks by (bz, by, bx), nodes inside a brick by
 *    (lz, ly, lx)); BC DOFs [N_S, N) follow, ordered by (curve, canonical order of
 *    their node).  With nrhs > 1, vectors are row-major [N][ld] (right-hand side
 *    index fastest, nrhs <= ld).
 *  - Threads: a context may be used from one host thread at a time.
 *  - Memory: the library allocates device memory only in cpm_band_build,
 *    cpm_set_boundary and cpm_reserve.  Products, solves, extensions, the heat
 *    steps and the boundary gradient allocate nothing: they use workspaces
 *    reserved for a leading dimension (cpm_set_boundary reserves ld = 1, i.e.
 *    single right-hand sides, for every form; cpm_reserve widens it) and
 *    return CPM_ERR_CAPACITY when a call needs more than was reserved.
 */
#ifndef CPM_H
#define CPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CPM_OK = 0,
  CPM_ERR_ARG = 1,           /* bad argument (null pointer, size, unknown kind) */
  CPM_ERR_OOM = 2,           /* a device or host allocation failed */
  CPM_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  CPM_ERR_CAPACITY = 4,      /* a fixed-size table (brick hash) overflowed after retries, or a call
                                needs a wider workspace than cpm_reserve set aside */
  CPM_ERR_CP_FAILED = 5,     /* a closest-point Newton iteration did not converge */
  CPM_ERR_OVERLAP = 6,       /* a band node lies within 2 r of two interior boundaries */
  CPM_ERR_BREAKDOWN = 7,     /* BiCGSTAB broke down after the allowed restarts */
  CPM_ERR_NOT_CONVERGED = 8, /* the solve reached maxit before the tolerance */
  CPM_ERR_TIMEOUT = 9,       /* a bounded device or host loop hit its cap */
  CPM_ERR_STATE = 10         /* call out of order (e.g. apply before set_boundary) */
} cpm_status;

typedef enum { CPM_SHAPE_CIRCLE = 1, CPM_SHAPE_SPHERE = 2, CPM_SHAPE_TORUS = 3, CPM_SHAPE_BUMPY = 4 } cpm_shape_kind;
typedef enum { CPM_CURVE_POINT = 1, CPM_CURVE_CIRCLE = 2 } cpm_curve_kind;
typedef enum { CPM_BC_DIR1 = 1, CPM_BC_DIR2 = 2, CPM_BC_NEU1 = 3, CPM_BC_NEU2 = 4 } cpm_bc_kind;
typedef enum { CPM_PREC_FP64 = 0, CPM_PREC_FP32 = 1 } cpm_prec;
typedef enum { CPM_SOLVE_FP64 = 0, CPM_SOLVE_FP32_IR = 1 } cpm_solve_mode;

/* Manifold S given by its closest-point function (Sec. 3.1, App. A).
 *  CIRCLE (dim 2): circle of radius R about the origin.
 *  SPHERE (dim 3): sphere of radius R about the origin.
 *  TORUS  (dim 3): major radius R, minor radius rt, axis z.
 *  BUMPY  (dim 3): level set |x| = rho(x/|x|), rho(w) = 1 + amp sum_k a_k
 *                  exp(-|w - c_k|^2 / width); closest points by the two-stage
 *                  Newton projection of App. A in FP64.
 * seed is a point on or near S from which the band search starts (Alg. 1). */
typedef struct {
  int kind;
  int dim;
  double R;
  double rt;
  int K;
  double amp;
  double width;
  const double *a; /* host [K] */
  const double *c; /* host [3K], unit vectors */
  double seed[3];
} cpm_shape_desc;

/* Interior boundary C (Sec. 4).  POINT: p.  CIRCLE: centre p, unit plane normal
 * nu, radius rad, angle-0 direction ref (unit, in the plane).  nu also orients
 * the two sides of C: a surface point y is on side sign((y - cp_C) . nu) (for a
 * point in 2D, nu is the unit tangent of S there; a point in 3D has no sides).
 * Dirichlet data: n_samples values per side at curve angles 2 pi k / n_samples,
 * linearly interpolated (periodic); a point takes one value per side.
 * BC types (Sec. 4.3): Dirichlet or zero-Neumann, first or second order, one
 * per side (mixed types, Sec. 4.2).  A BC DOF stands in for its node as seen
 * from the other side of C, so its row is the BC of the side opposite
 * cp_S(x_alpha):
 *   DIR1  u_alpha                 = g
 *   DIR2  u_alpha + sum wbar u    = 2 g     (stencil at cpbar_C = cp_S(2 cp_C - x))
 *   NEU1  u_alpha - sum w u       = 0       (stencil at cp_C(x_alpha))
 *   NEU2  u_alpha - sum wbar u    = 0       (stencil at cpbar_C)
 * where a stencil node keeps its BC twin unless the crossing test puts it on
 * the other side (Eq. 11).  Neumann types need sides: not for points in 3D.
 * With `projected` the normal and tangent come in closed form from the shape
 * (sphere, circle, torus: the radial directions; bumpy sphere: the level-set
 * gradient) and the circle (nu x (cp_C - p)). */
typedef struct {
  int kind;       /* cpm_curve_kind */
  int bc;         /* cpm_bc_kind on the plus side (and on both when bc_minus = 0) */
  double p[3];
  double nu[3];
  double rad;
  double ref[3];
  int two_sided;  /* 0: one sample set for both sides; 1: plus-side then minus-side sets */
  int n_samples;  /* >= 1 */
  int bc_minus;   /* cpm_bc_kind on the minus side, or 0 for the same as bc */
  int projected;  /* 1: the projected crossing test of Sec. 4.7 -- before the sign test of
                     Eq. (9) the vectors cp_{S-C} lose their components along the surface
                     normal n_S and the curve tangent t_C, both at cp_C(x) (a point: n_S
                     only), which keeps the test reliable where S bends strongly near C;
                     0: the plain test of Eq. (9) */
} cpm_curve_desc;

typedef enum { CPM_NORM_PLAIN = 0, CPM_NORM_SCALED = 1 } cpm_norm;

typedef struct {
  double tol;        /* relative tolerance: BiCGSTAB stops a right-hand side when its residual
                        |W r|_2 <= tol |W f|_2, where W is the identity (CPM_NORM_PLAIN, the default:
                        the paper's relative residual, Sec. 5.4) or the Jacobi scaling
                        diag(1/(m + n diag L)) on PDE rows and 1 on BC rows (CPM_NORM_SCALED).  The
                        solve then checks the true residual of x in FP64: a right-hand side has
                        converged when it is within tol, or within 4 times its FP64 rounding floor
                        (stats.relres_floor) where that floor lies above tol (fine grids: the
                        floor grows like 1/h^2) */
  int maxit;         /* BiCGSTAB iterations (both modes) */
  int mode;          /* cpm_solve_mode */
  double inner_tol;  /* FP32_IR: reduction in (0,1) of a column's FP32 recursive residual at
                        which its inner solve ends and the FP64 residual restarts it, i.e. what
                        one refinement step aims for (0 -> 1e-1; the FP32 product's rounding,
                        relative to the smallest eigenvalues, limits what one inner solve can
                        gain on fine grids) */
  int max_refine;    /* FP32_IR: maximum number of refinement steps (0 -> 200) */
  int check_every;   /* iterations between host convergence checks (0 -> 16) */
  int norm;          /* cpm_norm.  PLAIN is the paper's right-preconditioned form with the unscaled
                        residual; SCALED iterates on the row-scaled system W A x = W f */
  int inner_maxit;   /* reserved (0) */
} cpm_solve_opts;

typedef struct {
  int iterations;    /* BiCGSTAB iterations */
  int refinements;   /* FP32_IR: refinement steps taken */
  int restarts;      /* shadow-residual restarts after near breakdown */
  double relres;     /* final FP64 relative residual |W (f - A x)| / |W f| in the chosen norm (max over
                        right-hand sides) */
  int status;        /* cpm_status of this solve */
  int fp64_iterations; /* iterations run in FP64 (all of them in FP64 mode; the FP64 finish in FP32_IR) */
  double relres_floor; /* the FP64 rounding floor of relres (max over right-hand sides; 0 when not needed):
                          (u / sqrt 3) |W A (x o xi)| / |W f| for a fixed random sign vector xi, u = 2^-53,
                          the residual that rounding the exact solution to FP64 alone leaves */
} cpm_solve_stats;

typedef struct cpm_ctx cpm_ctx;

/* Builds the band Omega(S) = { grid nodes x = h (i,j,k) : |x - cp_S(x)| <= r }
 * (Sec. 3.2, Eq. 3 for r; Sec. 5.1 and Alg. 1 for the search), stores cp_S for
 * every node (FP64) and allocates the context.  p is the interpolation degree:
 * 3 (cubic, 4^d stencils with base floor(y/h) - 1) or 2 (quadratic, Sec. 7:
 * 3^d stencils of the nodes nearest y, base floor(y/h + 1/2) - 1).
 * r_band <= 0 selects Eq. (3) with q = 1: r = h sqrt(13) / h sqrt(17) (2D / 3D)
 * for p = 3, h sqrt(8.5) / h sqrt(10.75) for p = 2.  Synchronises `stream`.
 * Errors: ARG, OOM, CUDA, CAPACITY, CP_FAILED, TIMEOUT.  *out is NULL on error. */
cpm_status cpm_band_build(const cpm_shape_desc *shape, double h, int p, double r_band, void *stream,
                          cpm_ctx **out);

/* Sizes of the system: N_S PDE DOFs, N_C BC DOFs (0 before cpm_set_boundary),
 * the band radius used, and the number of 8^3 bricks.  Any output may be NULL. */
cpm_status cpm_band_info(const cpm_ctx *ctx, int64_t *n_s, int64_t *n_c, double *r_band, int64_t *n_bricks);

/* Workspace reservation.  Reserves, for leading dimension up to ld (1..256),
 * the intermediates of the products (cpm_apply, cpm_apply_transpose,
 * cpm_extend) and, for the solve forms in flags (CPM_RESERVE_FP64 and/or
 * CPM_RESERVE_FP32_IR), the Krylov vectors, refinement buffers and reduction
 * partials of cpm_solve and cpm_solve_adjoint; a batched solve of nrhs columns
 * with leading dimension ld needs ld reserved.  Reservations only grow; they
 * are dropped by cpm_set_boundary, which reserves ld = 1 for every form.  The
 * paper has no counterpart: this keeps allocation out of the products and the
 * iteration.  Synchronises the device.  Errors: ARG, STATE (no boundary set),
 * OOM. */
typedef enum { CPM_RESERVE_FP64 = 1, CPM_RESERVE_FP32_IR = 2 } cpm_reserve_flags;
cpm_status cpm_reserve(cpm_ctx *ctx, int64_t ld, int flags);

/* Copies the band to caller device buffers: grid indices ijk_dev [N_S][3]
 * (int32) and closest points cp_dev [N_S][3] (FP64), canonical order.  Either
 * may be NULL.  Asynchronous on `stream`. */
cpm_status cpm_export_band(const cpm_ctx *ctx, int32_t *ijk_dev, double *cp_dev, void *stream);

/* Sets the interior boundaries (replacing any previous set) and builds the
 * operator data: Omega(C) and the BC DOFs (Sec. 4.1), the crossing-test flips of
 * every stencil of rows within 2 r of a curve (Eqs. 10-11, Sec. 4.6), and the
 * Dirichlet BC rows (Sec. 4.3): u_alpha = g (first order) or
 * u_alpha + sum wbar u = 2 g with the stencil at cpbar_C = cp_S(2 cp_C - x)
 * (second order).  n_curves = 0 gives the plain closed-manifold operator.
 * Synchronises `stream` (the library's internal stream is the one passed to
 * cpm_band_build).  Errors: ARG, OOM, CUDA, OVERLAP, CP_FAILED. */
cpm_status cpm_set_boundary(cpm_ctx *ctx, const cpm_curve_desc *curves, int n_curves);

/* Per BC DOF (device outputs, [N_C] each, any may be NULL): PDE twin index,
 * curve id, cp_C(x_alpha) ([N_C][3]), side of cp_S(x_alpha) (+1/-1/0), the
 * curve angle of cp_C(x_alpha) in [0, 2pi) (0 for points) and the row's BC type
 * (cpm_bc_kind of the side opposite cp_S(x_alpha)).  Asynchronous. */
cpm_status cpm_export_boundary(const cpm_ctx *ctx, int64_t *twin_dev, int32_t *curve_dev, double *cpc_dev,
                               int32_t *side_dev, double *param_dev, int32_t *type_dev, void *stream);

/* Right-hand side f = [ s ; c_alpha g_alpha ] (Sec. 5.2): s_dev [N_S] (source
 * extended from cp_S, or NULL for 0) and Dirichlet values g_alpha from either
 * g_dev [N_C] (one value per BC DOF, for the side opposite cp_S(x_alpha)) or
 * samples_dev (all curves' sample sets concatenated; per curve n_samples values,
 * or 2 n_samples when two-sided: plus side first).  c_alpha = 1 for first-order
 * and 2 for second-order Dirichlet rows, 0 for zero-Neumann rows.  With
 * nrhs > 1 every array carries nrhs columns with leading dimension ld.
 * Asynchronous. */
cpm_status cpm_rhs(cpm_ctx *ctx, const double *s_dev, const double *g_dev, const double *samples_dev, double *f_dev,
                   int nrhs, int64_t ld, void *stream);

/* v = A u with A = m I + n [diag L + (L - diag L) E] on PDE rows and the BC rows
 * (Sec. 5.4's product, fused on the device).  prec selects FP64 (double*) or FP32
 * (float*) arithmetic and storage for u and v.  u_dev, v_dev: [N] or [N][ld].
 * The interpolation is summed in difference form, sum_j w_j (u_j - u_i) + u_i
 * (Eq. 1 with sum_j w_j = 1), so rounding stays relative to local differences.
 * Requires cpm_set_boundary (possibly with no curves) and ld reserved (see
 * cpm_reserve); allocates nothing.  Asynchronous.  Errors: ARG, STATE,
 * CAPACITY, CUDA. */
cpm_status cpm_apply(cpm_ctx *ctx, double m, double n, int prec, const void *u_dev, void *v_dev, int nrhs,
                     int64_t ld, void *stream);

/* cpm_apply through a fixed module array.  The paper has no counterpart: this is a
 * library-level variant for callers that cannot allocate device memory at the
 * time of the call -- for instance a host framework that has already handed all
 * device memory to its own pool (a cudaMalloc would fail), or a latency-bound
 * caller that must not pay the implicit device synchronisation of cudaMalloc /
 * cudaFree.  Same arguments, layout and result as cpm_apply; the E u
 * intermediate goes to one fixed device array of cpm_apply_noalloc_max_bytes()
 * bytes (16 MiB) inside the library instead of the context's scratch, which
 * cpm_apply grows on demand.
 *  - Size limit: element size x N_S x ld must not exceed that many bytes,
 *    otherwise CPM_ERR_CAPACITY is returned and nothing is launched.
 *  - The array's device address is looked up (cudaGetSymbolAddress) on the
 *    first call for each device, with that device current; make the first call
 *    on a device before any stream capture.  A failed lookup returns CPM_ERR_CUDA.
 *    The address is cached per device index for the life of the process, so
 *    resetting a device (cudaDeviceReset) or switching it to a different CUDA
 *    context between calls is not supported.
 *  - Nothing needs to start at zero: every element that is read was written
 *    earlier in the same call.
 *  - The array is shared by all contexts and streams on a device: calls that
 *    overlap in time on one device race on it and must be serialised by the
 *    caller.
 * Errors: ARG (null pointer, bad nrhs/ld, unknown prec), STATE (no boundary
 * set), CAPACITY, CUDA.  Asynchronous. */
cpm_status cpm_apply_noalloc(cpm_ctx *ctx, double m, double n, int prec, const void *u_dev, void *v_dev, int nrhs,
                             int64_t ld, void *stream);

/* Size in bytes of cpm_apply_noalloc's fixed intermediate array. */
size_t cpm_apply_noalloc_max_bytes(void);

/* v = A^T u, the transpose of cpm_apply's operator (the adjoint of Sec. 5.4's
 * product, needed for gradients of losses of the solution).  Same arguments,
 * precisions and layouts as cpm_apply.  Computed as gathers, without atomics:
 * b = (n/h^2) F_S^T u over the unflipped FD entries, then per node E^T b from the
 * rows of the stencil cells that hold it, plus per-column lists of the flipped FD
 * and E entries and of the BC-row entries built in cpm_set_boundary.  Its
 * intermediate b lives in the context's reserved scratch.  Asynchronous.
 * Errors: ARG, STATE (no boundary set), CAPACITY, CUDA. */
cpm_status cpm_apply_transpose(cpm_ctx *ctx, double m, double n, int prec, const void *u_dev, void *v_dev, int nrhs,
                               int64_t ld, void *stream);

/* a = E u on the PDE rows (Eq. 1 with the flips of Eq. 10): the side-correct
 * surface values at cp_S(x_i).  FP64, a_dev [N_S] (or [N_S][ld]).  Asynchronous. */
cpm_status cpm_extend(cpm_ctx *ctx, const double *u_dev, double *a_dev, int nrhs, int64_t ld, void *stream);

/* Surface gradient of a field for the heat method's step 2 (Sec. 7.2): at each
 * PDE row, central differences (a(x + h e_d) - a(x - h e_d)) / 2h over the FD
 * neighbours the Laplacian rows use (flipped across curves as in Eq. 11), with
 * a = E u on PDE DOFs and u on BC DOFs; a missing neighbour takes the row's own
 * value.  normalize != 0 returns X = -g / |g| (0 where g = 0).  A BC DOF takes
 * its twin node's value.  u_dev [N], X_dev [N][3] (z = 0 in 2D), FP64.
 * The extension goes to the context's reserved scratch.  Asynchronous. */
cpm_status cpm_surface_gradient(cpm_ctx *ctx, const double *u_dev, double *X_dev, int normalize, void *stream);

/* Surface divergence for the heat method's step 3 right-hand side (Sec. 7.2):
 * b_i = sum_d (X~_d(x_i + h e_d) - X~_d(x_i - h e_d)) / 2h at the PDE rows, with
 * X~ = E X on PDE DOFs and X on BC DOFs, over the same neighbours as above.
 * X_dev [N][3], b_dev [N_S], FP64.  Asynchronous. */
cpm_status cpm_surface_divergence(cpm_ctx *ctx, const double *X_dev, double *b_dev, void *stream);

/* Solves A x = f with diagonal-preconditioned BiCGSTAB (Sec. 5.4), preconditioner
 * diag(m I + n diag L) on PDE rows and 1 on BC rows.  x_dev holds the initial
 * guess on entry.  FP64 mode iterates in FP64.  FP32_IR is mixed-precision
 * iterative refinement: FP32 BiCGSTAB (FP32 operator and Krylov vectors)
 * iterates on the correction equation, the correction accumulated in FP32 and
 * added to x in FP64; whenever a right-hand side's FP32 residual has fallen by
 * inner_tol, the FP64 residual r = f - A x restarts its inner solve in a fresh
 * Krylov space (random shadow residual), and the right-hand side stops once r
 * meets tol.  One whose FP64 residual stops falling is finished by FP64
 * BiCGSTAB from its current iterate, so the result always meets tol in FP64.
 * All right-hand sides of a batch iterate together with their own scalars; every dot product is reduced on the device in a fixed
 * order (results do not depend on scheduling), and groups of check_every
 * iterations are replayed from a captured CUDA graph on the context's internal
 * stream, which is ordered after the caller's prior work on `stream` and before
 * its later work.  Allocates nothing: the workspace for ld must be reserved
 * (cpm_reserve; ld = 1 is reserved by cpm_set_boundary).  Synchronises the
 * internal stream.  stats may be NULL.  Errors: ARG, STATE, CAPACITY, CUDA,
 * BREAKDOWN, NOT_CONVERGED (x holds the last iterate), TIMEOUT (a bounded wait
 * of the fused single right-hand side product, single_mode 2, gave up since
 * the last check; the products since then are void). */
cpm_status cpm_solve(cpm_ctx *ctx, double m, double n, const double *f_dev, double *x_dev, int nrhs, int64_t ld,
                     const cpm_solve_opts *opts, cpm_solve_stats *stats, void *stream);

/* Solves A^T lambda = g (the adjoint system) with the same options.  The
 * iteration is right-preconditioned (A^T W mu = g, lambda = W mu: the transpose
 * of the row-scaled forward system) and tol applies to the unscaled relative
 * residual |g - A^T lambda| / |g| whatever opts->norm says. */
cpm_status cpm_solve_adjoint(cpm_ctx *ctx, double m, double n, const double *g_dev, double *lambda_dev, int nrhs,
                             int64_t ld, const cpm_solve_opts *opts, cpm_solve_stats *stats, void *stream);

/* Gradient of a loss with respect to the Dirichlet samples given the adjoint
 * state lambda (A^T lambda = dL/du): dL/dsamples = B^T (c_alpha lambda_alpha),
 * where B maps samples to g_alpha (periodic linear interpolation per curve and
 * side).  dLds_dev has the samples layout of cpm_rhs.  A fixed-order reduction
 * per sample; allocates nothing.  Asynchronous. */
cpm_status cpm_boundary_grad(cpm_ctx *ctx, const double *lambda_dev, double *dLds_dev, int nrhs, int64_t ld,
                             void *stream);

/* Releases the context and all device memory it owns.  NULL is allowed. */
void cpm_destroy(cpm_ctx *ctx);

/* Static string naming a status code. */
const char *cpm_status_str(cpm_status s);

/* Instrumentation for benchmarks.  enable = 1 resets the counters and starts
 * recording a CUDA event pair around every operator product (forward or
 * transposed, any precision) on the stream it is launched on, and counting
 * the library's kernel launches; enable = 0 stops recording, synchronises,
 * and reports the summed device time of the products (ms), their number, the
 * number of kernel launches since the reset and the number of PDE rows x
 * right-hand sides processed by the products.  Outputs may be NULL.  Paper:
 * no counterpart (measurement only). */
cpm_status cpm_profile(cpm_ctx *ctx, int enable, double *apply_ms, int64_t *apply_calls, int64_t *kernel_launches,
                       int64_t *row_rhs_processed);

/* Launch shapes chosen by cpm_autotune. */
typedef struct {
  int cells_xh;              /* x passes of the batched cell gather (0: the batch width does not use it) */
  int cells_blocks_per_sm;   /* grid cap of the cell gather, blocks of 8 warps per SM (0: default 16) */
  int combine_warps_per_sm;  /* grid cap of the warp-per-row combine (0: default 64) */
  int vec_blocks_per_sm;     /* blocks of 512 threads per SM of the Krylov vector kernels (1, 2 or 4) */
  int single_mode;           /* single right-hand side product: 0 = per-cell gather then combine (default),
                              * 1 = per-row gather then combine, 2 = fused persistent kernel (its bounded
                              * waits set a device flag if they give up, which the next solve reports
                              * as CPM_ERR_TIMEOUT) */
  double product_ms;         /* one operator product with the chosen shapes */
  double product_ms_default; /* the same with the built-in defaults */
  double vector_ms;          /* one two-product reduction over [N][ld] with the chosen blocks */
} cpm_tune_info;

/* Autotuner of the launch shapes.  Times, on this context's band and with
 * nrhs right-hand sides of leading dimension ld in precision prec, the
 * candidate shapes of the batched product (x passes of the cell gather, its
 * grid, the combine's grid) and of the Krylov vector kernels (blocks per SM),
 * by coordinate descent, and keeps the fastest in the context for every later
 * product and solve (a later call for another width or precision refines
 * them).  Uses the reserved solve workspace as scratch: ld and prec must be
 * reserved (cpm_reserve).  The paper has no counterpart (launch configuration
 * only; every candidate computes the same product).  Synchronises `stream`.
 * info may be NULL.  Errors: ARG, STATE, CAPACITY, CUDA. */
cpm_status cpm_autotune(cpm_ctx *ctx, int nrhs, int64_t ld, int prec, cpm_tune_info *info, void *stream);

/* Sets the launch shapes directly (for instance to reuse a tuned choice in a
 * new context of the same band, or to exercise one candidate): cells_xh applies
 * to batches of nrhs columns in precision prec; cells_blocks_per_sm,
 * combine_warps_per_sm, vec_blocks_per_sm and single_mode to every later
 * product and solve.  A zero field restores that field's default; the timing
 * fields are ignored.  Host-only, no stream work.  Errors: ARG (an x pass count
 * that does not divide the stencil width or that the precision does not hold in
 * registers, a grid cap outside 1..256, vec_blocks_per_sm outside 0..4,
 * single_mode outside 0..2), STATE (before cpm_set_boundary). */
cpm_status cpm_set_tune(cpm_ctx *ctx, int nrhs, int prec, const cpm_tune_info *info);

/* Measured arithmetic peaks of the current device, the denominators of the
 * products' rooflines (no counterpart in the paper): TFLOP/s of FP32 FMA
 * instructions, of packed-pair FP32 FMAs (two per instruction) and of FP64 FMAs,
 * from chains of independent FMAs in registers over 8 blocks of 256 threads per
 * SM, timed with CUDA events on the default stream after one warm-up launch.
 * Allocates and frees a small output buffer; synchronises the device's default
 * stream.  Any pointer may be NULL.  Errors: CUDA. */
cpm_status cpm_measure_fma_peak(double *fp32_tflops, double *fp32_pair_tflops, double *fp64_tflops);

/* Diagnostics: counts of crossing-test flips that found no BC twin (Sec. 4.2;
 * zero on smooth geometry within interpolation reach) and of special rows. */
cpm_status cpm_diagnostics(const cpm_ctx *ctx, int64_t *noflip_twin, int64_t *n_special_rows);

#ifdef __cplusplus
}
#endif

#endif /* CPM_H */
