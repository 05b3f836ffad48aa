// bumpy.cuh -- closest points to the bumpy sphere |x| = rho(x/|x|) by the
// two-stage projection of App. A, in FP64 on the device.
//
// phi(x) = |x| - rho(u), u = x/|x|, rho(u) = 1 + amp sum_k a_k exp(-|u - c_k|^2/width).
// With s = |x|, P = I - u u^T, g = grad_u rho, H = Hess_u rho and q = P g:
//   grad phi = u - q/s,   D^2 phi = P/s - [P H P - u q^T - q u^T - (u.g) P]/s^2.
// Stage 1: cp <- cp - phi grad/|grad|^2 until the step is below 1e-10.
// Stage 2: Newton on f(cp, lam) = |cp - x|^2/2 + lam phi(cp), lam_0 from stage 1,
// until |dy| < 1e-10.  Both stages stop after s.newton_maxit (200) iterations
// with failure.
#pragma once

namespace cpm_bumpy {

__device__ inline void bumpy_eval(const ShapeDev &s, const double *x, double *phi, double grad[3], double hess[9]) {
  double sn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double u[3] = {x[0] / sn, x[1] / sn, x[2] / sn};
  double rho = 1.0, g[3] = {0, 0, 0}, H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double iw = 1.0 / s.width;
  for (int k = 0; k < s.K; ++k) {
    double d[3] = {u[0] - s.c[3 * k], u[1] - s.c[3 * k + 1], u[2] - s.c[3 * k + 2]};
    double e = exp(-(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * iw);
    double coef = s.amp * s.a[k] * e;
    rho += coef;
    for (int i = 0; i < 3; ++i) g[i] += coef * (-2.0 * iw) * d[i];
    if (hess)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[3 * i + j] += coef * (4.0 * iw * iw * d[i] * d[j] - (i == j ? 2.0 * iw : 0.0));
  }
  *phi = sn - rho;
  double P[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[3 * i + j] = (i == j ? 1.0 : 0.0) - u[i] * u[j];
  double q[3];
  for (int i = 0; i < 3; ++i) q[i] = P[3 * i] * g[0] + P[3 * i + 1] * g[1] + P[3 * i + 2] * g[2];
  for (int i = 0; i < 3; ++i) grad[i] = u[i] - q[i] / sn;
  if (!hess) return;
  double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
  double PH[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) PH[3 * i + j] = P[3 * i] * H[j] + P[3 * i + 1] * H[3 + j] + P[3 * i + 2] * H[6 + j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double php = PH[3 * i] * P[j] + PH[3 * i + 1] * P[3 + j] + PH[3 * i + 2] * P[6 + j];
      hess[3 * i + j] = P[3 * i + j] / sn - (php - u[i] * q[j] - q[i] * u[j] - ug * P[3 * i + j]) / (sn * sn);
    }
}

// 4x4 Gaussian elimination with partial pivoting; returns nonzero if singular
__device__ inline int solve4(double A[16], double b[4], double x[4]) {
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

}  // namespace cpm_bumpy

__device__ inline int cpm_cp_bumpy(const ShapeDev &s, const double *x, double *cp) {
  using namespace cpm_bumpy;
  double y[3] = {x[0], x[1], x[2]}, phi, gr[3], H[9];
  int it;
  const int maxit = s.newton_maxit;
  for (it = 0; it < maxit; ++it) {
    bumpy_eval(s, y, &phi, gr, nullptr);
    double g2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    double st[3] = {phi * gr[0] / g2, phi * gr[1] / g2, phi * gr[2] / g2};
    y[0] -= st[0]; y[1] -= st[1]; y[2] -= st[2];
    if (sqrt(st[0] * st[0] + st[1] * st[1] + st[2] * st[2]) < 1e-10) break;
  }
  if (it == maxit) return 1;
  bumpy_eval(s, y, &phi, gr, nullptr);
  double lam = ((x[0] - y[0]) * gr[0] + (x[1] - y[1]) * gr[1] + (x[2] - y[2]) * gr[2]) /
               (gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
  for (it = 0; it < maxit; ++it) {
    bumpy_eval(s, y, &phi, gr, H);
    double J[16], F[4], dy[4];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) J[4 * i + j] = (i == j ? 1.0 : 0.0) + lam * H[3 * i + j];
      J[4 * i + 3] = gr[i];
      J[12 + i] = gr[i];
      F[i] = (y[i] - x[i]) + lam * gr[i];
    }
    J[15] = 0.0;
    F[3] = phi;
    if (solve4(J, F, dy)) return 1;
    y[0] -= dy[0]; y[1] -= dy[1]; y[2] -= dy[2];
    lam -= dy[3];
    if (sqrt(dy[0] * dy[0] + dy[1] * dy[1] + dy[2] * dy[2] + dy[3] * dy[3]) < 1e-10) break;
  }
  if (it == maxit) return 1;
  cp[0] = y[0]; cp[1] = y[1]; cp[2] = y[2];
  return 0;
}
