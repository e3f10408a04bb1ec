// Quadrature-point kernel of the explicit comparison path: the stress with the original
// tensor viscosity mu_exp (paper Sec. 3.4, the equation for mu_exp, whose ingredients the
// paper takes from Dobrev et al. 2012, Sec. 6.2):
//   (lambda_1, s_1)  smallest eigenvalue of eps(v) = sym(grad v) and its unit eigenvector,
//   l     = l0 |J J0^-1 s_1|   (the initial length l0 carried along s_1 by dx/dx0),
//   psi_1 = 1 under compression (lambda_1 < 0), else 0,
//   psi_0 = 1, or |div v| / (sqrt(dim) |grad v|_F) with the vorticity switch on,
//   mu    = rho (q2 l^2 |lambda_1| + q1 psi_1 psi_0 l c_s),   sigma = -p I + mu eps(v).
// FP64 throughout (the explicit path is not differentiated).
#pragma once
#include "lh_internal.h"
#include "lh_qp.cuh"

namespace lh {

// Smallest eigenvalue and a unit eigenvector of a symmetric DIM x DIM matrix.  2D: closed
// form.  3D: the trigonometric solution of the characteristic cubic (Smith 1961), then the
// eigenvector as the largest cross product of two rows of A - lambda_1 I.
template <int DIM>
__device__ __forceinline__ void sym_min_eig(const double (&A)[DIM][DIM], double& lam, double (&s)[DIM]) {
  if constexpr (DIM == 2) {
    const double a = A[0][0], b = A[0][1], c = A[1][1];
    const double hd = 0.5 * (a - c);
    const double r = sqrt(hd * hd + b * b);
    lam = 0.5 * (a + c) - r;
    // (a - lam, b) and (b, c - lam) are the rows of A - lam I; each row's normal solves it
    const double v1x = b, v1y = -(a - lam), v2x = c - lam, v2y = -b;
    const double n1 = v1x * v1x + v1y * v1y, n2 = v2x * v2x + v2y * v2y;
    if (n1 <= 0.0 && n2 <= 0.0) {
      s[0] = 1.0;
      s[1] = 0.0;
      return;
    }
    const bool one = n1 >= n2;
    const double inv = 1.0 / sqrt(one ? n1 : n2);
    s[0] = (one ? v1x : v2x) * inv;
    s[1] = (one ? v1y : v2y) * inv;
  } else {
    const double p1 = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double q = (A[0][0] + A[1][1] + A[2][2]) / 3.0;
    const double p2 = (A[0][0] - q) * (A[0][0] - q) + (A[1][1] - q) * (A[1][1] - q) +
                      (A[2][2] - q) * (A[2][2] - q) + 2.0 * p1;
    const double p = sqrt(p2 / 6.0);
    if (!(p > 0.0)) {
      lam = q;
      s[0] = 1.0;
      s[1] = s[2] = 0.0;
      return;
    }
    double B[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) B[i][j] = (A[i][j] - (i == j ? q : 0.0)) / p;
    const double detB = B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) -
                        B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
                        B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
    const double r = fmin(fmax(0.5 * detB, -1.0), 1.0);
    const double phi = acos(r) / 3.0;
    lam = q + 2.0 * p * cos(phi + 2.0 * 3.14159265358979323846 / 3.0);
    double M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] = A[i][j] - (i == j ? lam : 0.0);
    double best[3] = {1.0, 0.0, 0.0}, bn = 0.0;
    const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int t = 0; t < 3; ++t) {
      const double* x = M[pr[t][0]];
      const double* y = M[pr[t][1]];
      const double c0 = x[1] * y[2] - x[2] * y[1], c1 = x[2] * y[0] - x[0] * y[2], c2 = x[0] * y[1] - x[1] * y[0];
      const double n = c0 * c0 + c1 * c1 + c2 * c2;
      if (n > bn) {
        bn = n;
        best[0] = c0;
        best[1] = c1;
        best[2] = c2;
      }
    }
    const double inv = bn > 0.0 ? 1.0 / sqrt(bn) : 1.0;
    for (int i = 0; i < 3; ++i) s[i] = best[i] * inv;
  }
}

// Forward point kernel with mu_exp: outputs as qp_forward (S = alpha detJ sigma J^-T,
// E = alpha detJ sigma : grad v, detJ) plus the viscosity coefficient and rho.
template <int DIM>
__device__ __forceinline__ void qp_forward_exp(const double (&J)[DIM][DIM], const double (&Gv)[DIM][DIM], double e,
                                               const QpC<double>& c, const ExpC& x, double (&So)[DIM][DIM],
                                               double& Eo, double& detJ, double& mu_out, double& rho_out) {
  double A[DIM][DIM];
  const double det = det_adj<DIM>(J, A);
  detJ = det;
  const double inv_det = 1.0 / det;
  double Jinv[DIM][DIM];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) Jinv[i][j] = A[i][j] * inv_det;
  const double W = c.alpha * det;
  const double rho = c.mq / W;
  const double sq = sqrt(e * e + c.eps2);
  const double ep = e >= 0.0 ? 0.5 * (e + sq) : 0.5 * c.eps2 / (sq - e);   // Eq. (19)
  const double p = c.gm1 * rho * ep;                                         // Eq. (20)
  const double cs = sqrt(c.ggm1 * ep);
  double Lv[DIM][DIM];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) {
      double t = 0.0;
      for (int r = 0; r < DIM; ++r) t += Gv[i][r] * Jinv[r][j];
      Lv[i][j] = t;
    }
  double sig[DIM][DIM];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) sig[i][j] = i == j ? -p : 0.0;
  double mu = 0.0;
  if (c.visc) {
    double eps[DIM][DIM];
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) eps[i][j] = 0.5 * (Lv[i][j] + Lv[j][i]);
    double lam, s1[DIM];
    sym_min_eig<DIM>(eps, lam, s1);
    double l2 = 0.0;
    for (int i = 0; i < DIM; ++i) {
      double t = 0.0;
      for (int j = 0; j < DIM; ++j) t += J[i][j] * (x.inv_h[j] * s1[j]);
      l2 += t * t;
    }
    const double ell = x.l0 * sqrt(l2);
    double psi0 = 1.0;
    if (x.vorticity) {
      double fn = 0.0, div = 0.0;
      for (int i = 0; i < DIM; ++i) {
        div += Lv[i][i];
        for (int j = 0; j < DIM; ++j) fn += Lv[i][j] * Lv[i][j];
      }
      if (fn > 0.0) psi0 = fabs(div) / (sqrt((double)DIM) * sqrt(fn));
    }
    const double psi1 = lam < 0.0 ? 1.0 : 0.0;
    mu = rho * (x.q2 * ell * ell * fabs(lam) + x.q1 * psi1 * psi0 * ell * cs);
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) sig[i][j] += mu * eps[i][j];
  }
  double E = 0.0;
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) {
      E += sig[i][j] * Lv[i][j];
      double t = 0.0;
      for (int b = 0; b < DIM; ++b) t += sig[i][b] * Jinv[j][b];
      So[i][j] = W * t;
    }
  Eo = W * E;
  mu_out = mu;
  rho_out = rho;
}

}  // namespace lh
