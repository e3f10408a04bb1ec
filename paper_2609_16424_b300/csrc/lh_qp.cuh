// Quadrature-point kernel D of the force operator (paper Sec. 2.2, Eq. (8)): stress,
// equation of state and smooth artificial viscosity, with its tangent (via Dual) and a
// hand-written adjoint (reverse mode) for the transpose action.
#pragma once
#include "lh_common.cuh"

namespace lh {

// Per-quadrature-point constants.  Pointwise mass conservation (Sec. 2.1, after Eq. (7))
// makes rho * alpha * detJ = m_q = rho0 * alpha * detJ0 constant in time.
template <class T>
struct QpC {
  T mq;          // rho0 alpha_q detJ0
  T alpha;       // reference quadrature weight
  T inv_detJ0;   // 1 / detJ0 (Eq. (14))
  T gm1;         // gamma - 1           (Eq. (20))
  T ggm1;        // gamma (gamma - 1)   (Eq. (20))
  T h0, inv_hc;  // Eq. (14), (18)
  T q1, q2;      // Eq. (13)
  T scoef;       // 2 atanh(1 - 2 psi0): shift s = scoef * delta_s (Eq. (17))
  T eps2;        // eps_e^2 (Eq. (19))
  bool visc;
};

template <int DIM, class S>
__host__ __device__ __forceinline__ S det_adj(const S (&J)[DIM][DIM], S (&A)[DIM][DIM]) {
  if constexpr (DIM == 2) {
    A[0][0] = J[1][1];
    A[0][1] = -J[0][1];
    A[1][0] = -J[1][0];
    A[1][1] = J[0][0];
    return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  } else {
    A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
  }
}

// Forward quadrature-point kernel.
//   J  = d x / d xhat (reference-to-current Jacobian), Gv = d v / d xhat, e = e(x_q).
//   Outputs S = alpha detJ sigma J^{-T} (so that the H1 force row of node a, component c,
//   is sum_q sum_r S[c][r] d_r w_a), E = alpha detJ sigma : grad v (the L2 row weight),
//   and detJ.
// Works for S = T (residual) and S = Dual<T> (tangent of Eq. (10)).
template <int DIM, class S, class T>
__host__ __device__ __forceinline__ void qp_forward(const S (&J)[DIM][DIM], const S (&Gv)[DIM][DIM], S e,
                                           const QpC<T>& c, S (&So)[DIM][DIM], S& Eo, S& detJ) {
  S A[DIM][DIM];
  const S det = det_adj<DIM>(J, A);
  detJ = det;
  const S inv_det = T(1) / det;
  S Jinv[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) Jinv[i][j] = A[i][j] * inv_det;
  const S W = c.alpha * det;                       // current-domain quadrature weight
  const S rho = c.mq / W;                          // rho = rho0 detJ0 / detJ
  // Eq. (19); for e < 0 the identical expression eps^2 / (2 (sqrt(e^2 + eps^2) - e)) is
  // used, free of the cancellation that would round e+ to 0 for strongly negative e
  const S sq = lsqrt(e * e + c.eps2);
  const S ep = value_of(e) >= T(0) ? T(0.5) * (e + sq) : T(0.5) * c.eps2 / (sq - e);
  const S p = c.gm1 * rho * ep;                    // Eq. (20)
  const S cs = lsqrt(c.ggm1 * ep);                 // Eq. (20)
  S Lv[DIM][DIM];                                  // physical velocity gradient
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      S s = Gv[i][0] * Jinv[0][j];
#pragma unroll
      for (int r = 1; r < DIM; ++r) s = s + Gv[i][r] * Jinv[r][j];
      Lv[i][j] = s;
    }
  S sig[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) sig[i][j] = (i == j) ? -p : S(T(0));
  if (c.visc) {
    const S h = c.h0 * root_dim<DIM>(det * c.inv_detJ0);    // Eq. (14)
    S div = Lv[0][0];
#pragma unroll
    for (int i = 1; i < DIM; ++i) div = div + Lv[i][i];
    const S dv = h * div;                                    // Eq. (15)
    const S ds = (T(2) * c.inv_hc) * (h * cs);               // Eq. (18)
    const S ab = lsqrt(dv * dv + ds * ds);                   // Eq. (16)
    const S arg = (-dv - c.scoef * ds) / (T(2) * ds);
    const S psi = T(0.5) + T(0.5) * ltanh(arg);              // Eq. (17)
    const S mu = rho * h * (c.q2 * ab + c.q1 * cs * psi);    // Eq. (13)
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int j = 0; j < DIM; ++j) sig[i][j] = sig[i][j] + mu * (T(0.5) * (Lv[i][j] + Lv[j][i]));  // Eq. (11)
  }
  S E = sig[0][0] * Lv[0][0];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      if (i || j) E = E + sig[i][j] * Lv[i][j];
      S s = sig[i][0] * Jinv[j][0];
#pragma unroll
      for (int b = 1; b < DIM; ++b) s = s + sig[i][b] * Jinv[j][b];
      So[i][j] = W * s;
    }
  Eo = W * E;
}

// Taylor-Green manufactured energy source per unit volume (gamma = 5/3):
//   s = (3 pi / 8) [cos 3 pi x cos pi y - cos pi x cos 3 pi y]
template <class S, class T>
__host__ __device__ __forceinline__ S tg_source(S x, S y) {
  const T pi = T(3.14159265358979323846);
  return (T(3) * pi / T(8)) * (lcos(T(3) * pi * x) * lcos(pi * y) - lcos(pi * x) * lcos(T(3) * pi * y));
}

template <class T>
__host__ __device__ __forceinline__ void tg_source_grad(T x, T y, T& sx, T& sy) {
  const T pi = T(3.14159265358979323846);
  const T c = T(3) * pi / T(8);
  sx = c * (-T(3) * pi * lsin(T(3) * pi * x) * lcos(pi * y) + pi * lsin(pi * x) * lcos(T(3) * pi * y));
  sy = c * (-pi * lcos(T(3) * pi * x) * lsin(pi * y) + T(3) * pi * lcos(pi * x) * lsin(T(3) * pi * y));
}

// Reverse mode of qp_forward: given the output adjoints Sb (of S) and Eb (of E) and an
// extra adjoint detb_in on detJ, return Jb, Gvb, eb.  Hand-written: the primal is
// recomputed, then each statement of qp_forward is transposed in reverse order.
template <int DIM, class T>
__host__ __device__ __forceinline__ void qp_adjoint(const T (&J)[DIM][DIM], const T (&Gv)[DIM][DIM], T e,
                                           const QpC<T>& c, const T (&Sb)[DIM][DIM], T Eb, T detb_in,
                                           T (&Jb)[DIM][DIM], T (&Gvb)[DIM][DIM], T& eb) {
  // ---- primal
  T A[DIM][DIM];
  const T det = det_adj<DIM>(J, A);
  const T inv_det = T(1) / det;
  T Jinv[DIM][DIM];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) Jinv[i][j] = A[i][j] * inv_det;
  const T W = c.alpha * det;
  const T rho = c.mq / W;
  const T sq = lsqrt(e * e + c.eps2);
  const T ep = e >= T(0) ? T(0.5) * (e + sq) : T(0.5) * c.eps2 / (sq - e);
  const T p = c.gm1 * rho * ep;
  const T cs = lsqrt(c.ggm1 * ep);
  T Lv[DIM][DIM];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) {
      T s = 0;
      for (int r = 0; r < DIM; ++r) s += Gv[i][r] * Jinv[r][j];
      Lv[i][j] = s;
    }
  T h = 0, div = 0, dv = 0, ds = 0, ab = 0, t = 0, psi = 0, X = 0, mu = 0;
  T sig[DIM][DIM];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) sig[i][j] = (i == j) ? -p : T(0);
  if (c.visc) {
    h = c.h0 * root_dim<DIM>(det * c.inv_detJ0);
    for (int i = 0; i < DIM; ++i) div += Lv[i][i];
    dv = h * div;
    ds = T(2) * c.inv_hc * h * cs;
    ab = lsqrt(dv * dv + ds * ds);
    const T arg = (-dv - c.scoef * ds) / (T(2) * ds);
    t = ltanh(arg);
    psi = T(0.5) + T(0.5) * t;
    X = c.q2 * ab + c.q1 * cs * psi;
    mu = rho * h * X;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) sig[i][j] += mu * T(0.5) * (Lv[i][j] + Lv[j][i]);
  }
  // ---- reverse
  T sigb[DIM][DIM], Lvb[DIM][DIM], Jinvb[DIM][DIM];
  T Wb = 0, sigL = 0;
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) {
      sigL += sig[i][j] * Lv[i][j];
      sigb[i][j] = Eb * W * Lv[i][j];           // E = W sig : Lv
      Lvb[i][j] = Eb * W * sig[i][j];
    }
  Wb += Eb * sigL;
  for (int i = 0; i < DIM; ++i)                 // S_ir = W sum_b sig_ib Jinv_rb
    for (int r = 0; r < DIM; ++r) {
      T s = 0;
      for (int b = 0; b < DIM; ++b) s += sig[i][b] * Jinv[r][b];
      Wb += Sb[i][r] * s;
    }
  for (int i = 0; i < DIM; ++i)
    for (int b = 0; b < DIM; ++b) {
      T s = 0;
      for (int r = 0; r < DIM; ++r) s += Sb[i][r] * Jinv[r][b];
      sigb[i][b] += W * s;
    }
  for (int r = 0; r < DIM; ++r)
    for (int b = 0; b < DIM; ++b) {
      T s = 0;
      for (int i = 0; i < DIM; ++i) s += Sb[i][r] * sig[i][b];
      Jinvb[r][b] = W * s;
    }
  T pb = 0;                                     // sig = -p I + mu sym(Lv)
  for (int i = 0; i < DIM; ++i) pb -= sigb[i][i];
  T rhob = 0, csb = 0, detb = detb_in;
  if (c.visc) {
    T mub = 0;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        mub += sigb[i][j] * T(0.5) * (Lv[i][j] + Lv[j][i]);
      }
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) Lvb[i][j] += mu * T(0.5) * (sigb[i][j] + sigb[j][i]);
    rhob += mub * h * X;                        // mu = rho h X
    T hb = mub * rho * X;
    const T Xb = mub * rho * h;
    const T abb = Xb * c.q2;                    // X = q2 ab + q1 cs psi
    csb += Xb * c.q1 * psi;
    const T psib = Xb * c.q1 * cs;
    const T argb = T(0.5) * psib * (T(1) - t * t);   // psi = 1/2 + tanh(arg)/2
    T dvb = -argb / (T(2) * ds);                // arg = -dv/(2 ds) - scoef/2
    T dsb = argb * dv / (T(2) * ds * ds);
    dvb += abb * dv / ab;                       // ab = sqrt(dv^2 + ds^2)
    dsb += abb * ds / ab;
    hb += dsb * T(2) * c.inv_hc * cs;           // ds = 2 h cs / h_coarse
    csb += dsb * T(2) * c.inv_hc * h;
    hb += dvb * div;                            // dv = h div
    const T divb = dvb * h;
    for (int i = 0; i < DIM; ++i) Lvb[i][i] += divb;
    detb += hb * h / (T(DIM) * det);            // h = h0 (det / detJ0)^(1/DIM)
  }
  T epb = csb * c.ggm1 / (T(2) * cs);           // cs = sqrt(g(g-1) ep)
  rhob += pb * c.gm1 * ep;                      // p = (g-1) rho ep
  epb += pb * c.gm1 * rho;
  // d e+ / d e = (1 + e / sq) / 2, written as eps^2 / (2 sq (sq - e)) for e < 0
  eb = epb * (e >= T(0) ? T(0.5) * (T(1) + e / sq) : T(0.5) * c.eps2 / (sq * (sq - e)));
  for (int i = 0; i < DIM; ++i)                 // Lv = Gv Jinv
    for (int r = 0; r < DIM; ++r) {
      T s = 0;
      for (int b = 0; b < DIM; ++b) s += Lvb[i][b] * Jinv[r][b];
      Gvb[i][r] = s;
    }
  for (int r = 0; r < DIM; ++r)
    for (int b = 0; b < DIM; ++b) {
      T s = 0;
      for (int i = 0; i < DIM; ++i) s += Gv[i][r] * Lvb[i][b];
      Jinvb[r][b] += s;
    }
  Wb += -rhob * rho / W;                        // rho = m_q / W
  detb += Wb * c.alpha;                         // W = alpha det
  for (int a = 0; a < DIM; ++a)                 // Jinv = J^{-1}; det = det(J)
    for (int b = 0; b < DIM; ++b) {
      T s = 0;
      for (int r = 0; r < DIM; ++r)
        for (int q = 0; q < DIM; ++q) s += Jinv[r][a] * Jinvb[r][q] * Jinv[b][q];
      Jb[a][b] = -s + detb * det * Jinv[b][a];
    }
}

}  // namespace lh
