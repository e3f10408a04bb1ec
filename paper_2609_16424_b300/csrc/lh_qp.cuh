// Quadrature-point kernel D of the force operator (paper Sec. 2.2, Eq. (8)): stress,
// equation of state and smooth artificial viscosity, with its tangent (via Dual) and a
// hand-written adjoint (reverse mode) for the transpose action.
#pragma once
#include "lh_common.cuh"
#include "lh_dd.cuh"
#if defined(__CUDACC__)
#include "lh_f2.cuh"
#endif

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

// Primal intermediates of qp_forward at one point (filled on request by the residual
// kernel, from which the linearisation record of the tangent is formed).
template <int DIM, class T>
struct QpPrimal {
  T Jinv[DIM][DIM], Lv[DIM][DIM];
  T W, rho, sq, ep, p, cs;
  T h, ds, ab, t, mu;
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
                                           const QpC<T>& c, S (&So)[DIM][DIM], S& Eo, S& detJ,
                                           QpPrimal<DIM, T>* prim = nullptr) {
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
  if (prim) {
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        prim->Jinv[i][j] = value_of(Jinv[i][j]);
        prim->Lv[i][j] = value_of(Lv[i][j]);
      }
    prim->W = value_of(W);
    prim->rho = value_of(rho);
    prim->sq = value_of(sq);
    prim->ep = value_of(ep);
    prim->p = value_of(p);
    prim->cs = value_of(cs);
    prim->h = prim->ds = prim->ab = prim->t = prim->mu = T(0);
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
    const S th = ltanh(arg);
    const S psi = T(0.5) + T(0.5) * th;                      // Eq. (17)
    const S mu = rho * h * (c.q2 * ab + c.q1 * cs * psi);    // Eq. (13)
    if (prim) {
      prim->h = value_of(h);
      prim->ds = value_of(ds);
      prim->ab = value_of(ab);
      prim->t = value_of(th);
      prim->mu = value_of(mu);
    }
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

// ---- Linearisation record of the quadrature-point map (partial assembly of the tangent,
// paper Sec. 2.2: the point data are stored once per Newton iterate and reused by every
// Jacobian action).  Fields per point, float:
//   [0, D^2) J^-1, [D^2, 2 D^2) grad v, then W = alpha detJ, p, pe = (gamma-1) rho e+',
//   mu, and the three coefficients of the linearised viscosity chain of Eqs. (13)-(18),
//   dmu = a_th theta + a_div d(div v) + a_e de  (theta = tr(J^-1 dJ) = d detJ / detJ);
//   in 2D also the Taylor-Green source s and its gradient at x_q.
// The chain (tq = theta / dim, e+' = e+ / sqrt(e^2 + eps^2) in both branches of Eq. (19),
// ke = e+' / (2 e+) = 1 / (2 sqrt(e^2 + eps^2)), rh = rho h, delta_v = h div v):
//   d delta_v = tq delta_v + h d(div v),   d delta_s = delta_s (tq + ke de),
//   d|.|  = tq |.| + (delta_v h d(div v) + delta_s^2 ke de) / |.|,
//   d arg = -(h d(div v) - delta_v ke de) / (2 delta_s),   d psi = (1 - t^2)/2 d arg,
//   dmu   = mu (1/dim - 1) theta + rh [q2 d|.| + q1 (c_s ke psi de + c_s d psi)]
// collects into
//   a_th  = mu (1/dim - 1) + rh q2 |.| / dim = rh (q2 |.| (2/dim - 1) + q1 c_s psi (1/dim - 1)),
//   a_div = rh h (q2 delta_v / |.| - q1 c_s (1 - t^2) / (4 delta_s)),
//   a_e   = rh ke (q2 delta_s^2 / |.| + q1 c_s psi + q1 c_s (1 - t^2) delta_v / (4 delta_s)),
// formed from the residual's own intermediates.
template <int DIM>
__host__ __device__ constexpr int lin_len() { return DIM == 3 ? 25 : 18; }

enum LinField : int { LF_W = 0, LF_P, LF_PE, LF_MU, LF_ATH, LF_ADIV, LF_AE, LF_TGS, LF_TGX, LF_TGY };

// conversion of a primal intermediate (double or double-word) to the record's precision
template <class R>
__host__ __device__ __forceinline__ R rcv(double x) { return R(x); }
template <class R>
__host__ __device__ __forceinline__ R rcv(const DD& x) {
  if constexpr (sizeof(R) == sizeof(float)) return x.hi;   // hi is x rounded to float
  else return R(to_double(x));
}

template <int DIM, class R = float, class PT = double>
__host__ __device__ __forceinline__ void lin_record(const QpPrimal<DIM, PT>& pr, PT gm1, R q1, R q2, bool visc,
                                                    double tgs, double tgx, double tgy, R (&L)[lin_len<DIM>()]) {
  constexpr int O = 2 * DIM * DIM;
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      L[i * DIM + j] = rcv<R>(pr.Jinv[i][j]);
      L[DIM * DIM + i * DIM + j] = rcv<R>(pr.Lv[i][j]);
    }
  // the chain is formed in the record's precision R (float on the GPU), from the primal
  // intermediates rounded once; 1 - t^2 and psi in the primal precision (1 - t^2 cancels)
  const R isq = R(1) / rcv<R>(pr.sq);
  L[O + LF_W] = rcv<R>(pr.W);
  L[O + LF_P] = rcv<R>(pr.p);
  L[O + LF_PE] = rcv<R>(gm1 * pr.rho) * rcv<R>(pr.ep) * isq;
  if (visc) {
    PT div = pr.Lv[0][0];
#pragma unroll
    for (int i = 1; i < DIM; ++i) div = div + pr.Lv[i][i];
    const R h = rcv<R>(pr.h), dv = rcv<R>(pr.h * div), rh = rcv<R>(pr.rho * pr.h), ds = rcv<R>(pr.ds);
    const R ab = rcv<R>(pr.ab), cs = rcv<R>(pr.cs);
    const R ke = R(0.5) * isq, iab = R(1) / ab;
    const R g4 = rcv<R>(PT(0.25) * (PT(1) - pr.t * pr.t)) / ds;   // (1 - t^2) / (4 delta_s)
    const R psi = rcv<R>(PT(0.5) + PT(0.5) * pr.t);
    L[O + LF_MU] = rcv<R>(pr.mu);
    // a_th = mu (1/dim - 1) + rh q2 |.| / dim with mu = rh (q2 |.| + q1 c_s psi), cancellation-free
    L[O + LF_ATH] = rh * (q2 * ab * R(2.0 / DIM - 1.0) + q1 * cs * psi * R(1.0 / DIM - 1.0));
    L[O + LF_ADIV] = rh * h * (q2 * dv * iab - q1 * cs * g4);
    L[O + LF_AE] = rh * ke * (q2 * ds * ds * iab + q1 * cs * (psi + g4 * dv));
  } else {
    L[O + LF_MU] = L[O + LF_ATH] = L[O + LF_ADIV] = L[O + LF_AE] = R(0);
  }
  if constexpr (DIM == 2) {
    L[O + LF_TGS] = R(tgs);
    L[O + LF_TGX] = R(tgx);
    L[O + LF_TGY] = R(tgy);
  }
}

// Tangent of qp_forward from the record: given dJ = d(grad_hat x), dGv = d(grad_hat v), de,
// returns dS, dE and dW = d(alpha detJ).  With theta = tr(J^-1 dJ) (= d detJ / detJ):
//   d grad v = (dGv - grad v dJ) J^-1,  drho = -rho theta,  dp = -p theta + pe de,
//   dcs = cs ke de,  dh = h theta / dim,  and the chain of Eqs. (13)-(18) for dmu;
//   dsigma = -dp I + dmu eps(grad v) + mu eps(d grad v),
//   dS = W [theta sigma + dsigma - sigma J^-T dJ^T] J^-T,
//   dE = W [theta sigma : grad v + dsigma : grad v + sigma : d grad v].
template <int DIM, class T = float>
__host__ __device__ __forceinline__ void qp_tangent_lin(const T (&L)[lin_len<DIM>()], const T (&dJ)[DIM][DIM],
                                                        const T (&dGv)[DIM][DIM], T de, T q1, T q2,
                                                        bool visc, T (&dSo)[DIM][DIM], T& dEo, T& dW) {
  constexpr int O = 2 * DIM * DIM;
  T Ji[DIM][DIM], Lv[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      Ji[i][j] = L[i * DIM + j];
      Lv[i][j] = L[DIM * DIM + i * DIM + j];
    }
  const T W = L[O + LF_W], p = L[O + LF_P];
  T th = T(0.);
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r) th += Ji[i][r] * dJ[r][i];
  T dL[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    T Y[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      T y = dGv[i][r];
#pragma unroll
      for (int b = 0; b < DIM; ++b) y -= Lv[i][b] * dJ[b][r];
      Y[r] = y;
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      T v = T(0.);
#pragma unroll
      for (int r = 0; r < DIM; ++r) v += Y[r] * Ji[r][j];
      dL[i][j] = v;
    }
  }
  const T dp = -p * th + L[O + LF_PE] * de;
  T mu = T(0.), dmu = T(0.);
  if (visc) {
    T ddiv = dL[0][0];
#pragma unroll
    for (int i = 1; i < DIM; ++i) ddiv += dL[i][i];
    mu = L[O + LF_MU];
    dmu = L[O + LF_ATH] * th + L[O + LF_ADIV] * ddiv + L[O + LF_AE] * de;
  }
  T sg[DIM][DIM], dsg[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const T ep = T(0.5) * (Lv[i][j] + Lv[j][i]), dep = T(0.5) * (dL[i][j] + dL[j][i]);
      sg[i][j] = (i == j ? -p : T(0.)) + mu * ep;
      dsg[i][j] = (i == j ? -dp : T(0.)) + dmu * ep + mu * dep;
    }
  T E = T(0.), dE = T(0.);
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      E += sg[i][j] * Lv[i][j];
      dE += dsg[i][j] * Lv[i][j] + sg[i][j] * dL[i][j];
    }
  dEo = W * (th * E + dE);
  dW = W * th;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    T M[DIM], N[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {   // M = sigma J^-T (row i)
      T v = T(0.);
#pragma unroll
      for (int k = 0; k < DIM; ++k) v += sg[i][k] * Ji[b][k];
      M[b] = v;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {   // N = theta sigma + dsigma - M dJ^T (row i)
      T v = th * sg[i][a] + dsg[i][a];
#pragma unroll
      for (int b = 0; b < DIM; ++b) v -= M[b] * dJ[a][b];
      N[a] = v;
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      T v = T(0.);
#pragma unroll
      for (int a = 0; a < DIM; ++a) v += N[a] * Ji[j][a];
      dSo[i][j] = W * v;
    }
  }
}

#if defined(__CUDACC__)
// qp_tangent_lin for two quadrature points at once (paired FP32 operations, lh_f2.cuh), in
// the form the record J.w uses: dJ and dGv are the reference gradients of the direction's
// x and v fields (not yet multiplied by tau), de its energy value, and tW = tau W.  The map
// is linear in (dJ, dGv, de), so scaling W by tau scales every output by tau.  sigma and
// d sigma are symmetric: only i <= j is formed.
template <int DIM>
__device__ __forceinline__ void qp_tangent_lin_x2(const float2 (&L)[lin_len<DIM>()], const float2 (&dJ)[DIM][DIM],
                                                  const float2 (&dGv)[DIM][DIM], float2 de, float2 tW, bool visc,
                                                  float2 (&dSo)[DIM][DIM], float2& dEo, float2& dW) {
  constexpr int O = 2 * DIM * DIM;
  auto Ji = [&](int i, int j) -> const float2& { return L[i * DIM + j]; };
  auto Lv = [&](int i, int j) -> const float2& { return L[DIM * DIM + i * DIM + j]; };
  // theta = tr(J^-1 dJ)
  float2 th = f2mul(Ji(0, 0), dJ[0][0]);
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r)
      if (i + r > 0) th = f2fma(Ji(i, r), dJ[r][i], th);
  // d grad v = (dGv - grad v dJ) J^-1
  float2 dL[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    float2 Y[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      float2 y = dGv[i][r];
#pragma unroll
      for (int b = 0; b < DIM; ++b) y = f2fma(f2neg(Lv(i, b)), dJ[b][r], y);
      Y[r] = y;
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      float2 v = f2mul(Y[0], Ji(0, j));
#pragma unroll
      for (int r = 1; r < DIM; ++r) v = f2fma(Y[r], Ji(r, j), v);
      dL[i][j] = v;
    }
  }
  const float2 np = f2neg(L[O + LF_P]);
  const float2 dp = f2fma(np, th, f2mul(L[O + LF_PE], de));
  float2 mu = f2s(0.f), dmu = f2s(0.f);
  if (visc) {
    float2 ddiv = dL[0][0];
#pragma unroll
    for (int i = 1; i < DIM; ++i) ddiv = f2add(ddiv, dL[i][i]);
    mu = L[O + LF_MU];
    dmu = f2fma(L[O + LF_AE], de, f2fma(L[O + LF_ADIV], ddiv, f2mul(L[O + LF_ATH], th)));
  }
  const float2 ndp = f2neg(dp);
  float2 sg[DIM][DIM], dsg[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = i; j < DIM; ++j) {
      if (i == j) {
        sg[i][i] = f2fma(mu, Lv(i, i), np);
        dsg[i][i] = f2fma(mu, dL[i][i], f2fma(dmu, Lv(i, i), ndp));
      } else {
        const float2 ep = f2mul(f2s(0.5f), f2add(Lv(i, j), Lv(j, i)));
        const float2 dep = f2mul(f2s(0.5f), f2add(dL[i][j], dL[j][i]));
        sg[i][j] = sg[j][i] = f2mul(mu, ep);
        dsg[i][j] = dsg[j][i] = f2fma(mu, dep, f2mul(dmu, ep));
      }
    }
  float2 E = f2s(0.f), dE = f2s(0.f);
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      E = (i + j == 0) ? f2mul(sg[0][0], Lv(0, 0)) : f2fma(sg[i][j], Lv(i, j), E);
      dE = (i + j == 0) ? f2mul(dsg[0][0], Lv(0, 0)) : f2fma(dsg[i][j], Lv(i, j), dE);
      dE = f2fma(sg[i][j], dL[i][j], dE);
    }
  dEo = f2mul(tW, f2fma(th, E, dE));
  dW = f2mul(tW, th);
  float2 nsg[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = i; j < DIM; ++j) nsg[i][j] = nsg[j][i] = f2neg(sg[i][j]);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    float2 nM[DIM], N[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {   // -M = -sigma J^-T (row i)
      float2 v = f2mul(nsg[i][0], Ji(b, 0));
#pragma unroll
      for (int k = 1; k < DIM; ++k) v = f2fma(nsg[i][k], Ji(b, k), v);
      nM[b] = v;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {   // N = theta sigma + d sigma - M dJ^T (row i)
      float2 v = f2fma(th, sg[i][a], dsg[i][a]);
#pragma unroll
      for (int b = 0; b < DIM; ++b) v = f2fma(nM[b], dJ[a][b], v);
      N[a] = v;
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      float2 v = f2mul(N[0], Ji(j, 0));
#pragma unroll
      for (int a = 1; a < DIM; ++a) v = f2fma(N[a], Ji(j, a), v);
      dSo[i][j] = f2mul(tW, v);
    }
  }
}
#endif

// Transpose of qp_tangent_lin (the adjoint of the linearised point map, for the
// reduced-precision J^T y): given the adjoints Sb of dS, Eb of dE and Wb of dW, returns the
// adjoints Jb of dJ, Gvb of dGv and eb of de.  Each statement of qp_tangent_lin is
// transposed in reverse order; the map is linear, so only record values enter.
template <int DIM, class T = float>
__host__ __device__ __forceinline__ void qp_tangent_lin_adj(const T (&L)[lin_len<DIM>()], const T (&Sb)[DIM][DIM],
                                                            T Eb, T Wb, T q1, T q2, bool visc,
                                                            T (&Jb)[DIM][DIM], T (&Gvb)[DIM][DIM], T& eb) {
  constexpr int O = 2 * DIM * DIM;
  T Ji[DIM][DIM], Lv[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      Ji[i][j] = L[i * DIM + j];
      Lv[i][j] = L[DIM * DIM + i * DIM + j];
      Jb[i][j] = T(0);
    }
  const T W = L[O + LF_W], p = L[O + LF_P];
  const T mu = visc ? L[O + LF_MU] : T(0);
  // primal stress, strain rate and their products
  T sg[DIM][DIM], ep[DIM][DIM], E = T(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      ep[i][j] = T(0.5) * (Lv[i][j] + Lv[j][i]);
      sg[i][j] = (i == j ? -p : T(0)) + mu * ep[i][j];
    }
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) E += sg[i][j] * Lv[i][j];
  // dS = W N J^-T  ->  Nb = W Sb J^-1
  T Nb[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      T v = T(0);
#pragma unroll
      for (int j = 0; j < DIM; ++j) v += Sb[i][j] * Ji[j][a];
      Nb[i][a] = W * v;
    }
  // dE = W (theta E + dE_in), dW = W theta
  T thb = W * E * Eb + W * Wb;
  const T dEinb = W * Eb;
  // N = theta sg + dsg - M dJ^T,  M = sg J^-T
  T dsgb[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    T M[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      T v = T(0);
#pragma unroll
      for (int k = 0; k < DIM; ++k) v += sg[i][k] * Ji[b][k];
      M[b] = v;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      thb += Nb[i][a] * sg[i][a];
      dsgb[i][a] = Nb[i][a] + dEinb * Lv[i][a];          // also from dE_in = dsg : grad v
#pragma unroll
      for (int b = 0; b < DIM; ++b) Jb[a][b] -= Nb[i][a] * M[b];
    }
  }
  // dE_in also = sg : dL;  dsg = -dp I + dmu eps + mu eps(dL)
  T dLb[DIM][DIM];
  T dpb = T(0), dmub = T(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    dpb -= dsgb[i][i];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      dmub += dsgb[i][j] * ep[i][j];
      dLb[i][j] = dEinb * sg[i][j] + mu * T(0.5) * (dsgb[i][j] + dsgb[j][i]);
    }
  }
  T ebv = T(0);
  if (visc) {   // dmu = a_th theta + a_div tr(dL) + a_e de
    thb += L[O + LF_ATH] * dmub;
    ebv += L[O + LF_AE] * dmub;
    const T ddivb = L[O + LF_ADIV] * dmub;
#pragma unroll
    for (int i = 0; i < DIM; ++i) dLb[i][i] += ddivb;
  }
  // dp = -p theta + pe de
  thb += -p * dpb;
  ebv += L[O + LF_PE] * dpb;
  // dL = Y J^-1 -> Yb = dLb J^-T;  Y = dGv - grad v dJ
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      T v = T(0);
#pragma unroll
      for (int j = 0; j < DIM; ++j) v += dLb[i][j] * Ji[r][j];
      Gvb[i][r] = v;
    }
#pragma unroll
  for (int b = 0; b < DIM; ++b)
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      T v = T(0);
#pragma unroll
      for (int i = 0; i < DIM; ++i) v += Gvb[i][r] * Lv[i][b];
      Jb[b][r] -= v;
    }
  // theta = sum_{i,r} J^-1[i][r] dJ[r][i]
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r) Jb[r][i] += thb * Ji[i][r];
  eb = ebv;
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
