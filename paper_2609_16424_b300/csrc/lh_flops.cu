// Exact operation counts of the quadrature-point kernels (measurement support).
//
// The templated quadrature-point code of lh_qp.cuh is run on the host with a counting
// scalar: every +, -, *, / and every sqrt, tanh, cbrt, cos, sin counts one operation
// (negation counts none).  The counts feed the algorithmic FLOP totals that the
// benchmark divides by measured kernel time.
#include <cmath>
#include "../../include/lh.h"

// the counting scalar is host-only; the templated kernel code it runs is host+device
#pragma nv_diag_suppress 20011
#pragma nv_diag_suppress 20014

namespace {

long long g_ops = 0;

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double a) : v(a) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }   // branches are not counted
inline Cnt& operator+=(Cnt& a, Cnt b) { ++g_ops; a.v += b.v; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { ++g_ops; a.v -= b.v; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { ++g_ops; a.v *= b.v; return a; }
// found by argument-dependent lookup from the templated kernel code
inline Cnt lsqrt(Cnt a) { ++g_ops; return Cnt(std::sqrt(a.v)); }
inline Cnt ltanh(Cnt a) { ++g_ops; return Cnt(std::tanh(a.v)); }
inline Cnt lcbrt(Cnt a) { ++g_ops; return Cnt(std::cbrt(a.v)); }
inline Cnt lcos(Cnt a) { ++g_ops; return Cnt(std::cos(a.v)); }
inline Cnt lsin(Cnt a) { ++g_ops; return Cnt(std::sin(a.v)); }

}  // namespace

#include "lh_qp.cuh"

namespace {

using lh::Dual;
using lh::QpC;

QpC<Cnt> consts(bool visc) {
  QpC<Cnt> c;
  c.mq = 0.01; c.alpha = 0.1; c.inv_detJ0 = 1000.0; c.gm1 = 0.4; c.ggm1 = 0.56;
  c.h0 = 0.1; c.inv_hc = 10.0; c.q1 = 0.5; c.q2 = 1.0; c.scoef = 0.0; c.eps2 = 1e-12;
  c.visc = visc;
  return c;
}

template <int DIM>
long long count(int kind, bool visc) {
  const QpC<Cnt> c = consts(visc);
  g_ops = 0;
  if (kind == 0) {
    Cnt J[DIM][DIM], Gv[DIM][DIM], S[DIM][DIM], E, det;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        J[i][j] = i == j ? 0.1 : 0.01;
        Gv[i][j] = 0.1 * (i + 1) - 0.05 * j;
      }
    g_ops = 0;
    lh::qp_forward<DIM>(J, Gv, Cnt(2.0), c, S, E, det);
  } else if (kind == 1) {
    Dual<Cnt> J[DIM][DIM], Gv[DIM][DIM], S[DIM][DIM], E, det;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        J[i][j] = Dual<Cnt>(i == j ? 0.1 : 0.01, 0.001);
        Gv[i][j] = Dual<Cnt>(0.1 * (i + 1) - 0.05 * j, 0.01);
      }
    g_ops = 0;
    lh::qp_forward<DIM>(J, Gv, Dual<Cnt>(Cnt(2.0), Cnt(0.1)), c, S, E, det);
  } else if (kind == 3) {   // tangent from the linearisation record (reduced-precision J.w)
    Cnt L[lh::lin_len<DIM>()], dJ[DIM][DIM], dGv[DIM][DIM], dS[DIM][DIM], dE, dW;
    for (int f = 0; f < lh::lin_len<DIM>(); ++f) L[f] = 0.1 + 0.01 * f;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        dJ[i][j] = 0.001 * (i + j + 1);
        dGv[i][j] = 0.01 * (i - j);
      }
    g_ops = 0;
    lh::qp_tangent_lin<DIM, Cnt>(L, dJ, dGv, Cnt(0.1), Cnt(0.5), Cnt(1.0), visc, dS, dE, dW);
  } else {
    Cnt J[DIM][DIM], Gv[DIM][DIM], Sb[DIM][DIM], Jb[DIM][DIM], Gvb[DIM][DIM], eb;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        J[i][j] = i == j ? 0.1 : 0.01;
        Gv[i][j] = 0.1 * (i + 1) - 0.05 * j;
        Sb[i][j] = 0.3;
      }
    g_ops = 0;
    lh::qp_adjoint<DIM>(J, Gv, Cnt(2.0), c, Sb, Cnt(0.2), Cnt(0.0), Jb, Gvb, eb);
  }
  return g_ops;
}

}  // namespace

extern "C" lh_status lh_qp_flops(int dim, int kind, int visc, long long* ops) {
  if (!ops || (dim != 2 && dim != 3) || kind < 0 || kind > 3) return LH_EINVAL;
  *ops = dim == 2 ? count<2>(kind, visc != 0) : count<3>(kind, visc != 0);
  return LH_OK;
}
