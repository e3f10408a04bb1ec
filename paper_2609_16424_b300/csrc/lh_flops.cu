// Exact operation counts of the quadrature-point kernels (measurement support).
//
// The templated quadrature-point code of lh_qp.cuh is run on the host with a counting
// scalar: every +, -, *, / and every sqrt, tanh, cbrt, cos, sin counts one operation
// (negation counts none).  The counts feed the algorithmic FLOP totals that the
// benchmark divides by measured kernel time.
#include <algorithm>
#include <cmath>
#include <vector>
#include "../../include/lh.h"

// the counting scalar is host-only; the templated kernel code it runs is host+device
#pragma nv_diag_suppress 20011
#pragma nv_diag_suppress 20014

namespace {

long long g_ops = 0;
// per-kind counts (kind 4 weighs them by the float operations of the double-word arithmetic)
long long g_add = 0, g_mul = 0, g_div = 0, g_sqrt = 0, g_tanh = 0, g_cbrt = 0;

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double a) : v(a) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops; ++g_add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops; ++g_add; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops; ++g_mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops; ++g_div; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }   // branches are not counted
inline Cnt& operator+=(Cnt& a, Cnt b) { ++g_ops; ++g_add; a.v += b.v; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { ++g_ops; ++g_add; a.v -= b.v; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { ++g_ops; ++g_mul; a.v *= b.v; return a; }
// found by argument-dependent lookup from the templated kernel code
inline Cnt lsqrt(Cnt a) { ++g_ops; ++g_sqrt; return Cnt(std::sqrt(a.v)); }
inline Cnt ltanh(Cnt a) { ++g_ops; ++g_tanh; return Cnt(std::tanh(a.v)); }
inline Cnt lcbrt(Cnt a) { ++g_ops; ++g_cbrt; return Cnt(std::cbrt(a.v)); }
inline Cnt lcos(Cnt a) { ++g_ops; return Cnt(std::cos(a.v)); }
inline Cnt lsin(Cnt a) { ++g_ops; return Cnt(std::sin(a.v)); }

}  // namespace

#include "lh_qp.cuh"

namespace {

using lh::Dual;
using lh::QpC;

// float operations (+, -, *, fma, /, sqrt, cbrt, rint, ldexp: one each) of the double-word
// primitives of lh_dd.cuh: sum 2 TwoSum + 2 FastTwoSum + 2 adds; product TwoProd + 2 + 1 +
// FastTwoSum; quotient 2 divisions + product + sum + FastTwoSum; square and cube roots one
// Newton correction; tanh = exp (range reduction, degree-12 Horner) + sum, difference, quotient
constexpr long long kDwAdd = 20, kDwMul = 8, kDwDiv = 33, kDwSqrt = 28, kDwCbrt = 36;
constexpr long long kDwTanh = 8 + (2 + 22 + 22 + 21 + 12 * (kDwMul + kDwAdd) + 2) + 2 * kDwAdd + kDwDiv;

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
  if (kind == 0 || kind == 4) {
    Cnt J[DIM][DIM], Gv[DIM][DIM], S[DIM][DIM], E, det;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        J[i][j] = i == j ? 0.1 : 0.01;
        Gv[i][j] = 0.1 * (i + 1) - 0.05 * j;
      }
    g_ops = g_add = g_mul = g_div = g_sqrt = g_tanh = g_cbrt = 0;
    lh::qp_forward<DIM>(J, Gv, Cnt(2.0), c, S, E, det);
    if (kind == 4)   // float operations of the same code in double-word arithmetic (lh_dd.cuh)
      return g_add * kDwAdd + g_mul * kDwMul + g_div * kDwDiv + g_sqrt * kDwSqrt + g_cbrt * kDwCbrt +
             g_tanh * kDwTanh;
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

extern "C" lh_status lh_record_len(int dim, int* len) {
  if (!len || (dim != 2 && dim != 3)) return LH_EINVAL;
  *len = dim == 2 ? lh::lin_len<2>() : lh::lin_len<3>();
  return LH_OK;
}

extern "C" lh_status lh_qp_flops(int dim, int kind, int visc, long long* ops) {
  if (!ops || (dim != 2 && dim != 3) || kind < 0 || kind > 4) return LH_EINVAL;
  *ops = dim == 2 ? count<2>(kind, visc != 0) : count<3>(kind, visc != 0);
  return LH_OK;
}

// ---- host check of the linearised tangent (lin_record + qp_tangent_lin) against the
// dual-number tangent of qp_forward on random states near the undeformed element
namespace {
struct Lcg {
  unsigned long long s;
  double next() {   // uniform in [-1, 1)
    s = s * 6364136223846793005ULL + 1442695040888963407ULL;
    return (double)(s >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
};
template <int DIM>
void tangent_check(bool visc, int trials, unsigned seed, double* max_double, double* median_float) {
  lh::QpC<double> c;
  c.alpha = 0.3; c.mq = 1.3 * 0.3 * 0.002; c.inv_detJ0 = 500.0; c.gm1 = 0.4; c.ggm1 = 0.56;
  c.h0 = 0.05; c.inv_hc = 20.0; c.q1 = 0.5; c.q2 = 1.0; c.scoef = 0.3; c.eps2 = 1e-12; c.visc = visc;
  Lcg g{0x9E3779B97F4A7C15ULL ^ seed};
  std::vector<double> ef;
  double md = 0.0;
  const double s = DIM == 3 ? 0.126 : 0.045;
  for (int tr = 0; tr < trials; ++tr) {
    double J[DIM][DIM], Gv[DIM][DIM], dJ[DIM][DIM], dGv[DIM][DIM];
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        J[i][j] = s * ((i == j) + 0.2 * g.next());
        Gv[i][j] = g.next();
        dJ[i][j] = 0.01 * s * g.next();
        dGv[i][j] = g.next();
      }
    const double e = g.next(), de = g.next();
    lh::Dual<double> Jd[DIM][DIM], Gd[DIM][DIM], Sd[DIM][DIM], Ed, dd;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        Jd[i][j] = lh::Dual<double>(J[i][j], dJ[i][j]);
        Gd[i][j] = lh::Dual<double>(Gv[i][j], dGv[i][j]);
      }
    lh::qp_forward<DIM>(Jd, Gd, lh::Dual<double>(e, de), c, Sd, Ed, dd);
    double So[DIM][DIM], Eo, det;
    lh::QpPrimal<DIM, double> pr;
    lh::qp_forward<DIM>(J, Gv, e, c, So, Eo, det, &pr);
    double Ld[lh::lin_len<DIM>()], dSd[DIM][DIM], dEd, dWd;
    lh::lin_record<DIM, double>(pr, c.gm1, c.q1, c.q2, visc, 0, 0, 0, Ld);
    lh::qp_tangent_lin<DIM, double>(Ld, dJ, dGv, de, c.q1, c.q2, visc, dSd, dEd, dWd);
    float Lf[lh::lin_len<DIM>()], dJf[DIM][DIM], dGf[DIM][DIM], dSf[DIM][DIM], dEf, dWf;
    lh::lin_record<DIM, float>(pr, c.gm1, (float)c.q1, (float)c.q2, visc, 0, 0, 0, Lf);
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        dJf[i][j] = (float)dJ[i][j];
        dGf[i][j] = (float)dGv[i][j];
      }
    lh::qp_tangent_lin<DIM, float>(Lf, dJf, dGf, (float)de, (float)c.q1, (float)c.q2, visc, dSf, dEf, dWf);
    double n = 0.0, nd = 0.0, nf = 0.0;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        n += Sd[i][j].d * Sd[i][j].d;
        nd += (dSd[i][j] - Sd[i][j].d) * (dSd[i][j] - Sd[i][j].d);
        nf += (dSf[i][j] - Sd[i][j].d) * (dSf[i][j] - Sd[i][j].d);
      }
    const double rd = std::max({std::sqrt(nd / n), std::fabs(dEd - Ed.d) / std::fabs(Ed.d),
                                std::fabs(dWd - c.alpha * dd.d) / std::fabs(c.alpha * dd.d)});
    md = std::max(md, rd);
    ef.push_back(std::sqrt(nf / n));
  }
  std::sort(ef.begin(), ef.end());
  *max_double = md;
  *median_float = ef[ef.size() / 2];
}
}  // namespace

extern "C" lh_status lh_qp_tangent_check(int dim, int visc, int trials, unsigned seed, double* max_err_double,
                                         double* median_err_float) {
  if (!max_err_double || !median_err_float || (dim != 2 && dim != 3) || trials < 1) return LH_EINVAL;
  if (dim == 2) tangent_check<2>(visc != 0, trials, seed, max_err_double, median_err_float);
  else tangent_check<3>(visc != 0, trials, seed, max_err_double, median_err_float);
  return LH_OK;
}

// ---- host check of the transposed linearised map: <L x, yb> = <x, L^T yb> on random data
namespace {
template <int DIM>
double adjoint_check(bool visc, int trials, unsigned seed) {
  Lcg g{0x51ED270B27A8D5A1ULL ^ seed};
  double worst = 0.0;
  for (int tr = 0; tr < trials; ++tr) {
    double L[lh::lin_len<DIM>()];
    for (int f = 0; f < lh::lin_len<DIM>(); ++f) L[f] = g.next();
    double dJ[DIM][DIM], dGv[DIM][DIM], Sb[DIM][DIM], dS[DIM][DIM], Jb[DIM][DIM], Gvb[DIM][DIM];
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        dJ[i][j] = g.next();
        dGv[i][j] = g.next();
        Sb[i][j] = g.next();
      }
    const double de = g.next(), Eb = g.next(), Wb = g.next();
    double dE, dW, eb;
    lh::qp_tangent_lin<DIM, double>(L, dJ, dGv, de, 0.5, 1.0, visc, dS, dE, dW);
    lh::qp_tangent_lin_adj<DIM, double>(L, Sb, Eb, Wb, 0.5, 1.0, visc, Jb, Gvb, eb);
    double lhs = dE * Eb + dW * Wb, rhs = de * eb, scale = std::fabs(dE * Eb) + std::fabs(dW * Wb) + std::fabs(de * eb);
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        lhs += dS[i][j] * Sb[i][j];
        rhs += dJ[i][j] * Jb[i][j] + dGv[i][j] * Gvb[i][j];
        scale += std::fabs(dS[i][j] * Sb[i][j]) + std::fabs(dJ[i][j] * Jb[i][j]) + std::fabs(dGv[i][j] * Gvb[i][j]);
      }
    worst = std::max(worst, std::fabs(lhs - rhs) / scale);
  }
  return worst;
}
}  // namespace

extern "C" lh_status lh_qp_adjoint_check(int dim, int visc, int trials, unsigned seed, double* max_rel) {
  if (!max_rel || (dim != 2 && dim != 3) || trials < 1) return LH_EINVAL;
  *max_rel = dim == 2 ? adjoint_check<2>(visc != 0, trials, seed) : adjoint_check<3>(visc != 0, trials, seed);
  return LH_OK;
}

// ---- host check of the double-word arithmetic and of the residual's point kernel in it
namespace {
double rel(double got, double ref) { return std::fabs(got - ref) / std::fmax(std::fabs(ref), 1e-300); }

template <int DIM>
double dd_point_check(bool visc, int trials, Lcg& g) {
  lh::QpC<double> c;
  c.alpha = 0.3; c.mq = 1.3 * 0.3 * 0.002; c.inv_detJ0 = 500.0; c.gm1 = 0.4; c.ggm1 = 0.56;
  c.h0 = 0.05; c.inv_hc = 20.0; c.q1 = 0.5; c.q2 = 1.0; c.scoef = 0.3; c.eps2 = 1e-12; c.visc = visc;
  lh::QpC<lh::DD> cd;
  cd.alpha = lh::DD(c.alpha); cd.mq = lh::DD(c.mq); cd.inv_detJ0 = lh::DD(c.inv_detJ0); cd.gm1 = lh::DD(c.gm1);
  cd.ggm1 = lh::DD(c.ggm1); cd.h0 = lh::DD(c.h0); cd.inv_hc = lh::DD(c.inv_hc); cd.q1 = lh::DD(c.q1);
  cd.q2 = lh::DD(c.q2); cd.scoef = lh::DD(c.scoef); cd.eps2 = lh::DD(c.eps2); cd.visc = visc;
  const double s = DIM == 3 ? 0.126 : 0.045;
  double worst = 0.0;
  for (int tr = 0; tr < trials; ++tr) {
    double J[DIM][DIM], Gv[DIM][DIM];
    lh::DD Jd[DIM][DIM], Gd[DIM][DIM];
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        // inputs representable in double-word exactly: round through the pair
        Jd[i][j] = lh::DD(s * ((i == j) + 0.2 * g.next()));
        Gd[i][j] = lh::DD(g.next() * (tr % 3 == 0 ? 30.0 : 1.0));
        J[i][j] = lh::to_double(Jd[i][j]);
        Gv[i][j] = lh::to_double(Gd[i][j]);
      }
    const lh::DD ed = lh::DD(g.next() * (tr % 5 == 0 ? 1e-5 : 2.0));
    const double e = lh::to_double(ed);
    double S[DIM][DIM], E, det;
    lh::DD Sd[DIM][DIM], Ed, detd;
    lh::QpPrimal<DIM, double> pr;
    lh::qp_forward<DIM>(J, Gv, e, c, S, E, det, &pr);
    lh::qp_forward<DIM>(Jd, Gd, ed, cd, Sd, Ed, detd);
    // error scale: the size of the stress terms before cancellation, W |J^-1| (|p| + mu_max |grad v|)
    // with mu_max = rho h (q2 (h |grad v| + delta_s) + q1 c_s); divergence and trace
    // cancellations make any finite precision lose relative accuracy below that scale
    double nj = 0.0, nl = 0.0;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        nj += pr.Jinv[i][j] * pr.Jinv[i][j];
        nl += pr.Lv[i][j] * pr.Lv[i][j];
      }
    nj = std::sqrt(nj);
    nl = std::sqrt(nl);
    const double mu_max = visc ? pr.rho * pr.h * (c.q2 * (pr.h * nl + pr.ds) + c.q1 * pr.cs) : 0.0;
    const double scale = std::fabs(pr.W) * nj * (std::fabs(pr.p) + mu_max * nl);
    double d = 0.0;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        const double x = lh::to_double(Sd[i][j]) - S[i][j];
        d += x * x;
      }
    worst = std::max({worst, std::sqrt(d) / scale, rel(lh::to_double(detd), det),
                      std::fabs(lh::to_double(Ed) - E) / (scale * nl / nj + 1e-300)});
  }
  return worst;
}
}  // namespace

extern "C" lh_status lh_dd_check(int which, int trials, unsigned seed, double* max_err) {
  if (!max_err || trials < 1 || which < 0 || which > 9) return LH_EINVAL;
  Lcg g{0x2545F4914F6CDD1DULL ^ seed};
  double worst = 0.0;
  using lh::DD;
  if (which >= 6) {
    *max_err = which == 6 ? dd_point_check<2>(false, trials, g) : which == 7 ? dd_point_check<2>(true, trials, g)
             : which == 8 ? dd_point_check<3>(false, trials, g) : dd_point_check<3>(true, trials, g);
    return LH_OK;
  }
  for (int t = 0; t < trials; ++t) {
    const double a = g.next() * std::ldexp(1.0, (int)(g.next() * 20)), b = g.next() * std::ldexp(1.0, (int)(g.next() * 20));
    const DD A(a), B(b);
    const double ad = lh::to_double(A), bd = lh::to_double(B);
    switch (which) {
      case 0: {   // sum and difference (relative to the operands' size: cancellation is exact)
        worst = std::max(worst, std::fabs(lh::to_double(A + B) - (ad + bd)) / (std::fabs(ad) + std::fabs(bd)));
        worst = std::max(worst, std::fabs(lh::to_double(A - B) - (ad - bd)) / (std::fabs(ad) + std::fabs(bd)));
        break;
      }
      case 1: worst = std::max(worst, rel(lh::to_double(A * B), ad * bd)); break;
      case 2: worst = std::max(worst, rel(lh::to_double(A / B), ad / bd)); break;
      case 3: worst = std::max(worst, rel(lh::to_double(lh::lsqrt(DD(std::fabs(ad)))), std::sqrt(std::fabs(ad)))); break;
      case 4: worst = std::max(worst, rel(lh::to_double(lh::lcbrt(DD(std::fabs(ad)))), std::cbrt(std::fabs(ad)))); break;
      case 5: {   // tanh on [-25, 25] (absolute error: |tanh| <= 1)
        const DD z(25.0 * g.next());
        worst = std::max(worst, std::fabs(lh::to_double(lh::ltanh(z)) - std::tanh(lh::to_double(z))));
        break;
      }
    }
  }
  *max_err = worst;
  return LH_OK;
}

