// Element kernels (residual, tangent, adjoint, mass) and node-centric H1 assembly.
//
// Operator decomposition of paper Sec. 2.2, Eq. (8), A = P^T G^T B^T D B G P, with P = I
// on one GPU.  Element kernels fuse G (gather from the node lattice by index arithmetic),
// B (sum-factorised contractions, lh_contract.cuh), D (quadrature-point kernel, lh_qp.cuh)
// and B^T; they write element vectors of the H1 rows to a scratch buffer and L2 rows
// (element-local, G = I) directly.  G^T is a separate node-centric kernel that sums the
// up to 2^dim element contributions of each node in a fixed order (deterministic, no
// atomics).
#include <cfloat>
#include "lh_internal.h"
#include "lh_kernels.h"
#include "lh_qp.cuh"
#include "lh_contract.cuh"
#include "lh_elem.cuh"
#include "lh_tc.cuh"

namespace lh {

// =====================================================================================
// Residual: H1 rows (M_V k_v + F(w).1) to the element scratch, L2 rows
// (M_E k_e - F(w)^T w_v - b) directly, per-block min det J.
template <int DIM, int K>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_residual(ElemParams P, const double* __restrict__ u, const double* __restrict__ kk, double tau,
           double* __restrict__ ev, double* __restrict__ Re, double* __restrict__ blockmin,
           float* __restrict__ rec) {
  // Element contractions (DF) and the quadrature-point kernel (DD) in double-word arithmetic
  // on the FP32 pipe; gathers, the element outputs and the det J minimum in FP64.  Positions
  // enter the contractions relative to the element's first node (the reference gradients of
  // the basis sum to zero, so J is unchanged), which keeps J accurate to ~2^-46 relative on
  // fine meshes.
  using C = Cfg<DIM, K>;
  constexpr int D = C::D, Q = C::Q, ND = C::ND, NL = C::NL, NQ = C::NQ;
  constexpr int NCH = 2 * DIM;
  using PL = Plan<DIM, K, NCH, DIM, 2, DIM>;
  using TB = Tab<K>;
  static_assert(sizeof(DF) == sizeof(double), "the shared-memory plan counts 8-byte entries");
  extern __shared__ double smem[];
  DF* sdf = reinterpret_cast<DF*>(smem);
  const DF* sB = sdf + TB::B;
  const DF* sG = sdf + TB::G;
  const DF* sBl = sdf + TB::BL;
  const DF* sW = sdf + TB::W;
  double* red = smem + TB::SMEM;
  for (int i = threadIdx.x; i < TB::SMEM; i += blockDim.x) sdf[i] = DF(P.tab[i]);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  DF* s_h = sdf + PL::HEAD + eb * PL::PER;   // [2 DIM][ND]: w_x - w_x(node 0), w_v
  DF* s_kv = s_h + NCH * ND;                 // [DIM][ND]: k_v
  DF* s_l = s_kv + DIM * ND;                 // [2][NL]: w_e, k_e
  // [3] per element: rho0 detJ0, gamma - 1, gamma (gamma - 1), in the reduction buffer (which
  // the final det J minimum overwrites only after many barriers)
  DF* s_c = reinterpret_cast<DF*>(red) + 3 * eb;
  DF* t1 = s_l + 2 * NL;
  DF* t2 = t1 + PL::T1;
  DF* sf = t2 + PL::T2;
  const ElemIdx E = elem_index<DIM, K>(P);
  double x0[DIM];   // position of the element's first node at w = u + tau k
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    x0[c] = 0.0;
    if (E.valid) {
      const long long g = c * P.NV + node_of<DIM, K>(P, E, 0);
      x0[c] = u[g] + tau * kk[g];
    }
  }
  for (int i = lt; i < NCH * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    double v = 0.0;
    if (E.valid) {
      const long long g = comp * P.NV + node_of<DIM, K>(P, E, a);
      v = u[g] + tau * kk[g];
      if (comp < DIM) v -= x0[comp];
    }
    s_h[i] = DF(v);
  }
  for (int i = lt; i < DIM * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    s_kv[i] = DF(E.valid ? kk[(DIM + comp) * P.NV + node_of<DIM, K>(P, E, a)] : 0.0);
  }
  for (int i = lt; i < NL; i += NQ) {
    double we = 0.0, ke = 0.0;
    if (E.valid) {
      const long long g = 2 * DIM * P.NV + E.e * NL + i;
      ke = kk[g];
      we = u[g] + tau * ke;
    }
    s_l[i] = DF(we);
    s_l[NL + i] = DF(ke);
  }
  if (lt == 0) {   // per-element material constants, split once per element
    const double rho0 = E.valid ? P.rho0[E.e] : 1.0, gam = E.valid ? P.gamma[E.e] : 1.4;
    s_c[0] = DF(rho0 * P.detJ0);
    s_c[1] = DF(gam - 1.0);
    s_c[2] = DF(gam * (gam - 1.0));
  }
  __syncthreads();
  DF hvd[NCH], hgd[NCH][DIM];
  // positions at the quadrature points are only needed by the 2D Taylor-Green source
  h1_fwd<DIM, K, NCH, DF, DIM == 2>(s_h, t1, t2, sB, sG, lt, hvd, hgd);
  DF kvd[DIM];
  l2_fwd<DIM, K, DIM, DF, D>(s_kv, t1, t2, sB, lt, kvd);
  DF lqd[2];
  l2_fwd<DIM, K, 2, DF>(s_l, t1, t2, sBl, lt, lqd);
  // quadrature-point constants in double-word (mesh constants split on the host)
  QpC<DD> c;
  {
    const int q0 = lt % Q, q1 = (lt / Q) % Q, q2 = lt / (Q * Q);
    DD a = dd_of(sW[q0]) * dd_of(sW[q1]);
    if constexpr (DIM == 3) a = a * dd_of(sW[q2]);
    c.alpha = a;
    c.mq = dd_of(s_c[0]) * a;
    c.gm1 = dd_of(s_c[1]);
    c.ggm1 = dd_of(s_c[2]);
    c.inv_detJ0 = DD(P.dw_inv_detJ0[0], P.dw_inv_detJ0[1]);
    c.h0 = DD(P.dw_h0[0], P.dw_h0[1]);
    c.inv_hc = DD(P.dw_inv_hc[0], P.dw_inv_hc[1]);
    c.q1 = DD(P.dw_q1[0], P.dw_q1[1]);
    c.q2 = DD(P.dw_q2[0], P.dw_q2[1]);
    c.scoef = DD(P.dw_scoef[0], P.dw_scoef[1]);
    c.eps2 = DD(P.dw_eps2[0], P.dw_eps2[1]);
    c.visc = P.visc != 0;
  }
  DD J[DIM][DIM], Gv[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      J[i][r] = dd_of(hgd[i][r]);
      Gv[i][r] = dd_of(hgd[DIM + i][r]);
    }
  if (!E.valid) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) J[i][i] = DD(1.f);   // keep the idle lanes finite
  }
  DD So[DIM][DIM], Eo, detJd;
  QpPrimal<DIM, DD> pr;
  qp_forward<DIM>(J, Gv, dd_of(lqd[0]), c, So, Eo, detJd, rec ? &pr : nullptr);
  const double detJ = to_double(detJd);
  double hv[DIM];
#pragma unroll
  for (int cc = 0; cc < DIM; ++cc) hv[cc] = DIM == 2 ? to_double(hvd[cc]) + x0[cc] : 0.0;
  if (rec && E.valid) {   // linearisation record of the tangent (float, [NE][fields][NQ])
    double tgs = 0.0, tgx = 0.0, tgy = 0.0;
    if constexpr (DIM == 2) {
      if (P.tg) {
        tgs = tg_source<double, double>(hv[0], hv[1]);
        tg_source_grad<double>(hv[0], hv[1], tgx, tgy);
      }
    }
    float L[lin_len<DIM>()];
    lin_record<DIM, float, DD>(pr, c.gm1, P.fq1, P.fq2, c.visc, tgs, tgx, tgy, L);
    float* rq = rec + E.e * lin_len<DIM>() * NQ + lt;
#pragma unroll
    for (int f = 0; f < lin_len<DIM>(); ++f) rq[f * NQ] = L[f];
  }
  DF fval[DIM], Sd[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    fval[i] = df_of(c.mq * dd_of(kvd[i]));
#pragma unroll
    for (int r = 0; r < DIM; ++r) Sd[i][r] = df_of(So[i][r]);
  }
  DD g = c.mq * dd_of(lqd[1]) - Eo;
  if constexpr (DIM == 2) {
    if (P.tg) g = g - c.alpha * detJd * DD(tg_source<double, double>(hv[0], hv[1]));
  }
  h1_bwd<DIM, K, DIM>(fval, Sd, sf, t1, t2, sB, sG, lt, s_h);
  if (E.valid)
    for (int i = lt; i < DIM * ND; i += NQ) ev[E.e * (DIM * ND) + i] = to_double(s_h[i]);
  DF gv[1] = {df_of(g)};
  l2_bwd<DIM, K, 1>(gv, sf, t1, t2, sBl, lt, s_l);
  if (E.valid)
    for (int i = lt; i < NL; i += NQ) Re[E.e * NL + i] = to_double(s_l[i]);
  const double m = block_min(E.valid ? detJ : DBL_MAX, red);
  if (threadIdx.x == 0) blockmin[blockIdx.x] = m;
}

// =====================================================================================
// Jacobian action (tangent of the residual along dw = tau dk, plus the mass terms).
// State gathered in double; in float mode positions are re-centred on the element's
// first node before rounding so that J keeps full float accuracy.
template <int DIM, int K, class T, class TO>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_jvp(ElemParams P, const double* __restrict__ u, const double* __restrict__ kk, double tau,
      const T* __restrict__ dk, T* __restrict__ ev, TO* __restrict__ oute) {
  using C = Cfg<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ;
  constexpr int NCH = 4 * DIM;   // w_x, w_v, dk_x, dk_v
  using PL = Plan<DIM, K, NCH, 0, 2, DIM>;
  using TB = Tab<K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  T* sB = smem + TB::B;
  T* sG = smem + TB::G;
  T* sBl = smem + TB::BL;
  T* sW = smem + TB::W;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  T* s_h = smem + PL::HEAD + eb * PL::PER;
  T* s_l = s_h + NCH * ND;
  T* t1 = s_l + 2 * NL;
  T* t2 = t1 + PL::T1;
  T* sf = t2 + PL::T2;
  const ElemIdx E = elem_index<DIM, K>(P);
  // element origin for the re-centring of positions
  double org[DIM];
#pragma unroll
  for (int cc = 0; cc < DIM; ++cc) {
    org[cc] = 0.0;
    if (E.valid && sizeof(T) < sizeof(double)) {
      const long long g = cc * P.NV + node_of<DIM, K>(P, E, 0);
      org[cc] = u[g] + tau * kk[g];
    }
  }
  for (int i = lt; i < NCH * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    T v = T(0);
    if (E.valid) {
      const long long nd = node_of<DIM, K>(P, E, a);
      if (comp < 2 * DIM) {
        const long long g = comp * P.NV + nd;
        double w = u[g] + tau * kk[g];
        if (comp < DIM) w -= org[comp];
        v = T(w);
      } else {
        v = dk[(comp - 2 * DIM) * P.NV + nd];
      }
    }
    s_h[i] = v;
  }
  for (int i = lt; i < NL; i += NQ) {
    T we = T(0), de = T(0);
    if (E.valid) {
      const long long g = 2 * DIM * P.NV + E.e * NL + i;
      we = T(u[g] + tau * kk[g]);
      de = dk[g];
    }
    s_l[i] = we;
    s_l[NL + i] = de;
  }
  __syncthreads();
  T hv[NCH], hg[NCH][DIM];
  h1_fwd<DIM, K, NCH>(s_h, t1, t2, sB, sG, lt, hv, hg);
  T lq[2];
  l2_fwd<DIM, K, 2>(s_l, t1, t2, sBl, lt, lq);

  const QpC<T> c = qp_consts<DIM, K, T>(P, E, sW, lt);
  const T tf = T(tau);
  Dual<T> J[DIM][DIM], Gv[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      J[i][r] = Dual<T>(hg[i][r], tf * hg[2 * DIM + i][r]);
      Gv[i][r] = Dual<T>(hg[DIM + i][r], tf * hg[3 * DIM + i][r]);
    }
  if (!E.valid) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) J[i][i] = Dual<T>(T(1), T(0));
  }
  Dual<T> So[DIM][DIM], Eo, detJ;
  qp_forward<DIM>(J, Gv, Dual<T>(lq[0], tf * lq[1]), c, So, Eo, detJ);
  T fval[DIM], fgrad[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    fval[i] = c.mq * hv[3 * DIM + i];
#pragma unroll
    for (int r = 0; r < DIM; ++r) fgrad[i][r] = So[i][r].d;
  }
  T g = c.mq * lq[1] - Eo.d;
  if constexpr (DIM == 2) {
    if (P.tg) {
      const Dual<T> xq(T(org[0]) + hv[0], tf * hv[2 * DIM + 0]);
      const Dual<T> yq(T(org[1]) + hv[1], tf * hv[2 * DIM + 1]);
      const Dual<T> ws = c.alpha * detJ * tg_source<Dual<T>, T>(xq, yq);
      g -= ws.d;
    }
  }
  h1_bwd<DIM, K, DIM>(fval, fgrad, sf, t1, t2, sB, sG, lt, s_h);
  if (E.valid)
    for (int i = lt; i < DIM * ND; i += NQ) ev[E.e * (DIM * ND) + i] = s_h[i];
  T gv[1] = {g};
  l2_bwd<DIM, K, 1>(gv, sf, t1, t2, sBl, lt, s_l);
  if (E.valid)
    for (int i = lt; i < NL; i += NQ) oute[E.e * NL + i] = TO(s_l[i]);
}

// =====================================================================================
// FP32 Jacobian action from the linearisation record: the direction dk is gathered and
// contracted, and the linearised point map stored by the FP64 residual at the same w
// (lh_qp.cuh, lin_record / qp_tangent_lin) turns its reference gradients and values into
// the stress and energy tangents; no point-kernel re-evaluation.
template <int DIM, int K, class TO>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_jvp_rec(ElemParams P, const float* __restrict__ rec, float tau, const float* __restrict__ dk,
          float* __restrict__ ev, TO* __restrict__ oute) {
  using C = Cfg<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ, Q = C::Q;
  constexpr int NCH = 2 * DIM;   // dk_x, dk_v
  constexpr int NR = lin_len<DIM>();
  using L2S = ln::L2Scratch<DIM, K, 1>;   // the L2 stages share the H1 stages' barriers
  using PL = Plan<DIM, K, NCH, 0, 1, DIM, L2S::ALL>;
  using TB = Tab<K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* smem = reinterpret_cast<float*>(smem_raw);
  float* sB = smem + TB::B;
  float* sG = smem + TB::G;
  float* sBl = smem + TB::BL;
  float* sW = smem + TB::W;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  float* s_h = smem + PL::HEAD + eb * PL::PER;
  float* s_l = s_h + NCH * ND;
  float* t1 = s_l + NL;
  float* t2 = t1 + PL::T1;
  float* sf = t2 + PL::T2;
  float* u1 = sf + PL::SF;
  float* u2 = u1 + L2S::U1;
  float* sfl = u2 + L2S::U2;
  const ElemIdx E = elem_index<DIM, K>(P);
  for (int i = lt; i < NCH * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    s_h[i] = E.valid ? dk[comp * P.NV + node_of<DIM, K>(P, E, a)] : 0.f;
  }
  for (int i = lt; i < NL; i += NQ) s_l[i] = E.valid ? dk[2 * DIM * P.NV + E.e * NL + i] : 0.f;
  // linearisation record of this quadrature point (zeros on idle lanes: the linear
  // tangent divides by nothing)
  float Lr[NR];
  {
    const float* rq = rec + (E.valid ? E.e : 0) * NR * NQ + lt;
#pragma unroll
    for (int f = 0; f < NR; ++f) Lr[f] = E.valid ? rq[f * NQ] : 0.f;
  }
  __syncthreads();
  float hv[NCH], hg[NCH][DIM];
  float lq[1];
  ln::h1l2_fwd<DIM, K, NCH, 1, float, true>(s_h, s_l, t1, t2, u1, u2, sB, sG, sBl, lt, hv, hg, lq);
  float mq;
  {
    const int q0 = lt % Q, q1 = (lt / Q) % Q, q2 = lt / (Q * Q);
    float a = sW[q0] * sW[q1];
    if constexpr (DIM == 3) a *= sW[q2];
    mq = P.fmq0[E.valid ? E.e : 0] * a;
  }
  float dJ[DIM][DIM], dGv[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      dJ[i][r] = tau * hg[i][r];
      dGv[i][r] = tau * hg[DIM + i][r];
    }
  float fgrad[DIM][DIM], dEo, dW;
  qp_tangent_lin<DIM>(Lr, dJ, dGv, tau * lq[0], P.fq1, P.fq2, P.visc != 0, fgrad, dEo, dW);
  float fval[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) fval[i] = mq * hv[DIM + i];
  float g = mq * lq[0] - dEo;
  if constexpr (DIM == 2) {
    if (P.tg) {   // d(W s(x_q)) = dW s + W grad s . dx
      constexpr int O = 2 * DIM * DIM;
      g -= dW * Lr[O + LF_TGS] + Lr[O + LF_W] * (Lr[O + LF_TGX] * tau * hv[0] + Lr[O + LF_TGY] * tau * hv[1]);
    }
  }
  float gv[1] = {g};
  ln::h1l2_bwd<DIM, K, DIM, 1, float>(fval, fgrad, gv, sf, t1, t2, sfl, u1, u2, lt, s_h, s_l);
  if (E.valid) {
    for (int i = lt; i < DIM * ND; i += NQ) ev[E.e * (DIM * ND) + i] = s_h[i];
    for (int i = lt; i < NL; i += NQ) oute[E.e * NL + i] = TO(s_l[i]);
  }
}

// Shared-memory plan of the paired record J.w (units of float): per element the gathered
// direction, the H1 and L2 scratch of the line stages; every region starts at an even
// offset so that the paired point stages can store both points with one 8-byte access.
template <int DIM, int K, int NCH>
struct PlanX2 {
  using C = Cfg<DIM, K>;
  using PL = Plan<DIM, K, NCH, 0, 1, DIM>;
  using L2S = ln::L2Scratch<DIM, K, 1>;
  static constexpr int ev(int x) { return (x + 1) & ~1; }
  static constexpr int OL = NCH * C::ND, OT1 = ev(OL + C::NL), OT2 = ev(OT1 + PL::T1), OSF = ev(OT2 + PL::T2),
                       OU1 = ev(OSF + PL::SF), OU2 = ev(OU1 + L2S::U1), OSFL = ev(OU2 + L2S::U2),
                       PER = ev(OSFL + L2S::SF);
  static constexpr int HEAD = ev(Tab<K>::SMEM);
  static constexpr size_t bytes() { return sizeof(float) * (size_t)(HEAD + Cfg2<DIM, K>::EPB * PER); }
};

// The record J.w with two quadrature points per thread (Cfg2): the same stages as k_jvp_rec,
// with the per-point work (the last forward direction, the linearised point map, the first
// backward phase) in paired FP32 operations on the two points (q0, q1, q2) and
// (q0 + 1, q1, q2), q0 = 2 (lt % (Q/2)), whose record entries are adjacent (one 8-byte load
// per field); the line stages stride over the element's NQ / 2 threads; the gather takes one
// thread per local node for all components.  The map is linear in the direction, so tau
// scales W instead of the reference gradients.
template <int DIM, int K, class TO>
__global__ void __launch_bounds__(Cfg2<DIM, K>::THREADS)
k_jvp_rec2(ElemParams P, const float* __restrict__ rec, float tau, const float* __restrict__ dk,
           float* __restrict__ ev, TO* __restrict__ oute) {
  using C = Cfg<DIM, K>;
  using C2 = Cfg2<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ, Q = C::Q, NT = C2::NT, QH = Q / 2;
  constexpr int NCH = 2 * DIM;   // dk_x, dk_v
  constexpr int NR = lin_len<DIM>(), O = 2 * DIM * DIM;
  using PX = PlanX2<DIM, K, NCH>;
  using TB = Tab<K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* smem = reinterpret_cast<float*>(smem_raw);
  const float* sB = smem + TB::B;
  const float* sG = smem + TB::G;
  const float* sBl = smem + TB::BL;
  const float* sW = smem + TB::W;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NT, lt = threadIdx.x % NT;
  float* s_h = smem + PX::HEAD + eb * PX::PER;
  float* s_l = s_h + PX::OL;
  float* t1 = s_h + PX::OT1;
  float* t2 = s_h + PX::OT2;
  float* sf = s_h + PX::OSF;
  float* u1 = s_h + PX::OU1;
  float* u2 = s_h + PX::OU2;
  float* sfl = s_h + PX::OSFL;
  const ElemIdx E = elem_index_nt<DIM, NT, C2::EPB>(P);
  for (int a = lt; a < ND; a += NT) {
    const long long nd = node_of<DIM, K>(P, E, a);
#pragma unroll
    for (int c = 0; c < NCH; ++c) s_h[c * ND + a] = E.valid ? dk[c * P.NV + nd] : 0.f;
  }
  for (int i = lt; i < NL; i += NT) s_l[i] = E.valid ? dk[2 * DIM * P.NV + E.e * NL + i] : 0.f;
  // record of this thread's two points (idle lanes read element 0's: finite, never written)
  const int p0 = 2 * (lt % QH) + Q * (lt / QH);
  float2 Lr[NR];
  {
    const float2* rq = reinterpret_cast<const float2*>(rec + (E.valid ? E.e : 0) * NR * NQ + p0);
#pragma unroll
    for (int f = 0; f < NR; ++f) Lr[f] = rq[f * (NQ / 2)];
  }
  __syncthreads();
  float2 hv[NCH], hg[NCH][DIM], lq[1];
  ln::h1l2_fwd_x2<DIM, K, NCH, 1, NT, C2::WARP>(s_h, s_l, t1, t2, u1, u2, sB, sG, sBl, lt, hv, hg, lq);
  float2 mq;
  {
    const int q0 = 2 * (lt % QH), q1 = (lt / QH) % Q, q2 = lt / (QH * Q);
    float2 a = f2mul(make_float2(sW[q0], sW[q0 + 1]), f2s(sW[q1]));
    if constexpr (DIM == 3) a = f2mul(a, f2s(sW[q2]));
    mq = f2mul(f2s(P.fmq0[E.valid ? E.e : 0]), a);
  }
  float2 dJ[DIM][DIM], dGv[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      dJ[i][r] = hg[i][r];
      dGv[i][r] = hg[DIM + i][r];
    }
  const float2 tW = f2mul(f2s(tau), Lr[O + LF_W]);
  float2 fgrad[DIM][DIM], dEo, dW;
  qp_tangent_lin_x2<DIM>(Lr, dJ, dGv, lq[0], tW, P.visc != 0, fgrad, dEo, dW);
  float2 fval[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) fval[i] = f2mul(mq, hv[DIM + i]);
  float2 g = f2fma(mq, lq[0], f2neg(dEo));
  if constexpr (DIM == 2) {
    if (P.tg) {   // d(W s(x_q)) = dW s + W grad s . dx
      const float2 dx = f2mul(f2s(tau), f2fma(Lr[O + LF_TGX], hv[0], f2mul(Lr[O + LF_TGY], hv[1])));
      g = f2add(g, f2neg(f2fma(Lr[O + LF_W], dx, f2mul(dW, Lr[O + LF_TGS]))));
    }
  }
  float2 gv[1] = {g};
  ln::h1l2_bwd_x2<DIM, K, DIM, 1, NT, C2::WARP>(fval, fgrad, gv, sf, t1, t2, sfl, u1, u2, lt, s_h, s_l);
  if (E.valid) {
    for (int i = lt; i < DIM * ND; i += NT) ev[E.e * (DIM * ND) + i] = s_h[i];
    for (int i = lt; i < NL; i += NT) oute[E.e * NL + i] = TO(s_l[i]);
  }
}

// Pipelined record J.w (elements of 64 quadrature points, one warp per element, two points
// per lane): each warp walks a strided list of elements; the record of its next element
// (one contiguous block) arrives by a bulk asynchronous copy into the warp's shared-memory
// slot while the current element's last backward stages and the next forward stages run,
// and the next element's direction is loaded into registers while the current one
// computes.  Per-warp slot (floats): record (whose space also holds the first backward
// phase's point values, dead before the next record is requested) | gathered direction
// (H1, L2) | line-stage scratch.
constexpr int kPipeWarps = 8;   // warps (elements in flight) per block
template <int DIM, int K>
struct PipeX2 {
  using C = Cfg<DIM, K>;
  using PL = Plan<DIM, K, 2 * DIM, 0, 1, DIM>;
  using L2S = ln::L2Scratch<DIM, K, 1>;
  static constexpr int ev(int x) { return (x + 1) & ~1; }
  static constexpr int a4(int x) { return (x + 3) & ~3; }
  static constexpr int REC = lin_len<DIM>() * C::NQ;   // one element's record
  static constexpr int OSFL = ev(PL::SF);               // sf at 0, sfl after it, both inside the record
  static constexpr int OG = a4(REC), OGL = OG + 2 * DIM * C::ND, OT1 = ev(OGL + C::NL), OT2 = ev(OT1 + PL::T1),
                       OU1 = ev(OT2 + PL::T2), OU2 = ev(OU1 + L2S::U1), SLOT = a4(OU2 + L2S::U2);
  static constexpr int HEAD = a4(2 * kPipeWarps + Tab<K>::SMEM);   // mbarriers, tables
  static constexpr size_t bytes() { return sizeof(float) * (size_t)(HEAD + kPipeWarps * SLOT); }
  static_assert((REC * sizeof(float)) % 16 == 0, "bulk copies move multiples of 16 bytes");
  static_assert(OSFL + L2S::SF <= REC, "the backward point values fit in the record's space");
};
constexpr unsigned kPipePolls = 1u << 22;   // mbarrier polls before a record copy is given up

template <int DIM, int K, class TO>
__global__ void __launch_bounds__(32 * kPipeWarps, 2)
k_jvp_rec_pipe(ElemParams P, const float* __restrict__ rec, float tau, const float* __restrict__ dk,
               float* __restrict__ ev, TO* __restrict__ oute, int* __restrict__ err) {
  using C = Cfg<DIM, K>;
  using PX = PipeX2<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ, Q = C::Q, QH = Q / 2;
  static_assert(NQ == 64, "one warp per element, two points per lane");
  constexpr int NCH = 2 * DIM;   // dk_x, dk_v
  constexpr int NR = lin_len<DIM>(), O = 2 * DIM * DIM, REC = PX::REC;
  using TB = Tab<K>;
  using S = ln::H1F<DIM, K, NCH, float, 32>;
  using SL = ln::L2F<DIM, K, 1, float, K, 32>;
  using SB = ln::H1B<DIM, K, DIM, float, 32>;
  using SLB = ln::L2B<DIM, K, 1, float, K, 32>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);
  float* tab = reinterpret_cast<float*>(smem_raw) + 2 * kPipeWarps;
  const float* sB = tab + TB::B;
  const float* sG = tab + TB::G;
  const float* sBl = tab + TB::BL;
  const float* sW = tab + TB::W;
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  float* slot = reinterpret_cast<float*>(smem_raw) + PX::HEAD + w * PX::SLOT;
  float* R = slot;
  float* G = slot + PX::OG;
  float* GL = slot + PX::OGL;
  float* t1 = slot + PX::OT1;
  float* t2 = slot + PX::OT2;
  float* sf = R;
  float* sfl = R + PX::OSFL;
  float* u1 = slot + PX::OU1;
  float* u2 = slot + PX::OU2;
  load_tables(P, tab, TB::SMEM);
  if (lane == 0) {
    tc::mbar_init(&mbar[w], 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  const long long TW = (long long)gridDim.x * kPipeWarps;
  long long e = (long long)blockIdx.x * kPipeWarps + w;
  if (e >= P.NE) return;
  // the element's direction: lane a < ND holds node a's NCH components, lane j < NL the
  // j-th L2 value
  float gx[NCH], gl = 0.f;
  auto fetch = [&](long long el) {
    const unsigned n0 = (unsigned)P.n0, n1 = (unsigned)P.n1, eu = (unsigned)el;
    const unsigned t = eu / n0, ex = eu - t * n0, ey = t % n1, ez = t / n1;
    if (lane < ND) {
      const int a0 = lane % (K + 1), a1 = (lane / (K + 1)) % (K + 1), a2 = lane / ((K + 1) * (K + 1));
      const unsigned i0 = ex * K + a0, i1 = ey * K + a1, i2 = ez * K + a2;
      const long long nd = (long long)(i0 + (unsigned)P.N0 * (i1 + (unsigned)P.N1 * i2));
#pragma unroll
      for (int c = 0; c < NCH; ++c) gx[c] = dk[c * P.NV + nd];
    }
    if (lane < NL) gl = dk[2 * DIM * P.NV + el * NL + lane];
  };
  auto place = [&]() {
    if (lane < ND) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) G[c * ND + lane] = gx[c];
    }
    if (lane < NL) GL[lane] = gl;
  };
  if (lane == 0) {
    tc::mbar_arrive_expect_tx(&mbar[w], REC * (uint32_t)sizeof(float));
    tc::bulk_g2s(R, rec + e * REC, REC * (uint32_t)sizeof(float), &mbar[w]);
  }
  fetch(e);
  place();
  __syncwarp();
  const int p0 = 2 * (lane % QH) + Q * (lane / QH);
  uint32_t phase = 0;
  bool ok = true;
  for (;;) {
    const long long en = e + TW;
    const bool next = en < P.NE;
    S::s1(G, t1, lane);
    SL::s1(GL, u1, lane);
    __syncwarp();
    if (next) fetch(en);   // G is free until the outputs
    S::s2(t1, t2, lane);
    SL::s2(u1, u2, lane);
    __syncwarp();
    float2 hv[NCH], hg[NCH][DIM], lq[1];
    S::template s3x2<true>(DIM == 3 ? t2 : t1, sB, sG, lane, hv, hg);
    SL::s3x2(DIM == 3 ? u2 : u1, sBl, lane, lq);
    float2 mq;
    {
      const int q0 = 2 * (lane % QH), q1 = (lane / QH) % Q, q2 = lane / (QH * Q);
      float2 a = f2mul(make_float2(sW[q0], sW[q0 + 1]), f2s(sW[q1]));
      if constexpr (DIM == 3) a = f2mul(a, f2s(sW[q2]));
      mq = f2mul(f2s(P.fmq0[e]), a);
    }
    if (ok) {
      ok = tc::mbar_wait(&mbar[w], phase, kPipePolls);
      if (ok) phase ^= 1u;
    }
    float2 Lr[NR];
#pragma unroll
    for (int f = 0; f < NR; ++f) Lr[f] = *reinterpret_cast<const float2*>(R + f * NQ + p0);
    float2 dJ[DIM][DIM], dGv[DIM][DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int r = 0; r < DIM; ++r) {
        dJ[i][r] = hg[i][r];
        dGv[i][r] = hg[DIM + i][r];
      }
    const float2 tW = f2mul(f2s(tau), Lr[O + LF_W]);
    float2 fgrad[DIM][DIM], dEo, dW;
    qp_tangent_lin_x2<DIM>(Lr, dJ, dGv, lq[0], tW, P.visc != 0, fgrad, dEo, dW);
    float2 fval[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) fval[i] = f2mul(mq, hv[DIM + i]);
    float2 g = f2fma(mq, lq[0], f2neg(dEo));
    if constexpr (DIM == 2) {
      if (P.tg) {   // d(W s(x_q)) = dW s + W grad s . dx
        const float2 dx = f2mul(f2s(tau), f2fma(Lr[O + LF_TGX], hv[0], f2mul(Lr[O + LF_TGY], hv[1])));
        g = f2add(g, f2neg(f2fma(Lr[O + LF_W], dx, f2mul(dW, Lr[O + LF_TGS]))));
      }
    }
    __syncwarp();   // every lane has read R and t2
    float2 gv[1] = {g};
    SB::p0x2(fval, fgrad, sf, lane);
    SLB::p0x2(gv, sfl, lane);
    __syncwarp();
    SB::p1(sf, t1, t2, lane);
    SLB::p1(sfl, u1, u2, lane);
    __syncwarp();   // sf and sfl read: the record's space is free
    if (next && ok && lane == 0) {   // the next record (async proxy after the generic reads)
      tc::fence_proxy_async();
      tc::mbar_arrive_expect_tx(&mbar[w], REC * (uint32_t)sizeof(float));
      tc::bulk_g2s(R, rec + en * REC, REC * (uint32_t)sizeof(float), &mbar[w]);
    }
    SB::p2(t1, t2, lane, G);
    SLB::p2(u1, u2, lane, GL);
    __syncwarp();
    if constexpr (DIM == 3) {
      SB::p3(t1, lane, G);
      SLB::p3(u1, lane, GL);
      __syncwarp();
    }
    const float bad = ok ? 1.f : __int_as_float(0x7fc00000);
    for (int i = lane; i < DIM * ND; i += 32) ev[e * (DIM * ND) + i] = G[i] * bad;
    if (lane < NL) oute[e * NL + lane] = TO(GL[lane] * bad);
    if (!next) break;
    __syncwarp();   // outputs read before G is refilled
    place();
    __syncwarp();
    e = en;
  }
  // after a copy was given up on (no later copy is issued) it may still be in flight: wait
  // once more, bounded, before the block's shared memory is released; the flag tells the host
  if (!ok) {
    tc::mbar_wait(&mbar[w], phase, kPipePolls);
    if (err && lane == 0) atomicOr(err, kWaitErrPipe);
  }
}

// =====================================================================================
// FP32 transpose action from the linearisation record: y_v (fixed rows masked) and y_e are
// gathered and contracted; the transpose of the linearised point map (qp_tangent_lin_adj)
// gives the adjoints of the reference gradients and values; contributions to the x and v
// rows go to the element scratch ([e][2 DIM][ND]), e rows directly.
template <int DIM, int K>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_jtvp_rec(ElemParams P, const float* __restrict__ rec, float tau, const float* __restrict__ y,
           float* __restrict__ ev, float* __restrict__ oute) {
  using C = Cfg<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ, Q = C::Q;
  constexpr int NR = lin_len<DIM>();
  using PL = Plan<DIM, K, 2 * DIM, 0, 1, 2 * DIM>;
  using TB = Tab<K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* smem = reinterpret_cast<float*>(smem_raw);
  float* sB = smem + TB::B;
  float* sG = smem + TB::G;
  float* sBl = smem + TB::BL;
  float* sW = smem + TB::W;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  float* s_h = smem + PL::HEAD + eb * PL::PER;   // [DIM][ND] y_v in, [2 DIM][ND] out
  float* s_l = s_h + 2 * DIM * ND;
  float* t1 = s_l + NL;
  float* t2 = t1 + PL::T1;
  float* sf = t2 + PL::T2;
  const ElemIdx E = elem_index<DIM, K>(P);
  for (int i = lt; i < DIM * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    float v = 0.f;
    if (E.valid) {
      const long long nd = node_of<DIM, K>(P, E, a);
      v = fixed_node<DIM>(P, nd, comp) ? 0.f : y[(DIM + comp) * P.NV + nd];
    }
    s_h[i] = v;
  }
  for (int i = lt; i < NL; i += NQ) s_l[i] = E.valid ? y[2 * DIM * P.NV + E.e * NL + i] : 0.f;
  float Lr[NR];
  {
    const float* rq = rec + (E.valid ? E.e : 0) * NR * NQ + lt;
#pragma unroll
    for (int f = 0; f < NR; ++f) Lr[f] = E.valid ? rq[f * NQ] : 0.f;
  }
  __syncthreads();
  float hv[DIM], hg[DIM][DIM];
  h1_fwd<DIM, K, DIM, float, true>(s_h, t1, t2, sB, sG, lt, hv, hg);
  float lq[1];
  l2_fwd<DIM, K, 1>(s_l, t1, t2, sBl, lt, lq);
  float mq;
  {
    const int q0 = lt % Q, q1 = (lt / Q) % Q, q2 = lt / (Q * Q);
    float a = sW[q0] * sW[q1];
    if constexpr (DIM == 3) a *= sW[q2];
    mq = P.fmq0[E.valid ? E.e : 0] * a;
  }
  // adjoints of the point outputs: dS against grad y_v, dE against -y_e (g = mq e - dE)
  const float Eb = -lq[0];
  float Wb = 0.f, xb[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) xb[i] = 0.f;
  if constexpr (DIM == 2) {
    if (P.tg) {   // g -= dW s + W grad s . dx
      constexpr int O = 2 * DIM * DIM;
      Wb = -lq[0] * Lr[O + LF_TGS];
      xb[0] = -lq[0] * Lr[O + LF_W] * Lr[O + LF_TGX];
      xb[1] = -lq[0] * Lr[O + LF_W] * Lr[O + LF_TGY];
    }
  }
  float Jb[DIM][DIM], Gvb[DIM][DIM], ebv;
  qp_tangent_lin_adj<DIM>(Lr, hg, Eb, Wb, P.fq1, P.fq2, P.visc != 0, Jb, Gvb, ebv);
  float fval[2 * DIM], fgrad[2 * DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    fval[i] = tau * xb[i];
    fval[DIM + i] = mq * hv[i];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      fgrad[i][r] = tau * Jb[i][r];
      fgrad[DIM + i][r] = tau * Gvb[i][r];
    }
  }
  const float g = mq * lq[0] + tau * ebv;
  h1_bwd<DIM, K, 2 * DIM>(fval, fgrad, sf, t1, t2, sB, sG, lt, s_h);
  if (E.valid)
    for (int i = lt; i < 2 * DIM * ND; i += NQ) ev[E.e * (2 * DIM * ND) + i] = s_h[i];
  float gv[1] = {g};
  l2_bwd<DIM, K, 1>(gv, sf, t1, t2, sBl, lt, s_l);
  if (E.valid)
    for (int i = lt; i < NL; i += NQ) oute[E.e * NL + i] = s_l[i];
}

// =====================================================================================
// Transpose action: adjoint of the element residual map, contributions to the x and v
// rows in the element scratch ([e][2 DIM][ND]), e rows directly.
template <int DIM, int K>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_jtvp(ElemParams P, const double* __restrict__ u, const double* __restrict__ kk, double tau,
       const double* __restrict__ y, double* __restrict__ ev, double* __restrict__ oute) {
  using C = Cfg<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ;
  constexpr int NCH = 3 * DIM;   // w_x, w_v, y_v (fixed rows masked)
  using PL = Plan<DIM, K, NCH, 0, 2, 2 * DIM>;
  using TB = Tab<K>;
  extern __shared__ double smem[];
  double* sB = smem + TB::B;
  double* sG = smem + TB::G;
  double* sBl = smem + TB::BL;
  double* sW = smem + TB::W;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  double* s_h = smem + PL::HEAD + eb * PL::PER;
  double* s_l = s_h + NCH * ND;
  double* t1 = s_l + 2 * NL;
  double* t2 = t1 + PL::T1;
  double* sf = t2 + PL::T2;
  const ElemIdx E = elem_index<DIM, K>(P);
  for (int i = lt; i < NCH * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    double v = 0.0;
    if (E.valid) {
      const long long nd = node_of<DIM, K>(P, E, a);
      if (comp < 2 * DIM) {
        const long long g = comp * P.NV + nd;
        v = u[g] + tau * kk[g];
      } else {
        const int cc = comp - 2 * DIM;
        v = fixed_node<DIM>(P, nd, cc) ? 0.0 : y[(DIM + cc) * P.NV + nd];
      }
    }
    s_h[i] = v;
  }
  for (int i = lt; i < NL; i += NQ) {
    double we = 0.0, ye = 0.0;
    if (E.valid) {
      const long long g = 2 * DIM * P.NV + E.e * NL + i;
      we = u[g] + tau * kk[g];
      ye = y[g];
    }
    s_l[i] = we;
    s_l[NL + i] = ye;
  }
  __syncthreads();
  double hv[NCH], hg[NCH][DIM];
  h1_fwd<DIM, K, NCH>(s_h, t1, t2, sB, sG, lt, hv, hg);
  double lq[2];
  l2_fwd<DIM, K, 2>(s_l, t1, t2, sBl, lt, lq);

  const QpC<double> c = qp_consts<DIM, K, double>(P, E, sW, lt);
  double J[DIM][DIM], Gv[DIM][DIM], Sb[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      J[i][r] = hg[i][r];
      Gv[i][r] = hg[DIM + i][r];
      Sb[i][r] = hg[2 * DIM + i][r];
    }
  if (!E.valid) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) J[i][i] = 1.0;
  }
  const double Eb = -lq[1];
  double detb = 0.0, xb[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) xb[i] = 0.0;
  if constexpr (DIM == 2) {
    if (P.tg) {   // -alpha det(J) s(x_q) in the e rows
      double A[DIM][DIM];
      const double det = det_adj<DIM>(J, A);
      const double wb = -lq[1];
      detb = wb * c.alpha * tg_source<double, double>(hv[0], hv[1]);
      double sx, sy;
      tg_source_grad<double>(hv[0], hv[1], sx, sy);
      xb[0] = wb * c.alpha * det * sx;
      xb[1] = wb * c.alpha * det * sy;
    }
  }
  double Jb[DIM][DIM], Gvb[DIM][DIM], eb_ = 0.0;
  qp_adjoint<DIM>(J, Gv, lq[0], c, Sb, Eb, detb, Jb, Gvb, eb_);
  double fval[2 * DIM], fgrad[2 * DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    fval[i] = tau * xb[i];
    fval[DIM + i] = c.mq * hv[2 * DIM + i];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      fgrad[i][r] = tau * Jb[i][r];
      fgrad[DIM + i][r] = tau * Gvb[i][r];
    }
  }
  const double g = c.mq * lq[1] + tau * eb_;
  h1_bwd<DIM, K, 2 * DIM>(fval, fgrad, sf, t1, t2, sB, sG, lt, s_h);
  if (E.valid)
    for (int i = lt; i < 2 * DIM * ND; i += NQ) ev[E.e * (2 * DIM * ND) + i] = s_h[i];
  double gv[1] = {g};
  l2_bwd<DIM, K, 1>(gv, sf, t1, t2, sBl, lt, s_l);
  if (E.valid)
    for (int i = lt; i < NL; i += NQ) oute[E.e * NL + i] = s_l[i];
}

// =====================================================================================
// H1 mass: element vectors of M_V f for NC = DIM components (f component-major [DIM][NV]).
template <int DIM, int K>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_mass_h1(ElemParams P, const double* __restrict__ f, double* __restrict__ ev) {
  using C = Cfg<DIM, K>;
  constexpr int D = C::D, ND = C::ND, NQ = C::NQ;
  using PL = Plan<DIM, K, DIM, 0, 0, DIM>;
  using TB = Tab<K>;
  extern __shared__ double smem[];
  double* sB = smem + TB::B;
  double* sW = smem + TB::W;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  double* s_h = smem + PL::HEAD + eb * PL::PER;
  double* t1 = s_h + DIM * ND;
  double* t2 = t1 + PL::T1;
  double* sf = t2 + PL::T2;
  const ElemIdx E = elem_index<DIM, K>(P);
  for (int i = lt; i < DIM * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    s_h[i] = E.valid ? f[comp * P.NV + node_of<DIM, K>(P, E, a)] : 0.0;
  }
  __syncthreads();
  double fq[DIM];
  l2_fwd<DIM, K, DIM, double, D>(s_h, t1, t2, sB, lt, fq);
  const QpC<double> c = qp_consts<DIM, K, double>(P, E, sW, lt);
#pragma unroll
  for (int i = 0; i < DIM; ++i) fq[i] *= c.mq;
  l2_bwd<DIM, K, DIM, double, D>(fq, sf, t1, t2, sB, lt, s_h);
  if (E.valid)
    for (int i = lt; i < DIM * ND; i += NQ) ev[E.e * (DIM * ND) + i] = s_h[i];
}

// L2 mass: out = M_E g (element-local, no assembly)
template <int DIM, int K>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_mass_l2(ElemParams P, const double* __restrict__ gin, double* __restrict__ out) {
  using C = Cfg<DIM, K>;
  constexpr int NL = C::NL, NQ = C::NQ;
  using PL = Plan<DIM, K, 1, 0, 0, 1>;
  using TB = Tab<K>;
  extern __shared__ double smem[];
  double* sBl = smem + TB::BL;
  double* sW = smem + TB::W;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  double* s_l = smem + PL::HEAD + eb * PL::PER;
  double* t1 = s_l + C::ND;
  double* t2 = t1 + PL::T1;
  double* sf = t2 + PL::T2;
  const ElemIdx E = elem_index<DIM, K>(P);
  for (int i = lt; i < NL; i += NQ) s_l[i] = E.valid ? gin[E.e * NL + i] : 0.0;
  __syncthreads();
  double gq[1];
  l2_fwd<DIM, K, 1>(s_l, t1, t2, sBl, lt, gq);
  const QpC<double> c = qp_consts<DIM, K, double>(P, E, sW, lt);
  gq[0] *= c.mq;
  l2_bwd<DIM, K, 1>(gq, sf, t1, t2, sBl, lt, s_l);
  if (E.valid)
    for (int i = lt; i < NL; i += NQ) out[E.e * NL + i] = s_l[i];
}

// =====================================================================================
// Explicit time-step estimate per block: min_q h_min / (c_s + mu / (rho h_min)),
template <int DIM, int K>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_dt_estimate(ElemParams P, const double* __restrict__ u, double* __restrict__ blockmin) {
  using C = Cfg<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ;
  constexpr int NCH = 2 * DIM;
  using PL = Plan<DIM, K, NCH, 0, 1, 1>;
  using TB = Tab<K>;
  extern __shared__ double smem[];
  double* sB = smem + TB::B;
  double* sG = smem + TB::G;
  double* sBl = smem + TB::BL;
  double* sW = smem + TB::W;
  double* red = smem + TB::SMEM;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  double* s_h = smem + PL::HEAD + eb * PL::PER;
  double* s_l = s_h + NCH * ND;
  double* t1 = s_l + NL;
  double* t2 = t1 + PL::T1;
  const ElemIdx E = elem_index<DIM, K>(P);
  for (int i = lt; i < NCH * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    s_h[i] = E.valid ? u[comp * P.NV + node_of<DIM, K>(P, E, a)] : 0.0;
  }
  for (int i = lt; i < NL; i += NQ) s_l[i] = E.valid ? u[2 * DIM * P.NV + E.e * NL + i] : 0.0;
  __syncthreads();
  double hv[NCH], hg[NCH][DIM];
  h1_fwd<DIM, K, NCH>(s_h, t1, t2, sB, sG, lt, hv, hg);
  double lq[1];
  l2_fwd<DIM, K, 1>(s_l, t1, t2, sBl, lt, lq);
  const QpC<double> c = qp_consts<DIM, K, double>(P, E, sW, lt);
  double J[DIM][DIM], Gv[DIM][DIM];
  for (int i = 0; i < DIM; ++i)
    for (int r = 0; r < DIM; ++r) {
      J[i][r] = hg[i][r];
      Gv[i][r] = hg[DIM + i][r];
    }
  if (!E.valid)
    for (int i = 0; i < DIM; ++i) J[i][i] = 1.0;
  double A[DIM][DIM];
  const double det = det_adj<DIM>(J, A);
  const double rho = c.mq / (c.alpha * det);
  const double e = lq[0];
  const double sq = sqrt(e * e + c.eps2);
  const double ep = e >= 0.0 ? 0.5 * (e + sq) : 0.5 * c.eps2 / (sq - e);
  const double cs = sqrt(c.ggm1 * ep);
  double mu = 0.0;
  if (c.visc) {
    double Lv[DIM][DIM];
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        double s = 0;
        for (int r = 0; r < DIM; ++r) s += Gv[i][r] * A[r][j] / det;
        Lv[i][j] = s;
      }
    const double h = c.h0 * root_dim<DIM>(det * c.inv_detJ0);
    double div = 0;
    for (int i = 0; i < DIM; ++i) div += Lv[i][i];
    const double dv = h * div;
    const double ds = 2.0 * c.inv_hc * h * cs;
    const double ab = sqrt(dv * dv + ds * ds);
    const double psi = 0.5 + 0.5 * tanh((-dv - c.scoef * ds) / (2.0 * ds));
    mu = rho * h * (c.q2 * ab + c.q1 * cs * psi);
  }
  const double hmin = sigma_min<DIM>(J) / K;
  const double dt = hmin / (cs + mu / (rho * hmin));
  const double m = block_min(E.valid ? dt : DBL_MAX, red);
  if (threadIdx.x == 0) blockmin[blockIdx.x] = m;
}

// =====================================================================================
// Node-centric G^T: sum of the element contributions of lattice node nd, component comp,
// from an element scratch laid out [e][ncomp][ND], in a fixed order.
// R_x = k_x - w_v; R_v = sum of element rows, or k_v on fixed rows
template <int DIM, int K>
__global__ void k_assemble_residual(ElemParams P, const double* __restrict__ u, const double* __restrict__ kk,
                                    double tau, const double* __restrict__ ev, double* __restrict__ r) {
  for_asm_nodes<DIM>(P, [&](int comp, const int (&ic)[3], long long nd) {
    const long long i = comp * P.NV + nd, iv = DIM * P.NV + i;
    r[i] = kk[i] - (u[iv] + tau * kk[iv]);
    r[iv] = fixed_node_ic<DIM>(P, ic, comp) ? kk[iv] : gather_node_ic<DIM, K>(P, ev, DIM, comp, ic);
  });
}

template <int DIM, int K, class T, class TO>
__global__ void k_assemble_jvp(ElemParams P, const T* __restrict__ dk, double tau, const T* __restrict__ ev,
                               TO* __restrict__ out) {
  for_asm_nodes<DIM>(P, [&](int comp, const int (&ic)[3], long long nd) {
    const long long i = comp * P.NV + nd, iv = DIM * P.NV + i;
    out[i] = TO(dk[i] - T(tau) * dk[iv]);
    out[iv] = TO(fixed_node_ic<DIM>(P, ic, comp) ? dk[iv] : gather_node_ic<DIM, K>(P, ev, DIM, comp, ic));
  });
}

template <int DIM, int K, class T>
__global__ void k_assemble_jtvp(ElemParams P, const T* __restrict__ y, double tau,
                                  const T* __restrict__ ev, T* __restrict__ out) {
  for_asm_nodes<DIM>(P, [&](int comp, const int (&ic)[3], long long nd) {
    const long long i = comp * P.NV + nd, iv = DIM * P.NV + i;
    out[i] = y[i] + gather_node_ic<DIM, K>(P, ev, 2 * DIM, comp, ic);
    T s = T(-tau) * y[i] + gather_node_ic<DIM, K>(P, ev, 2 * DIM, DIM + comp, ic);
    if (fixed_node_ic<DIM>(P, ic, comp)) s += y[iv];
    out[iv] = s;
  });
}

// =====================================================================================
// Diagonal of the velocity block dR_v/dk_v = M_V + tau dF.1/dw_v of the stage Jacobian
// (the block of the paper's Eq. (23) preconditioner), element part, from the linearisation
// record.  The point map is linear in the reference velocity gradient, so per point the
// responses dS to the d^2 unit directions E_{c,l} give K_c[r][l] = dS(E_{c,l})[c][r], and
// dof (c, a) of the element collects sum_q g_a(q)^T K_c(q) g_a(q), g_a(q) the reference
// gradient of basis function a at point q (one tangent per direction, not per dof).
template <int DIM, int K>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_jvv_diag(ElemParams P, const float* __restrict__ rec, float* __restrict__ ev) {
  using C = Cfg<DIM, K>;
  constexpr int D = K + 1, ND = C::ND, NQ = C::NQ, Q = C::Q;
  constexpr int NR = lin_len<DIM>();
  constexpr int KK = DIM * DIM * DIM;
  using TB = Tab<K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* smem = reinterpret_cast<float*>(smem_raw);
  const float* sB = smem + TB::B;
  const float* sG = smem + TB::G;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  float* sK = smem + TB::SMEM + eb * NQ * KK;   // [q][c][r][l]
  const ElemIdx E = elem_index<DIM, K>(P);
  float Lr[NR];
  {
    const float* rq = rec + (E.valid ? E.e : 0) * NR * NQ + lt;
#pragma unroll
    for (int f = 0; f < NR; ++f) Lr[f] = E.valid ? rq[f * NQ] : 0.f;
  }
  float dJ[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) dJ[i][j] = 0.f;
#pragma unroll 1
  for (int c = 0; c < DIM; ++c) {
#pragma unroll 1
    for (int l = 0; l < DIM; ++l) {
      float dGv[DIM][DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) dGv[i][j] = (i == c && j == l) ? 1.f : 0.f;
      float dS[DIM][DIM], dE, dW;
      qp_tangent_lin<DIM>(Lr, dJ, dGv, 0.f, P.fq1, P.fq2, P.visc != 0, dS, dE, dW);
#pragma unroll
      for (int r = 0; r < DIM; ++r) sK[lt * KK + (c * DIM + r) * DIM + l] = dS[c][r];
    }
  }
  __syncthreads();
  if (!E.valid) return;   // no barrier follows
  for (int o = lt; o < DIM * ND; o += NQ) {
    const int c = o / ND, a = o % ND;
    const int a0 = a % D, a1 = (a / D) % D, a2 = a / (D * D);
    float acc = 0.f;
    for (int q = 0; q < NQ; ++q) {
      const int q0 = q % Q, q1 = (q / Q) % Q, q2 = q / (Q * Q);
      float g[DIM];
      if constexpr (DIM == 2) {
        g[0] = sG[q0 * D + a0] * sB[q1 * D + a1];
        g[1] = sB[q0 * D + a0] * sG[q1 * D + a1];
      } else {
        const float b0 = sB[q0 * D + a0], b1 = sB[q1 * D + a1], b2 = sB[q2 * D + a2];
        g[0] = sG[q0 * D + a0] * b1 * b2;
        g[1] = b0 * sG[q1 * D + a1] * b2;
        g[2] = b0 * b1 * sG[q2 * D + a2];
      }
      const float* Kc = sK + q * KK + c * DIM * DIM;
#pragma unroll
      for (int r = 0; r < DIM; ++r) {
        float t = 0.f;
#pragma unroll
        for (int l = 0; l < DIM; ++l) t += Kc[r * DIM + l] * g[l];
        acc += g[r] * t;
      }
    }
    ev[E.e * (DIM * ND) + o] = acc;
  }
}

// node-centric sum of the element parts: out = diag(M_V) + tau * sum (free rows), 1 (fixed)
template <int DIM, int K>
__global__ void k_assemble_jvv_diag(ElemParams P, const float* __restrict__ ev, const double* __restrict__ dmv,
                                    double tau, double floor, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= DIM * P.NV) return;
  const int comp = (int)(i / P.NV);
  const long long nd = i % P.NV;
  if (fixed_node<DIM>(P, nd, comp)) {
    out[i] = 1.0;
    return;
  }
  const double d = dmv[nd] + tau * (double)gather_node<DIM, K>(P, ev, DIM, comp, nd);
  out[i] = (floor > 0.0 && !(d >= floor * dmv[nd])) ? floor * dmv[nd] : d;
}

// diagonal of M_V, element part: rho0 detJ0 prod_d sum_q w_q B(q, a_d)^2
template <int DIM, int K>
__global__ void k_diag_mv_elem(ElemParams P, double* __restrict__ ev) {
  constexpr int D = K + 1, Q = 2 * K, ND = Cfg<DIM, K>::ND;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.NE * ND) return;
  const long long e = i / ND;
  const int a = (int)(i % ND);
  const int ad[3] = {a % D, (a / D) % D, a / (D * D)};
  double prod = P.rho0[e] * P.detJ0;
  for (int d = 0; d < DIM; ++d) {
    double s = 0;
    for (int q = 0; q < Q; ++q) {
      const double b = P.tab[Tab<K>::B + q * D + ad[d]];
      s += P.tab[Tab<K>::W + q] * b * b;
    }
    prod *= s;
  }
  ev[i] = prod;
}

// inverse of the L2 mass: Lagrange basis at the K Gauss points is orthogonal under
// exact integration, so M_E is diagonal, entry rho0 detJ0 sum_q alpha_q phi_j(q)^2
template <int DIM, int K>
__global__ void k_inv_me(ElemParams P, double* __restrict__ inv) {
  constexpr int L = K, Q = 2 * K, NL = Cfg<DIM, K>::NL;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.NE * NL) return;
  const long long e = i / NL;
  const int j = (int)(i % NL);
  const int jd[3] = {j % L, (j / L) % L, j / (L * L)};
  double prod = P.rho0[e] * P.detJ0;
  for (int d = 0; d < DIM; ++d) {
    double s = 0;
    for (int q = 0; q < Q; ++q) {
      const double b = P.tab[Tab<K>::BL + q * L + jd[d]];
      s += P.tab[Tab<K>::W + q] * b * b;
    }
    prod *= s;
  }
  inv[i] = 1.0 / prod;
}

template <int DIM, int K>
__global__ void k_initial_nodes(ElemParams P, double* __restrict__ x0) {
  constexpr int D = K + 1;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.NV) return;
  const int ic[3] = {(int)(i % P.N0), (int)((i / P.N0) % P.N1), DIM == 3 ? (int)(i / ((long long)P.N0 * P.N1)) : 0};
  const int nel[3] = {P.n0, P.n1, P.n2};
  const double* zh = P.tab + Tab<K>::W + 2 * K;    // H1 nodes follow the weights
  for (int d = 0; d < DIM; ++d) {
    int el = ic[d] / K;
    if (el >= nel[d]) el = nel[d] - 1;
    const int a = ic[d] - el * K;
    x0[d * P.NV + i] = P.lo[d] + P.h[d] * (el + zh[a]);
  }
  (void)D;
}

// =====================================================================================
// launchers
// raise the dynamic shared-memory limit once per kernel (the plan size is fixed per kernel)
static long long g_launches = 0;
void count_launches(int n) { __atomic_add_fetch(&g_launches, (long long)n, __ATOMIC_RELAXED); }
long long launches() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
cudaError_t init_const_tables() {
  const cudaError_t e = fill_const_tables();
  return e != cudaSuccess ? e : init_const_tables_explicit();
}

// blocks of KERN resident on the whole device at the given launch shape (once per device)
template <auto KERN>
static cudaError_t resident_blocks(int threads, size_t bytes, int* out) {
  static std::atomic<int> cache[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int v = cache[dev & 63].load(std::memory_order_acquire);
  if (v == 0) {
    int nb = 0, nsm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, KERN, threads, bytes);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    v = nb * nsm;
    cache[dev & 63].store(v, std::memory_order_release);
  }
  *out = v;
  return cudaSuccess;
}

template <int DIM, int K>
struct Launch {
  using C = Cfg<DIM, K>;
  static unsigned grid(const ElemParams& P) { return (unsigned)((P.NE + C::EPB - 1) / C::EPB); }
  // the record J.w in the form measured fastest per order: pipelined (elements of 64
  // points: 3D Q2, 2D Q4; one warp per element), one point per thread (3D Q1), else paired
  // (two points per thread)
  static constexpr bool kPipeRec = (DIM == 3 && K == 2) || (DIM == 2 && K == 4);
  static constexpr bool kPairRec = !(DIM == 3 && K == 1);

  static cudaError_t residual(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                              double* ev, double* Re, double* bmin, double* r, cudaEvent_t* ev2, float* rec) {
    using PL = Plan<DIM, K, 2 * DIM, DIM, 2, DIM>;
    const size_t by = PL::bytes(sizeof(double));
    cudaError_t e = prep<k_residual<DIM, K>>(by);
    if (e != cudaSuccess) return e;
    mark(ev2, 0, s);
    k_residual<DIM, K><<<grid(P), C::THREADS, by, s>>>(P, u, k, tau, ev, Re, bmin, rec);
    mark(ev2, 1, s);
    count_launches(2);
    k_assemble_residual<DIM, K><<<asm_grid(P), kAsmX, 0, s>>>(P, u, k, tau, ev, r);
    return cudaGetLastError();
  }
  template <class T, class TO>
  static cudaError_t jvp(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                         const T* dk, T* ev, TO* out, cudaEvent_t* ev2) {
    using PL = Plan<DIM, K, 4 * DIM, 0, 2, DIM>;
    const size_t by = PL::bytes(sizeof(T));
    cudaError_t e = prep<k_jvp<DIM, K, T, TO>>(by);
    if (e != cudaSuccess) return e;
    mark(ev2, 0, s);
    k_jvp<DIM, K, T, TO><<<grid(P), C::THREADS, by, s>>>(P, u, k, tau, dk, ev, out + 2 * DIM * P.NV);
    mark(ev2, 1, s);
    count_launches(2);
    k_assemble_jvp<DIM, K, T, TO><<<asm_grid(P), kAsmX, 0, s>>>(P, dk, tau, ev, out);
    return cudaGetLastError();
  }
  template <class TO>
  static cudaError_t jvp_rec(const ElemParams& P, cudaStream_t s, const float* rec, double tau, const float* dk,
                             float* ev, TO* out, cudaEvent_t* ev2, int* err) {
    if constexpr (kPipeRec) {
      const size_t by = PipeX2<DIM, K>::bytes();
      cudaError_t e = prep<k_jvp_rec_pipe<DIM, K, TO>>(by);
      int resident = 0;
      if (e == cudaSuccess) e = resident_blocks<k_jvp_rec_pipe<DIM, K, TO>>(32 * kPipeWarps, by, &resident);
      if (e != cudaSuccess) return e;
      const long long need = (P.NE + kPipeWarps - 1) / kPipeWarps;
      mark(ev2, 0, s);
      k_jvp_rec_pipe<DIM, K, TO><<<(unsigned)(need < resident ? need : resident), 32 * kPipeWarps, by, s>>>(
          P, rec, (float)tau, dk, ev, out + 2 * DIM * P.NV, err);
    } else if constexpr (kPairRec) {
      using C2 = Cfg2<DIM, K>;
      const size_t by = PlanX2<DIM, K, 2 * DIM>::bytes();
      cudaError_t e = prep<k_jvp_rec2<DIM, K, TO>>(by);
      if (e != cudaSuccess) return e;
      mark(ev2, 0, s);
      k_jvp_rec2<DIM, K, TO><<<(unsigned)((P.NE + C2::EPB - 1) / C2::EPB), C2::THREADS, by, s>>>(
          P, rec, (float)tau, dk, ev, out + 2 * DIM * P.NV);
    } else {
      using PL = Plan<DIM, K, 2 * DIM, 0, 1, DIM, ln::L2Scratch<DIM, K, 1>::ALL>;
      const size_t by = PL::bytes(sizeof(float));
      cudaError_t e = prep<k_jvp_rec<DIM, K, TO>>(by);
      if (e != cudaSuccess) return e;
      mark(ev2, 0, s);
      k_jvp_rec<DIM, K, TO><<<grid(P), C::THREADS, by, s>>>(P, rec, (float)tau, dk, ev, out + 2 * DIM * P.NV);
    }
    mark(ev2, 1, s);
    count_launches(2);
    k_assemble_jvp<DIM, K, float, TO><<<asm_grid(P), kAsmX, 0, s>>>(P, dk, tau, ev, out);
    return cudaGetLastError();
  }
  template <class TO>
  static cudaError_t assemble_jvp(const ElemParams& P, cudaStream_t s, const float* dk, double tau, const float* ev,
                                  TO* out) {
    count_launches(1);
    k_assemble_jvp<DIM, K, float, TO><<<asm_grid(P), kAsmX, 0, s>>>(P, dk, tau, ev, out);
    return cudaGetLastError();
  }
  static cudaError_t jvv_diag(const ElemParams& P, cudaStream_t s, const float* rec, double tau, float* ev,
                              const double* dmv, double* out, double floor) {
    const size_t by = sizeof(float) * ((size_t)Tab<K>::SMEM + (size_t)C::THREADS * DIM * DIM * DIM);
    cudaError_t e = prep<k_jvv_diag<DIM, K>>(by);
    if (e != cudaSuccess) return e;
    count_launches(2);
    k_jvv_diag<DIM, K><<<grid(P), C::THREADS, by, s>>>(P, rec, ev);
    k_assemble_jvv_diag<DIM, K><<<nblk(DIM * P.NV, 256), 256, 0, s>>>(P, ev, dmv, tau, floor, out);
    return cudaGetLastError();
  }
  static cudaError_t jtvp_rec(const ElemParams& P, cudaStream_t s, const float* rec, double tau, const float* y,
                              float* ev, float* out, cudaEvent_t* ev2) {
    using PL = Plan<DIM, K, 2 * DIM, 0, 1, 2 * DIM>;
    const size_t by = PL::bytes(sizeof(float));
    cudaError_t e = prep<k_jtvp_rec<DIM, K>>(by);
    if (e != cudaSuccess) return e;
    mark(ev2, 0, s);
    k_jtvp_rec<DIM, K><<<grid(P), C::THREADS, by, s>>>(P, rec, (float)tau, y, ev, out + 2 * DIM * P.NV);
    mark(ev2, 1, s);
    count_launches(2);
    k_assemble_jtvp<DIM, K, float><<<asm_grid(P), kAsmX, 0, s>>>(P, y, tau, ev, out);
    return cudaGetLastError();
  }
  static cudaError_t jtvp(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                          const double* y, double* ev, double* out, cudaEvent_t* ev2) {
    using PL = Plan<DIM, K, 3 * DIM, 0, 2, 2 * DIM>;
    const size_t by = PL::bytes(sizeof(double));
    cudaError_t e = prep<k_jtvp<DIM, K>>(by);
    if (e != cudaSuccess) return e;
    mark(ev2, 0, s);
    k_jtvp<DIM, K><<<grid(P), C::THREADS, by, s>>>(P, u, k, tau, y, ev, out + 2 * DIM * P.NV);
    mark(ev2, 1, s);
    count_launches(2);
    k_assemble_jtvp<DIM, K, double><<<asm_grid(P), kAsmX, 0, s>>>(P, y, tau, ev, out);
    return cudaGetLastError();
  }
  static cudaError_t mass_h1(const ElemParams& P, cudaStream_t s, const double* f, double* ev, double* out,
                             cudaEvent_t* ev2) {
    using PL = Plan<DIM, K, DIM, 0, 0, DIM>;
    const size_t by = PL::bytes(sizeof(double));
    cudaError_t e = prep<k_mass_h1<DIM, K>>(by);
    if (e != cudaSuccess) return e;
    mark(ev2, 0, s);
    k_mass_h1<DIM, K><<<grid(P), C::THREADS, by, s>>>(P, f, ev);
    mark(ev2, 1, s);
    count_launches(2);
    k_assemble_sum<DIM, K><<<nblk(DIM * P.NV, 256), 256, 0, s>>>(P, ev, DIM, out);
    return cudaGetLastError();
  }
  static cudaError_t mass_l2(const ElemParams& P, cudaStream_t s, const double* g, double* out) {
    using PL = Plan<DIM, K, 1, 0, 0, 1>;
    const size_t by = PL::bytes(sizeof(double));
    cudaError_t e = prep<k_mass_l2<DIM, K>>(by);
    if (e != cudaSuccess) return e;
    k_mass_l2<DIM, K><<<grid(P), C::THREADS, by, s>>>(P, g, out);
    count_launches(1);
    return cudaGetLastError();
  }
  static cudaError_t dt_estimate(const ElemParams& P, cudaStream_t s, const double* u, double* bmin) {
    using PL = Plan<DIM, K, 2 * DIM, 0, 1, 1>;
    const size_t by = PL::bytes(sizeof(double));
    cudaError_t e = prep<k_dt_estimate<DIM, K>>(by);
    if (e != cudaSuccess) return e;
    k_dt_estimate<DIM, K><<<grid(P), C::THREADS, by, s>>>(P, u, bmin);
    count_launches(1);
    return cudaGetLastError();
  }
  static cudaError_t setup(const ElemParams& P, cudaStream_t s, double* ev, double* diag, double* invme) {
    k_diag_mv_elem<DIM, K><<<nblk(P.NE * C::ND, 256), 256, 0, s>>>(P, ev);
    k_assemble_sum<DIM, K><<<nblk(P.NV, 256), 256, 0, s>>>(P, ev, 1, diag);
    k_inv_me<DIM, K><<<nblk(P.NE * C::NL, 256), 256, 0, s>>>(P, invme);
    count_launches(3);
    return cudaGetLastError();
  }
  static cudaError_t initial_nodes(const ElemParams& P, cudaStream_t s, double* x0) {
    k_initial_nodes<DIM, K><<<nblk(P.NV, 256), 256, 0, s>>>(P, x0);
    count_launches(1);
    return cudaGetLastError();
  }
};

#define LH_DISPATCH(P, ...)                                             \
  switch ((P).dim * 10 + (P).K) {                                        \
    case 21: return Launch<2, 1>::__VA_ARGS__;                                  \
    case 22: return Launch<2, 2>::__VA_ARGS__;                                  \
    case 23: return Launch<2, 3>::__VA_ARGS__;                                  \
    case 24: return Launch<2, 4>::__VA_ARGS__;                                  \
    case 31: return Launch<3, 1>::__VA_ARGS__;                                  \
    case 32: return Launch<3, 2>::__VA_ARGS__;                                  \
    case 33: return Launch<3, 3>::__VA_ARGS__;                                  \
    case 34: return Launch<3, 4>::__VA_ARGS__;                                  \
    default: return cudaErrorInvalidValue;                               \
  }

cudaError_t launch_residual(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                            double* ev, double* bmin, double* r, cudaEvent_t* ev2, float* rec) {
  double* Re = r + 2 * P.dim * P.NV;
  LH_DISPATCH(P, residual(P, s, u, k, tau, ev, Re, bmin, r, ev2, rec))
}
cudaError_t launch_jvp_rec_f32(const ElemParams& P, cudaStream_t s, const float* rec, double tau, const float* dk,
                               float* ev, float* out, cudaEvent_t* ev2, int* err) {
  LH_DISPATCH(P, template jvp_rec<float>(P, s, rec, tau, dk, ev, out, ev2, err))
}
cudaError_t launch_jvp_rec_f64out(const ElemParams& P, cudaStream_t s, const float* rec, double tau,
                                  const float* dk, float* ev, double* out, cudaEvent_t* ev2, int* err) {
  LH_DISPATCH(P, template jvp_rec<double>(P, s, rec, tau, dk, ev, out, ev2, err))
}
template <class TO>
cudaError_t launch_assemble_jvp(const ElemParams& P, cudaStream_t s, const float* dk, double tau, const float* ev,
                                TO* out) {
  LH_DISPATCH(P, template assemble_jvp<TO>(P, s, dk, tau, ev, out))
}
template cudaError_t launch_assemble_jvp<float>(const ElemParams&, cudaStream_t, const float*, double, const float*,
                                                float*);
template cudaError_t launch_assemble_jvp<double>(const ElemParams&, cudaStream_t, const float*, double,
                                                 const float*, double*);
cudaError_t launch_jvp_f64(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                           const double* dk, double* ev, double* out, cudaEvent_t* ev2) {
  LH_DISPATCH(P, template jvp<double, double>(P, s, u, k, tau, dk, ev, out, ev2))
}
cudaError_t launch_jvp_f32(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                           const float* dk, float* ev, float* out, cudaEvent_t* ev2) {
  LH_DISPATCH(P, template jvp<float, float>(P, s, u, k, tau, dk, ev, out, ev2))
}
cudaError_t launch_jvp_f32_to_f64(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                                  const float* dk, float* ev, double* out, cudaEvent_t* ev2) {
  LH_DISPATCH(P, template jvp<float, double>(P, s, u, k, tau, dk, ev, out, ev2))
}
cudaError_t launch_jtvp_rec_f32(const ElemParams& P, cudaStream_t s, const float* rec, double tau, const float* y,
                               float* ev, float* out, cudaEvent_t* ev2) {
  LH_DISPATCH(P, jtvp_rec(P, s, rec, tau, y, ev, out, ev2))
}
cudaError_t launch_jtvp(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                        const double* y, double* ev, double* out, cudaEvent_t* ev2) {
  LH_DISPATCH(P, jtvp(P, s, u, k, tau, y, ev, out, ev2))
}
cudaError_t launch_mass_h1(const ElemParams& P, cudaStream_t s, const double* f, double* ev, double* out,
                           cudaEvent_t* ev2) {
  LH_DISPATCH(P, mass_h1(P, s, f, ev, out, ev2))
}
cudaError_t launch_mass_l2(const ElemParams& P, cudaStream_t s, const double* g, double* out) {
  LH_DISPATCH(P, mass_l2(P, s, g, out))
}
template <int DIM>
__global__ void k_row_weights(ElemParams P, const double* __restrict__ diagMv, const double* __restrict__ invMe,
                              double* __restrict__ w, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long nx = (long long)DIM * P.NV;
  double v = 1.0;
  if (i >= 2 * nx) {
    v = invMe[i - 2 * nx];
  } else if (i >= nx) {
    const long long j = i - nx;
    const int comp = (int)(j / P.NV);
    const long long nd = j % P.NV;
    if (!fixed_node<DIM>(P, nd, comp)) v = 1.0 / diagMv[nd];
  }
  w[i] = v;
}

cudaError_t launch_row_weights(const ElemParams& P, cudaStream_t s, const double* diagMv, const double* invMe,
                               double* w) {
  const long long n = 2LL * P.dim * P.NV + P.NEd;
  const unsigned g = (unsigned)((n + 255) / 256);
  count_launches(1);
  if (P.dim == 2) k_row_weights<2><<<g, 256, 0, s>>>(P, diagMv, invMe, w, n);
  else k_row_weights<3><<<g, 256, 0, s>>>(P, diagMv, invMe, w, n);
  return cudaGetLastError();
}

cudaError_t launch_jvv_diag(const ElemParams& P, cudaStream_t s, const float* rec, double tau, float* ev,
                            const double* dmv, double* out, double floor) {
  LH_DISPATCH(P, jvv_diag(P, s, rec, tau, ev, dmv, out, floor))
}
cudaError_t launch_dt_estimate(const ElemParams& P, cudaStream_t s, const double* u, double* bmin) {
  LH_DISPATCH(P, dt_estimate(P, s, u, bmin))
}
cudaError_t launch_setup(const ElemParams& P, cudaStream_t s, double* ev, double* diag, double* invme) {
  LH_DISPATCH(P, setup(P, s, ev, diag, invme))
}
cudaError_t launch_initial_nodes(const ElemParams& P, cudaStream_t s, double* x0) {
  LH_DISPATCH(P, initial_nodes(P, s, x0))
}
unsigned elem_grid(const ElemParams& P) {
  switch (P.dim * 10 + P.K) {
    case 21: return Launch<2, 1>::grid(P);
    case 22: return Launch<2, 2>::grid(P);
    case 23: return Launch<2, 3>::grid(P);
    case 24: return Launch<2, 4>::grid(P);
    case 31: return Launch<3, 1>::grid(P);
    case 32: return Launch<3, 2>::grid(P);
    case 33: return Launch<3, 3>::grid(P);
    case 34: return Launch<3, 4>::grid(P);
    default: return 0;
  }
}

}  // namespace lh
