// Element kernels of the explicit comparison path (paper Sec. 2.2: in explicit runs the
// quadrature data of F are formed once per stage and applied twice, F.1 for the momentum
// equation and F^T w for the energy equation of Eqs. (6a)-(6b)).
//
// k_force   : at a state u, the point data S = alpha detJ sigma J^-T of every quadrature
//             point (stored, [NE][dim^2][NQ] doubles), the element rows of F.1, the
//             Taylor-Green source rows b (2D, optional) and the per-block minimum of the
//             explicit time-step estimate, with the viscosity mu_imp (Eqs. (13)-(18)) or
//             the original mu_exp (lh_qp_exp.cuh).
// k_force_t : (F^T w)_j = sum_q (S : grad_hat w) phi_j from the stored S (+ b).
// FP64 throughout; the contractions are the sum-factorised ones of the implicit path.
#include "lh_elem.cuh"
#include "lh_qp_exp.cuh"

namespace lh {

template <int DIM, int K, int VM>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_force(ElemParams P, ExpC X, const double* __restrict__ u, double* __restrict__ Sq, double* __restrict__ ev,
        double* __restrict__ bsrc, double* __restrict__ blockmin) {
  using C = Cfg<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ;
  constexpr int NCH = 2 * DIM;
  using PL = Plan<DIM, K, NCH, 0, 1, DIM>;
  using TB = Tab<K>;
  extern __shared__ double smem[];
  const double* sB = smem + TB::B;
  const double* sG = smem + TB::G;
  const double* sBl = smem + TB::BL;
  const double* sW = smem + TB::W;
  double* red = smem + TB::SMEM;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  double* s_h = smem + PL::HEAD + eb * PL::PER;   // [2 DIM][ND]: x - x(node 0), v
  double* s_l = s_h + NCH * ND;                   // [NL]: e
  double* t1 = s_l + NL;
  double* t2 = t1 + PL::T1;
  double* sf = t2 + PL::T2;
  const ElemIdx E = elem_index<DIM, K>(P);
  double x0[DIM];
  for (int c = 0; c < DIM; ++c) x0[c] = E.valid ? u[c * P.NV + node_of<DIM, K>(P, E, 0)] : 0.0;
  for (int i = lt; i < NCH * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    double v = 0.0;
    if (E.valid) {
      v = u[comp * P.NV + node_of<DIM, K>(P, E, a)];
      if (comp < DIM) v -= x0[comp];
    }
    s_h[i] = v;
  }
  for (int i = lt; i < NL; i += NQ) s_l[i] = E.valid ? u[2 * DIM * P.NV + E.e * NL + i] : 0.0;
  __syncthreads();
  double hv[NCH], hg[NCH][DIM];
  h1_fwd<DIM, K, NCH, double, DIM == 2>(s_h, t1, t2, sB, sG, lt, hv, hg);
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
    for (int i = 0; i < DIM; ++i) J[i][i] = 1.0;   // keep the idle lanes finite
  double So[DIM][DIM], Eo, detJ, mu, rho;
  if constexpr (VM == 0) {
    QpPrimal<DIM, double> pr;
    qp_forward<DIM>(J, Gv, lq[0], c, So, Eo, detJ, &pr);
    mu = pr.mu;
    rho = pr.rho;
  } else {
    qp_forward_exp<DIM>(J, Gv, lq[0], c, X, So, Eo, detJ, mu, rho);
  }
  if (E.valid) {
    double* sq = Sq + E.e * (DIM * DIM) * NQ + lt;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) sq[(i * DIM + j) * NQ] = So[i][j];
  }
  // F.1: the H1 rows sum_q S : grad_hat w_a (value part zero)
  double fval[DIM];
  for (int i = 0; i < DIM; ++i) fval[i] = 0.0;
  h1_bwd<DIM, K, DIM>(fval, So, sf, t1, t2, sB, sG, lt, s_h);
  if (E.valid)
    for (int i = lt; i < DIM * ND; i += NQ) ev[E.e * (DIM * ND) + i] = s_h[i];
  if constexpr (DIM == 2) {
    if (P.tg && bsrc) {   // b_j = sum_q alpha detJ s(x_q) phi_j on the current mesh
      double g[1] = {c.alpha * detJ * tg_source<double, double>(hv[0] + x0[0], hv[1] + x0[1])};
      l2_bwd<DIM, K, 1>(g, sf, t1, t2, sBl, lt, s_l);
      if (E.valid)
        for (int i = lt; i < NL; i += NQ) bsrc[E.e * NL + i] = s_l[i];
    }
  }
  // explicit time-step estimate min_q h_min / (c_s + mu / (rho h_min))
  const double e = lq[0];
  const double sqe = sqrt(e * e + c.eps2);
  const double ep = e >= 0.0 ? 0.5 * (e + sqe) : 0.5 * c.eps2 / (sqe - e);
  const double cs = sqrt(c.ggm1 * ep);
  const double hmin = sigma_min<DIM>(J) / K;
  const double dt = hmin / (cs + mu / (rho * hmin));
  const double m = block_min(E.valid ? dt : DBL_MAX, red);
  if (threadIdx.x == 0 && blockmin) blockmin[blockIdx.x] = m;
}

template <int DIM, int K>
__global__ void __launch_bounds__(Cfg<DIM, K>::THREADS)
k_force_t(ElemParams P, const double* __restrict__ Sq, const double* __restrict__ w,
          const double* __restrict__ bsrc, double* __restrict__ out) {
  using C = Cfg<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ;
  using PL = Plan<DIM, K, DIM, 0, 1, 1>;
  using TB = Tab<K>;
  extern __shared__ double smem[];
  const double* sB = smem + TB::B;
  const double* sG = smem + TB::G;
  const double* sBl = smem + TB::BL;
  load_tables(P, smem, TB::SMEM);
  const int eb = threadIdx.x / NQ, lt = threadIdx.x % NQ;
  double* s_h = smem + PL::HEAD + eb * PL::PER;   // [DIM][ND]: w
  double* s_l = s_h + DIM * ND;                   // [NL]: output rows
  double* t1 = s_l + NL;
  double* t2 = t1 + PL::T1;
  double* sf = t2 + PL::T2;
  const ElemIdx E = elem_index<DIM, K>(P);
  for (int i = lt; i < DIM * ND; i += NQ) {
    const int comp = i / ND, a = i % ND;
    s_h[i] = E.valid ? w[comp * P.NV + node_of<DIM, K>(P, E, a)] : 0.0;
  }
  __syncthreads();
  double hv[DIM], hg[DIM][DIM];
  h1_fwd<DIM, K, DIM, double, false>(s_h, t1, t2, sB, sG, lt, hv, hg);
  double g[1] = {0.0};
  if (E.valid) {
    const double* sq = Sq + E.e * (DIM * DIM) * NQ + lt;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) g[0] += sq[(i * DIM + j) * NQ] * hg[i][j];
  }
  l2_bwd<DIM, K, 1>(g, sf, t1, t2, sBl, lt, s_l);
  if (E.valid)
    for (int i = lt; i < NL; i += NQ) out[E.e * NL + i] = s_l[i] + (bsrc ? bsrc[E.e * NL + i] : 0.0);
}

// dst = src on the fixed rows of a velocity array [dim NV] (walls of bc_mask)
template <int DIM>
__global__ void k_copy_fixed(ElemParams P, const double* __restrict__ src, double* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= DIM * P.NV) return;
  if (fixed_node<DIM>(P, i % P.NV, (int)(i / P.NV))) dst[i] = src ? src[i] : 0.0;
}

namespace {

template <int DIM, int K>
struct ExplicitLaunch {
  using C = Cfg<DIM, K>;
  static unsigned grid(const ElemParams& P) { return (unsigned)((P.NE + C::EPB - 1) / C::EPB); }
  static cudaError_t force(const ElemParams& P, cudaStream_t s, int vm, const ExpC& X, const double* u, double* Sq,
                           double* ev, double* f1, double* bsrc, double* blockmin) {
    using PL = Plan<DIM, K, 2 * DIM, 0, 1, DIM>;
    const size_t by = PL::bytes(sizeof(double));
    cudaError_t e;
    if (vm == 0) {
      if ((e = prep<k_force<DIM, K, 0>>(by)) != cudaSuccess) return e;
      k_force<DIM, K, 0><<<grid(P), C::THREADS, by, s>>>(P, X, u, Sq, ev, bsrc, blockmin);
    } else {
      if ((e = prep<k_force<DIM, K, 1>>(by)) != cudaSuccess) return e;
      k_force<DIM, K, 1><<<grid(P), C::THREADS, by, s>>>(P, X, u, Sq, ev, bsrc, blockmin);
    }
    count_launches(2);
    k_assemble_sum<DIM, K><<<nblk(DIM * P.NV, 256), 256, 0, s>>>(P, ev, DIM, f1);
    return cudaGetLastError();
  }
  static cudaError_t force_t(const ElemParams& P, cudaStream_t s, const double* Sq, const double* w,
                             const double* bsrc, double* out) {
    using PL = Plan<DIM, K, DIM, 0, 1, 1>;
    const size_t by = PL::bytes(sizeof(double));
    cudaError_t e = prep<k_force_t<DIM, K>>(by);
    if (e != cudaSuccess) return e;
    k_force_t<DIM, K><<<grid(P), C::THREADS, by, s>>>(P, Sq, w, bsrc, out);
    count_launches(1);
    return cudaGetLastError();
  }
};

}  // namespace

#define LH_XDISPATCH(P, ...)                                     \
  switch ((P).dim * 10 + (P).K) {                                \
    case 21: return ExplicitLaunch<2, 1>::__VA_ARGS__;           \
    case 22: return ExplicitLaunch<2, 2>::__VA_ARGS__;           \
    case 23: return ExplicitLaunch<2, 3>::__VA_ARGS__;           \
    case 24: return ExplicitLaunch<2, 4>::__VA_ARGS__;           \
    case 31: return ExplicitLaunch<3, 1>::__VA_ARGS__;           \
    case 32: return ExplicitLaunch<3, 2>::__VA_ARGS__;           \
    case 33: return ExplicitLaunch<3, 3>::__VA_ARGS__;           \
    case 34: return ExplicitLaunch<3, 4>::__VA_ARGS__;           \
    default: return cudaErrorInvalidValue;                       \
  }

cudaError_t launch_force(const ElemParams& P, cudaStream_t s, int vm, const ExpC& X, const double* u, double* Sq,
                         double* ev, double* f1, double* bsrc, double* blockmin) {
  LH_XDISPATCH(P, force(P, s, vm, X, u, Sq, ev, f1, bsrc, blockmin))
}

cudaError_t launch_force_t(const ElemParams& P, cudaStream_t s, const double* Sq, const double* w, const double* bsrc,
                           double* out) {
  LH_XDISPATCH(P, force_t(P, s, Sq, w, bsrc, out))
}

cudaError_t init_const_tables_explicit() { return fill_const_tables(); }

cudaError_t launch_copy_fixed(const ElemParams& P, cudaStream_t s, const double* src, double* dst) {
  const long long n = (long long)P.dim * P.NV;
  if (P.dim == 2) k_copy_fixed<2><<<nblk(n, 256), 256, 0, s>>>(P, src, dst);
  else k_copy_fixed<3><<<nblk(n, 256), 256, 0, s>>>(P, src, dst);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace lh
