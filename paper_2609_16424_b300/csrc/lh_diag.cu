// Diagnostics of a state, outside the Newton path: the L1 velocity error of the 2D
// Taylor-Green vortex (Sec. 4.1, the error column of its convergence table).  The exact
// Taylor-Green velocity (sin pi x cos pi y, -cos pi x sin pi y) is steady, so the error of
// the discrete velocity at any time is
//   sum_e sum_q alpha_q detJ_q |v_h(x_q) - v*(x_q)|_2
// over the 2k-point Gauss rule of the residual, at the current (moved) points x_q.
#include "lh_internal.h"
#include "lh_kernels.h"
#include "lh_contract.cuh"

namespace lh {

namespace {

// one thread per (element, quadrature point); out[t] = that point's term of the sum
template <int K>
__global__ void k_tg_error(ElemParams P, const double* __restrict__ u, double* __restrict__ out) {
  using TB = Tab<K>;
  constexpr int D = K + 1, Q = 2 * K;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.NE * Q * Q) return;
  const int q = (int)(t % (Q * Q));
  const long long e = t / (Q * Q);
  const int qx = q % Q, qy = q / Q;
  const int ex = (int)(e % P.n0), ey = (int)(e / P.n0);
  const double* tab = P.tab;
  double x[2] = {0.0, 0.0}, v[2] = {0.0, 0.0}, J[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int b = 0; b < D; ++b) {
    const double by = tab[TB::B + qy * D + b], gy = tab[TB::G + qy * D + b];
    for (int a = 0; a < D; ++a) {
      const double bx = tab[TB::B + qx * D + a], gx = tab[TB::G + qx * D + a];
      const long long nd = (long long)(ex * K + a) + (long long)P.N0 * (ey * K + b);
      for (int c = 0; c < 2; ++c) {
        const double xc = u[c * P.NV + nd], vc = u[(2 + c) * P.NV + nd];
        x[c] += bx * by * xc;
        v[c] += bx * by * vc;
        J[c][0] += gx * by * xc;
        J[c][1] += bx * gy * xc;
      }
    }
  }
  const double detJ = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double sx = sinpi(x[0]), cx = cospi(x[0]), sy = sinpi(x[1]), cy = cospi(x[1]);
  const double d0 = v[0] - sx * cy, d1 = v[1] + cx * sy;
  out[t] = tab[TB::W + qx] * tab[TB::W + qy] * detJ * sqrt(d0 * d0 + d1 * d1);
}

template <int K>
cudaError_t launch_k(const ElemParams& P, cudaStream_t s, const double* u, double* out) {
  const long long n = P.NE * 4LL * K * K;
  count_launches(1);
  k_tg_error<K><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, u, out);
  return cudaGetLastError();
}

}  // namespace

long long tg_error_terms(const ElemParams& P) { return P.NE * 4LL * P.K * P.K; }

cudaError_t launch_tg_error(const ElemParams& P, cudaStream_t s, const double* u, double* out) {
  switch (P.K) {
    case 1: return launch_k<1>(P, s, u, out);
    case 2: return launch_k<2>(P, s, u, out);
    case 3: return launch_k<3>(P, s, u, out);
    case 4: return launch_k<4>(P, s, u, out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lh
