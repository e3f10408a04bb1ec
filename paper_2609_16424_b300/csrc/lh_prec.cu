// Kronecker mass preconditioner for the velocity block of the stage Jacobian.
//
// On the undeformed box the pointwise mass weights are m_q = rho0 alpha_q detJ0 (paper
// Sec. 2.1, mass is constant in time), the H1 basis and the quadrature are tensor
// products, so the assembled H1 mass matrix of Eq. (7) is, for uniform rho0, exactly
//     M_V = rho0 (M_x (x) M_y (x) M_z),
// M_d the assembled 1D mass matrix along axis d.  Rows of fixed normal velocity drop the
// boundary layer of M_d along that component's own axis.  Its inverse is therefore three
// dense 1D contractions, one per axis, with the inverse 1D matrices (precomputed in
// double on the host, applied in float).  For piecewise-constant rho0 the operator is
// scaled by the nodal mean of rho0^(-1/2) on both sides, an approximation.
#include "lh_kernels.h"

namespace lh {

static inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// one axis of the Kronecker inverse on the dim velocity components (component-major,
// NV nodes each): out[c, node] = sum_j A_c[i_axis][j] in[c, line(node) + j stride].
// At_free / At_fixed hold the transposed inverses (entry [j][i]) of the 1D matrix without
// and with the masked boundary rows of this axis; component c == axis uses At_fixed.
// The last pass (scale_out set) applies D^-1/2, leaves fixed rows to k_prec_xe and writes
// the x rows z_x = r_x + tau z_v.
template <class TI, class TO>
__global__ void k_kron_axis(long long nv, int dim, int N0, int N1, int axis, int Na,
                            const float* __restrict__ At_free, const float* __restrict__ At_fixed,
                            const TI* __restrict__ in, TO* __restrict__ out, const double* __restrict__ scale_out,
                            ElemParams P, const double* __restrict__ r, TO* __restrict__ zx, double tau) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * dim) return;
  const int c = (int)(t / nv);
  const long long node = t % nv;
  long long stride;
  int ia;
  if (axis == 0) {
    stride = 1;
    ia = (int)(node % N0);
  } else if (axis == 1) {
    stride = N0;
    ia = (int)((node / N0) % N1);
  } else {
    stride = (long long)N0 * N1;
    ia = (int)(node / ((long long)N0 * N1));
  }
  const float* At = c == axis ? At_fixed : At_free;
  const long long base = (long long)c * nv + node - (long long)ia * stride;
  float s = 0.f;
  for (int j = 0; j < Na; ++j) s += At[(long long)j * Na + ia] * (float)in[base + j * stride];
  if (scale_out) {
    // fixed rows were written by k_prec_xe; skip them here
    long long ic;
    int Nc;
    if (c == 0) { ic = node % P.N0; Nc = P.N0; }
    else if (c == 1) { ic = (node / P.N0) % P.N1; Nc = P.N1; }
    else { ic = node / ((long long)P.N0 * P.N1); Nc = P.N2; }
    const bool fixed = (((P.bc >> (2 * c)) & 1u) && ic == 0) || (((P.bc >> (2 * c + 1)) & 1u) && ic == Nc - 1);
    const double zv = fixed ? r[nv * dim + t] : (double)s * scale_out[node];
    if (!fixed) out[t] = TO(zv);
    zx[t] = TO(r[t] + tau * zv);   // x rows of the block upper-triangular preconditioner
  } else {
    out[t] = TO(s);
  }
}

// z = P^-1 r for the whole stage vector: x rows identity, v rows the Kronecker mass
// inverse (fixed rows identity), e rows the exact L2 mass inverse.
template <class TZ>
__global__ void k_prec_xe(long long n1, long long nv, int dim, int N0, int N1, int N2, unsigned bc, long long nEd,
                          const double* __restrict__ ime, const double* __restrict__ r, TZ* __restrict__ z,
                          const double* __restrict__ scale, float* __restrict__ rs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = 2 * n1 + nEd;
  if (i >= n) return;
  if (i < n1) {
    // x rows are written by the last axis pass (z_x = r_x + tau z_v)
  } else if (i < 2 * n1) {
    const long long j = i - n1;
    const int comp = (int)(j / nv);
    const long long nd = j % nv;
    long long ic;
    int Nc;
    if (comp == 0) { ic = nd % N0; Nc = N0; }
    else if (comp == 1) { ic = (nd / N0) % N1; Nc = N1; }
    else { ic = nd / ((long long)N0 * N1); Nc = N2; }
    const bool fixed = (((bc >> (2 * comp)) & 1u) && ic == 0) || (((bc >> (2 * comp + 1)) & 1u) && ic == Nc - 1);
    if (fixed) z[i] = TZ(r[i]);
    rs[j] = (float)(r[i] * scale[nd]);            // D^-1/2 r_v, input of the first axis pass
  } else {
    z[i] = TZ(r[i] * ime[i - 2 * n1]);
  }
}

template <class TZ>
static cudaError_t kron_apply(cudaStream_t s, const ElemParams& P, const KronPrec& K, const double* inv_me,
                              const double* r, TZ* z, double tau) {
  const long long nv = P.NV, n1 = (long long)P.dim * nv;
  const int Ns[3] = {P.N0, P.N1, P.N2};
  float* a = K.work;
  float* b = K.work + n1;
  TZ* zv = z + n1;
  const unsigned g = nb(n1, 256);
  const long long n = 2 * n1 + P.NEd;
  // x and e rows, fixed v rows, and the scaled float copy of the v rows
  k_prec_xe<TZ><<<nb(n, 256), 256, 0, s>>>(n1, nv, P.dim, P.N0, P.N1, P.N2, P.bc, P.NEd, inv_me, r, z, K.scale, a);
  if (P.dim == 2) {
    k_kron_axis<float, float><<<g, 256, 0, s>>>(nv, 2, P.N0, P.N1, 0, Ns[0], K.At_free[0], K.At_fixed[0], a, b,
                                                nullptr, P, nullptr, nullptr, 0.0);
    k_kron_axis<float, TZ><<<g, 256, 0, s>>>(nv, 2, P.N0, P.N1, 1, Ns[1], K.At_free[1], K.At_fixed[1], b, zv,
                                             K.scale, P, r, z, tau);
    count_launches(3);
  } else {
    k_kron_axis<float, float><<<g, 256, 0, s>>>(nv, 3, P.N0, P.N1, 0, Ns[0], K.At_free[0], K.At_fixed[0], a, b,
                                                nullptr, P, nullptr, nullptr, 0.0);
    k_kron_axis<float, float><<<g, 256, 0, s>>>(nv, 3, P.N0, P.N1, 1, Ns[1], K.At_free[1], K.At_fixed[1], b, a,
                                                nullptr, P, nullptr, nullptr, 0.0);
    k_kron_axis<float, TZ><<<g, 256, 0, s>>>(nv, 3, P.N0, P.N1, 2, Ns[2], K.At_free[2], K.At_fixed[2], a, zv,
                                             K.scale, P, r, z, tau);
    count_launches(4);
  }
  return cudaGetLastError();
}

cudaError_t launch_kron_prec(cudaStream_t s, const ElemParams& P, const KronPrec& K, const double* inv_me,
                             const double* r, double* z, double tau) {
  return kron_apply<double>(s, P, K, inv_me, r, z, tau);
}
cudaError_t launch_kron_prec_f32(cudaStream_t s, const ElemParams& P, const KronPrec& K, const double* inv_me,
                                 const double* r, float* z, double tau) {
  return kron_apply<float>(s, P, K, inv_me, r, z, tau);
}

}  // namespace lh
