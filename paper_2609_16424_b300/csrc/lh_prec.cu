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

// The axis passes of the Kronecker inverse act on the dim velocity components
// (component-major, NV nodes each): out[c, node] = sum_j A_c[i_axis][j] in[c, line + j*stride]
// with At_free / At_fixed the transposed inverses (entry [j][i]) of the 1D matrix without /
// with the masked boundary rows of this axis (component c == axis uses At_fixed).  The input
// line (or tile of lines) is staged in shared memory; the factor is read through L1
// (coalesced in the x pass, a warp broadcast in the y/z passes).
constexpr int kKronWarps = 4;
constexpr int kKronOut = 2;   // outputs per thread along the axis in the y/z passes

// x pass: one warp per contiguous line; lanes own outputs i = lane + 32 q.
__global__ void __launch_bounds__(32 * kKronWarps)
k_kron_x(long long nv, int dim, int N0, const float* __restrict__ At_free, const float* __restrict__ At_fixed,
         const float* __restrict__ in, float* __restrict__ out) {
  extern __shared__ float kx_lines[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long per_c = nv / N0;
  const long long line = (long long)blockIdx.x * kKronWarps + warp;
  if (line >= per_c * dim) return;
  float* buf = kx_lines + warp * N0;
  for (int j = lane; j < N0; j += 32) buf[j] = in[line * N0 + j];
  __syncwarp();
  const float* At = line / per_c == 0 ? At_fixed : At_free;
  for (int i0 = 0; i0 < N0; i0 += 32 * 4) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int j = 0; j < N0; ++j) {
      const float x = buf[j];
      const float* row = At + (long long)j * N0 + i0 + lane;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i0 + lane + 32 * q < N0) acc[q] += __ldg(row + 32 * q) * x;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (i0 + lane + 32 * q < N0) out[line * N0 + i0 + lane + 32 * q] = acc[q];
  }
}

// y / z pass: a block holds a tile of 32 consecutive x-positions times the whole line along
// the axis and computes kKronWarps * kKronOut outputs along the axis (blocks split the axis).
// The last pass (LAST) applies D^-1/2, skips fixed rows (written by k_prec_xe) and writes the
// x rows z_x = r_x + tau z_v of the block upper-triangular preconditioner.
template <class TO, class TR, bool LAST>
__global__ void __launch_bounds__(32 * kKronWarps)
k_kron_yz(long long nv, int dim, int N0, int N1, int N2, int axis, const float* __restrict__ At_free,
          const float* __restrict__ At_fixed, const float* __restrict__ in, TO* __restrict__ out,
          const double* __restrict__ scale, ElemParams P, const TR* __restrict__ r, TO* __restrict__ zx, double tau) {
  extern __shared__ float kyz_tile[];   // [Na][32]
  const int Na = axis == 1 ? N1 : N2;
  const long long stride = axis == 1 ? (long long)N0 : (long long)N0 * N1;
  const int other = axis == 1 ? N2 : N1;
  const int xblocks = (N0 + 31) / 32;
  constexpr int per_block = kKronWarps * kKronOut;
  const int ablocks = (Na + per_block - 1) / per_block;
  long long b = blockIdx.x;
  const int ab = (int)(b % ablocks);
  b /= ablocks;
  const int xb = (int)(b % xblocks);
  b /= xblocks;
  const int io = (int)(b % other);
  const int c = (int)(b / other);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = xb * 32 + lane;
  const bool xin = i0 < N0;
  const long long base = (long long)c * nv + i0 + (axis == 1 ? (long long)io * N0 * N1 : (long long)io * N0);
#pragma unroll 4
  for (int j = warp; j < Na; j += kKronWarps) kyz_tile[j * 32 + lane] = xin ? in[base + j * stride] : 0.f;
  __syncthreads();
  if (!xin) return;
  const float* At = c == axis ? At_fixed : At_free;
  const int ia0 = ab * per_block + warp * kKronOut;
  float acc[kKronOut];
#pragma unroll
  for (int q = 0; q < kKronOut; ++q) acc[q] = 0.f;
  for (int j = 0; j < Na; ++j) {
    const float x = kyz_tile[j * 32 + lane];
#pragma unroll
    for (int q = 0; q < kKronOut; ++q)
      if (ia0 + q < Na) acc[q] += __ldg(At + (long long)j * Na + ia0 + q) * x;
  }
#pragma unroll
  for (int q = 0; q < kKronOut; ++q) {
    const int ia = ia0 + q;
    if (ia >= Na) break;
    const long long t = base + ia * stride;             // index into the dim x nv velocity block
    if constexpr (LAST) {
      const long long node = t - (long long)c * nv;
      long long ic;
      int Nc;
      if (c == 0) { ic = node % P.N0; Nc = P.N0; }
      else if (c == 1) { ic = (node / P.N0) % P.N1; Nc = P.N1; }
      else { ic = node / ((long long)P.N0 * P.N1); Nc = P.N2; }
      const bool fixed = (((P.bc >> (2 * c)) & 1u) && ic == 0) || (((P.bc >> (2 * c + 1)) & 1u) && ic == Nc - 1);
      const double zv = fixed ? (double)r[nv * dim + t] : (double)acc[q] * scale[node];
      if (!fixed) out[t] = TO(zv);
      zx[t] = TO((double)r[t] + tau * zv);
    } else {
      out[t] = TO(acc[q]);
    }
  }
}

// z = P^-1 r for the whole stage vector: x rows identity, v rows the Kronecker mass
// inverse (fixed rows identity), e rows the exact L2 mass inverse.
template <class TR, class TZ>
__global__ void k_prec_xe(long long n1, long long nv, int dim, int N0, int N1, int N2, unsigned bc, long long nEd,
                          const double* __restrict__ ime, const TR* __restrict__ r, TZ* __restrict__ z,
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
    rs[j] = (float)((double)r[i] * scale[nd]);    // D^-1/2 r_v, input of the first axis pass
  } else {
    z[i] = TZ((double)r[i] * ime[i - 2 * n1]);
  }
}

template <class TR, class TZ>
static cudaError_t kron_apply(cudaStream_t s, const ElemParams& P, const KronPrec& K, const double* inv_me,
                              const TR* r, TZ* z, double tau) {
  const long long nv = P.NV, n1 = (long long)P.dim * nv;
  float* a = K.work;
  float* b = K.work + n1;
  TZ* zv = z + n1;
  const long long n = 2 * n1 + P.NEd;
  const int bs = 32 * kKronWarps;
  // e rows, fixed v rows, and the scaled float copy of the v rows
  k_prec_xe<TR, TZ><<<nb(n, 256), 256, 0, s>>>(n1, nv, P.dim, P.N0, P.N1, P.N2, P.bc, P.NEd, inv_me, r, z, K.scale, a);
  const long long lines = n1 / P.N0;
  k_kron_x<<<nb(lines, kKronWarps), bs, sizeof(float) * kKronWarps * P.N0, s>>>(nv, P.dim, P.N0, K.At_free[0],
                                                                                  K.At_fixed[0], a, b);
  const int xblocks = (P.N0 + 31) / 32, per_block = kKronWarps * kKronOut;
  auto grid = [&](int Na, int other) {
    return (unsigned)((long long)P.dim * other * xblocks * ((Na + per_block - 1) / per_block));
  };
  if (P.dim == 2) {
    k_kron_yz<TZ, TR, true><<<grid(P.N1, 1), bs, sizeof(float) * 32 * P.N1, s>>>(
        nv, 2, P.N0, P.N1, 1, 1, K.At_free[1], K.At_fixed[1], b, zv, K.scale, P, r, z, tau);
    count_launches(3);
  } else {
    k_kron_yz<float, TR, false><<<grid(P.N1, P.N2), bs, sizeof(float) * 32 * P.N1, s>>>(
        nv, 3, P.N0, P.N1, P.N2, 1, K.At_free[1], K.At_fixed[1], b, a, nullptr, P, nullptr, nullptr, 0.0);
    k_kron_yz<TZ, TR, true><<<grid(P.N2, P.N1), bs, sizeof(float) * 32 * P.N2, s>>>(
        nv, 3, P.N0, P.N1, P.N2, 2, K.At_free[2], K.At_fixed[2], a, zv, K.scale, P, r, z, tau);
    count_launches(4);
  }
  return cudaGetLastError();
}

// velocity rows of the diagonal (Jacobi) mass preconditioner, identity on fixed rows
template <class TR>
__device__ __forceinline__ double jacobi_v(const ElemParams& P, const double* __restrict__ dmv,
                                           const TR* __restrict__ r, long long n1, long long j) {
  const int comp = (int)(j / P.NV);
  const long long nd = j % P.NV;
  long long ic;
  int Nc;
  if (comp == 0) { ic = nd % P.N0; Nc = P.N0; }
  else if (comp == 1) { ic = (nd / P.N0) % P.N1; Nc = P.N1; }
  else { ic = nd / ((long long)P.N0 * P.N1); Nc = P.N2; }
  const bool fixed = (((P.bc >> (2 * comp)) & 1u) && ic == 0) || (((P.bc >> (2 * comp + 1)) & 1u) && ic == Nc - 1);
  return fixed ? (double)r[n1 + j] : (double)r[n1 + j] / dmv[nd];
}

// block upper-triangular preconditioner with the diagonal of M_V: z_v = D_V^-1 r_v,
// z_x = r_x + tau z_v (exact elimination of dR_x/dk_v = -tau I), z_e = M_E^-1 r_e
template <class TR, class TZ>
__global__ void k_precond(ElemParams P, const double* __restrict__ dmv, const double* __restrict__ ime,
                          const TR* __restrict__ r, TZ* __restrict__ z, double tau) {
  const long long n1 = (long long)P.dim * P.NV;
  const long long n = 2 * n1 + P.NEd;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i < n1) {
    z[i] = TZ((double)r[i] + tau * jacobi_v(P, dmv, r, n1, i));
  } else if (i < 2 * n1) {
    z[i] = TZ(jacobi_v(P, dmv, r, n1, i - n1));
  } else {
    z[i] = TZ((double)r[i] * ime[i - 2 * n1]);
  }
}

template <class TR, class TZ>
cudaError_t launch_prec(int kind, cudaStream_t s, const ElemParams& P, const KronPrec& K, const double* diag_mv,
                        const double* inv_me, const TR* r, TZ* z, double tau) {
  if (kind == 1) return kron_apply<TR, TZ>(s, P, K, inv_me, r, z, tau);
  const long long n = 2LL * P.dim * P.NV + P.NEd;
  k_precond<TR, TZ><<<nb(n, 256), 256, 0, s>>>(P, diag_mv, inv_me, r, z, tau);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_prec<double, double>(int, cudaStream_t, const ElemParams&, const KronPrec&,
                                                 const double*, const double*, const double*, double*, double);
template cudaError_t launch_prec<double, float>(int, cudaStream_t, const ElemParams&, const KronPrec&,
                                                const double*, const double*, const double*, float*, double);
template cudaError_t launch_prec<float, float>(int, cudaStream_t, const ElemParams&, const KronPrec&,
                                               const double*, const double*, const float*, float*, double);
template cudaError_t launch_prec<float, double>(int, cudaStream_t, const ElemParams&, const KronPrec&,
                                                const double*, const double*, const float*, double*, double);

}  // namespace lh
