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
#include <utility>
#include "lh_kernels.h"

namespace lh {

static inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// The axis passes of the Kronecker inverse act on the dim velocity components
// (component-major, NV nodes each).  Along axis a the nodes of one component form an array
// [outer][Na][inner] (inner = product of the extents of the axes before a, outer of those
// after it), and the pass is, per component, the product
//     C[i][col] = sum_j A[i][j] X[j][col],   col = (o, in),  X[j][col] = x[(o Na + j) inner + in]
// with A the inverse 1D matrix of the axis (At_fixed for the component normal to it: the
// masked boundary rows of that axis are identity rows).  One kernel serves every axis: a
// block computes a tile of kTI rows i by kTC columns, staging kTK rows j of A (from its
// stored transpose) and of X in shared memory per step; each thread owns a 4 x kCQ register
// tile (narrow column tiles: more blocks in flight, since the passes are latency bound).  The first pass reads r_v scaled by D^-1/2 (and extra blocks write the L2 rows
// z_e = M_E^-1 r_e); the last pass scales by D^-1/2, passes fixed rows through and writes
// the x rows z_x = r_x + tau z_v of the block upper-triangular preconditioner.
constexpr int kTI = 64, kTC = 16, kTK = 32, kKronThreads = 128;
constexpr int kCQ = 2;                   // columns per thread (thread tile 4 x kCQ)
constexpr int kTCP = kTC + 4;            // padded row of the X tile
constexpr int kERowsPerThread = 8;

struct KronPass {
  int axis, Na;
  long long inner, outer, nv;
  int tiles_c, tiles_i;     // column tiles per component, row tiles
  long long main_blocks;    // dim * tiles_c * tiles_i
};

template <int MODE, class TR, class TZ>
__global__ void __launch_bounds__(kKronThreads)
k_kron_pass(KronPass K, ElemParams P, const float* __restrict__ At_free, const float* __restrict__ At_fixed,
            const float* __restrict__ xin, const TR* __restrict__ r, const double* __restrict__ scale,
            const double* __restrict__ ime, float* __restrict__ fout, TZ* __restrict__ z, double tau) {
  __shared__ __align__(16) float As[kTK][kTI];
  __shared__ __align__(16) float Xs[kTK][kTCP];
  static_assert(kTI / 4 * (kTC / kCQ) == kKronThreads && kCQ == 2, "thread tiling");
  __shared__ long long s_cb[kTC];   // node of (column, j = 0): o Na inner + in; -1 past the end
  __shared__ bool s_cfix[kTC];      // row fixed by a coordinate other than the pass axis
  const long long n1 = (long long)P.dim * P.NV;
  if constexpr (MODE == 0) {
    if ((long long)blockIdx.x >= K.main_blocks) {   // L2 rows: z_e = M_E^-1 r_e
      const long long b = blockIdx.x - K.main_blocks;
      for (int q = 0; q < kERowsPerThread; ++q) {
        const long long e = (b * kERowsPerThread + q) * kKronThreads + threadIdx.x;
        if (e < P.NEd) z[2 * n1 + e] = TZ((double)r[2 * n1 + e] * ime[e]);
      }
      return;
    }
  }
  long long b = blockIdx.x;
  const int ti = (int)(b % K.tiles_i);
  b /= K.tiles_i;
  const int tcol = (int)(b % K.tiles_c);
  const int c = (int)(b / K.tiles_c);
  const float* At = c == K.axis ? At_fixed : At_free;
  const int Na = K.Na;
  const long long ncol = K.outer * K.inner;           // columns of one component
  const long long col0 = (long long)tcol * kTC;
  const int i0 = ti * kTI;
  const int t = threadIdx.x;
  const int ri = (t / (kTC / kCQ)) * 4, rc = (t % (kTC / kCQ)) * kCQ;   // this thread's 4 x kCQ tile
  float acc[4][kCQ];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < kCQ; ++q) acc[a][q] = 0.f;
  const long long cbase = (long long)c * K.nv;
  if (t < kTC) {
    const long long col = col0 + t;
    long long cb = -1;
    bool fx = false;
    if (col < ncol) {
      const long long o = col / K.inner, in = col - o * K.inner;
      cb = o * Na * K.inner + in;
      if constexpr (MODE == 2) {
        if (c != K.axis) {   // coordinate of component c's own axis, taken at j = 0
          const long long nd = cb;
          long long ic;
          int Nc;
          if (c == 0) { ic = nd % P.N0; Nc = P.N0; }
          else if (c == 1) { ic = (nd / P.N0) % P.N1; Nc = P.N1; }
          else { ic = nd / ((long long)P.N0 * P.N1); Nc = P.N2; }
          fx = (((P.bc >> (2 * c)) & 1u) && ic == 0) || (((P.bc >> (2 * c + 1)) & 1u) && ic == Nc - 1);
        }
      }
    }
    s_cb[t] = cb;
    s_cfix[t] = fx;
  }
  __syncthreads();
  const bool fix_lo = ((P.bc >> (2 * c)) & 1u) && c == K.axis;
  const bool fix_hi = ((P.bc >> (2 * c + 1)) & 1u) && c == K.axis;
  // A^T tile As[j][i] = At[(j0 + j) Na + i0 + i] (coalesced over i) and X tile
  // Xs[j][cc] = x[node(col0 + cc, j0 + j)].  All loads of a stage go to registers first
  // (fixed trip counts, unrolled) and the next stage's loads are issued before the current
  // stage's FMAs, so the L2 latency overlaps the compute.
  constexpr int LA = kTK * kTI / kKronThreads, LX = kTK * kTC / kKronThreads;
  float ra[LA], rx[LX];
  auto load_stage = [&](int j0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = t + u * kKronThreads, jj = e / kTI, ii = e % kTI;
      ra[u] = (j0 + jj < Na && i0 + ii < Na) ? __ldg(At + (long long)(j0 + jj) * Na + i0 + ii) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < LX; ++u) {
      const int e = t + u * kKronThreads;
      // lines contiguous (x pass): read along j; otherwise along the columns
      const int jj = K.inner == 1 ? e % kTK : e / kTC;
      const int cc = K.inner == 1 ? e / kTK : e % kTC;
      const long long cb = s_cb[cc];
      float v = 0.f;
      if (j0 + jj < Na && cb >= 0) {
        const long long node = cb + (long long)(j0 + jj) * K.inner;
        if constexpr (MODE == 0) v = (float)((double)r[n1 + cbase + node] * scale[node]);
        else v = xin[cbase + node];
      }
      rx[u] = v;
    }
  };
  load_stage(0);
  for (int j0 = 0; j0 < Na; j0 += kTK) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = t + u * kKronThreads;
      As[e / kTI][e % kTI] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < LX; ++u) {
      const int e = t + u * kKronThreads;
      const int jj = K.inner == 1 ? e % kTK : e / kTC;
      const int cc = K.inner == 1 ? e / kTK : e % kTC;
      Xs[jj][cc] = rx[u];
    }
    __syncthreads();
    if (j0 + kTK < Na) load_stage(j0 + kTK);
#pragma unroll 8
    for (int jj = 0; jj < kTK; ++jj) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[jj][ri]);
      const float2 x2 = *reinterpret_cast<const float2*>(&Xs[jj][rc]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, xv[2] = {x2.x, x2.y};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < kCQ; ++q) acc[a][q] += av[a] * xv[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ri + a;
    if (i >= Na) continue;
#pragma unroll
    for (int q = 0; q < kCQ; ++q) {
      const long long cb = s_cb[rc + q];
      if (cb < 0) continue;
      const long long node = cb + (long long)i * K.inner;
      if constexpr (MODE == 2) {
        const bool fixed = s_cfix[rc + q] || (fix_lo && i == 0) || (fix_hi && i == Na - 1);
        const long long tv = cbase + node;
        const double zv = fixed ? (double)r[n1 + tv] : (double)acc[a][q] * scale[node];
        z[n1 + tv] = TZ(zv);
        z[tv] = TZ((double)r[tv] + tau * zv);
      } else {
        fout[cbase + node] = acc[a][q];
      }
    }
  }
}

// Fused x and y passes for 3D meshes whose lattice planes fit in shared memory (N0, N1 <=
// kNP): one block per (component, z plane) reads the plane of D^-1/2 r_v (stored transposed),
// applies A_x along x and then A_y along y in shared memory (4 x 4 register tiles, float4
// loads, zero padding to kNP) and writes the plane for the z pass; extra blocks write the L2
// rows z_e = M_E^-1 r_e.  Same operator as k_kron_pass<0> followed by k_kron_pass<1>,
// without the global round trip between them.
constexpr int kNP = 52;   // padded plane extent, a multiple of 4
constexpr int kXYThreads = 256;

template <class TR, class TZ>
__global__ void __launch_bounds__(kXYThreads)
k_kron_xy(ElemParams P, const float* __restrict__ Ax_free, const float* __restrict__ Ax_fixed,
          const float* __restrict__ Ay_free, const float* __restrict__ Ay_fixed, const TR* __restrict__ r,
          const double* __restrict__ scale, const double* __restrict__ ime, float* __restrict__ fout,
          TZ* __restrict__ z, long long main_blocks) {
  __shared__ __align__(16) float sAx[kNP][kNP];   // [j][i] = A_x[i][j] (the stored transpose)
  __shared__ __align__(16) float sAy[kNP][kNP];   // [j][i] = A_y[i][j]
  __shared__ __align__(16) float sPT[kNP][kNP];   // input plane, transposed: [x][y]
  __shared__ __align__(16) float sQ[kNP][kNP];    // after the x pass: [y][x]
  const long long nv = P.NV, n1 = 3 * nv;
  const int t = threadIdx.x;
  if ((long long)blockIdx.x >= main_blocks) {
    const long long b = blockIdx.x - main_blocks;
    for (int q = 0; q < kERowsPerThread; ++q) {
      const long long e = (b * kERowsPerThread + q) * kXYThreads + t;
      if (e < P.NEd) z[2 * n1 + e] = TZ((double)r[2 * n1 + e] * ime[e]);
    }
    return;
  }
  const int N0 = P.N0, N1 = P.N1;
  const int c = (int)(blockIdx.x / P.N2), zp = (int)(blockIdx.x % P.N2);
  const float* Ax = c == 0 ? Ax_fixed : Ax_free;
  const float* Ay = c == 1 ? Ay_fixed : Ay_free;
  const long long plane = (long long)c * nv + (long long)N0 * N1 * zp;
  // all global loads of the stage first (independent, in flight together), then the stores:
  // a loop that alternates loads and shared-memory stores serialises their latencies
  constexpr int NL = (kNP * kNP + kXYThreads - 1) / kXYThreads;
  float ax[NL], ay[NL];
  double rv[NL], sv[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int i = t + l * kXYThreads;
    const int a = i / kNP, b = i % kNP;
    const bool in = i < kNP * kNP;
    ax[l] = (in && a < N0 && b < N0) ? __ldg(Ax + a * N0 + b) : 0.f;
    ay[l] = (in && a < N1 && b < N1) ? __ldg(Ay + a * N1 + b) : 0.f;
    const int y = a, x = b;   // plane read coalesced along x, stored transposed
    rv[l] = sv[l] = 0.0;
    if (in && x < N0 && y < N1) {
      const long long node = (long long)x + (long long)N0 * y + (plane - (long long)c * nv);
      rv[l] = (double)r[n1 + (long long)c * nv + node];
      sv[l] = scale[node];
    }
  }
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int i = t + l * kXYThreads;
    if (i >= kNP * kNP) break;
    const int a = i / kNP, b = i % kNP;
    sAx[a][b] = ax[l];
    sAy[a][b] = ay[l];
    sPT[b][a] = (float)(rv[l] * sv[l]);
  }
  __syncthreads();
  constexpr int NT = kNP / 4;
  for (int tile = t; tile < NT * NT; tile += kXYThreads) {   // x pass: Q[y][i] = sum_j A_x[i][j] X[y][j]
    const int i0 = (tile % NT) * 4, y0 = (tile / NT) * 4;
    float acc[4][4] = {};
    for (int j = 0; j < N0; ++j) {
      const float4 a4 = *reinterpret_cast<const float4*>(&sAx[j][i0]);
      const float4 p4 = *reinterpret_cast<const float4*>(&sPT[j][y0]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) acc[ii][yy] += av[ii] * pv[yy];
    }
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
      *reinterpret_cast<float4*>(&sQ[y0 + yy][i0]) = make_float4(acc[0][yy], acc[1][yy], acc[2][yy], acc[3][yy]);
  }
  __syncthreads();
  for (int tile = t; tile < NT * NT; tile += kXYThreads) {   // y pass: R[i][x] = sum_j A_y[i][j] Q[j][x]
    const int x0 = (tile % NT) * 4, i0 = (tile / NT) * 4;
    float acc[4][4] = {};
    for (int j = 0; j < N1; ++j) {
      const float4 a4 = *reinterpret_cast<const float4*>(&sAy[j][i0]);
      const float4 q4 = *reinterpret_cast<const float4*>(&sQ[j][x0]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int xx = 0; xx < 4; ++xx) acc[ii][xx] += av[ii] * qv[xx];
    }
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      if (i0 + ii >= N1) break;
#pragma unroll
      for (int xx = 0; xx < 4; ++xx)
        if (x0 + xx < N0) fout[plane + (long long)N0 * (i0 + ii) + x0 + xx] = acc[ii][xx];
    }
  }
}

static KronPass kron_pass(const ElemParams& P, int axis) {
  const long long N[3] = {P.N0, P.N1, P.N2};
  KronPass K;
  K.axis = axis;
  K.Na = (int)N[axis];
  K.inner = 1;
  for (int a = 0; a < axis; ++a) K.inner *= N[a];
  K.outer = 1;
  for (int a = axis + 1; a < P.dim; ++a) K.outer *= N[a];
  K.nv = P.NV;
  K.tiles_c = (int)((K.outer * K.inner + kTC - 1) / kTC);
  K.tiles_i = (K.Na + kTI - 1) / kTI;
  K.main_blocks = (long long)P.dim * K.tiles_c * K.tiles_i;
  return K;
}

template <class TR, class TZ>
static cudaError_t kron_apply(cudaStream_t s, const ElemParams& P, const KronPrec& K, const double* inv_me,
                              const TR* r, TZ* z, double tau) {
  float* a = K.work;
  float* b = K.work + (long long)P.dim * P.NV;
  // pass over x (+ L2 rows), [pass over y], last pass over the last axis
  if (P.dim == 3 && P.N0 <= kNP && P.N1 <= kNP) {   // x and y passes fused per z plane
    const long long main_blocks = 3LL * P.N2;
    const long long eblk = (P.NEd + (long long)kXYThreads * kERowsPerThread - 1) / ((long long)kXYThreads * kERowsPerThread);
    k_kron_xy<TR, TZ><<<(unsigned)(main_blocks + eblk), kXYThreads, 0, s>>>(
        P, K.At_free[0], K.At_fixed[0], K.At_free[1], K.At_fixed[1], r, K.scale, inv_me, a, z, main_blocks);
    const KronPass kl = kron_pass(P, 2);
    k_kron_pass<2, TR, TZ><<<(unsigned)kl.main_blocks, kKronThreads, 0, s>>>(
        kl, P, K.At_free[2], K.At_fixed[2], a, r, K.scale, inv_me, nullptr, z, tau);
    count_launches(2);
    return cudaGetLastError();
  }
  const KronPass k0 = kron_pass(P, 0);
  const long long eblocks = (P.NEd + (long long)kKronThreads * kERowsPerThread - 1) / ((long long)kKronThreads * kERowsPerThread);
  k_kron_pass<0, TR, TZ><<<(unsigned)(k0.main_blocks + eblocks), kKronThreads, 0, s>>>(
      k0, P, K.At_free[0], K.At_fixed[0], nullptr, r, K.scale, inv_me, a, z, tau);
  if (P.dim == 3) {
    const KronPass k1 = kron_pass(P, 1);
    k_kron_pass<1, TR, TZ><<<(unsigned)k1.main_blocks, kKronThreads, 0, s>>>(
        k1, P, K.At_free[1], K.At_fixed[1], a, r, K.scale, inv_me, b, z, tau);
    std::swap(a, b);
  }
  const KronPass kl = kron_pass(P, P.dim - 1);
  k_kron_pass<2, TR, TZ><<<(unsigned)kl.main_blocks, kKronThreads, 0, s>>>(
      kl, P, K.At_free[P.dim - 1], K.At_fixed[P.dim - 1], a, r, K.scale, inv_me, nullptr, z, tau);
  count_launches(P.dim);
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

// the same with a per-dof velocity diagonal dv [dim NV] (the diagonal of dR_v/dk_v, 1 on
// fixed rows): z_v = dv^-1 r_v, z_x = r_x + tau z_v, z_e = M_E^-1 r_e
template <class TR, class TZ>
__global__ void k_precond_dof(ElemParams P, const double* __restrict__ dv, const double* __restrict__ ime,
                              const TR* __restrict__ r, TZ* __restrict__ z, double tau) {
  const long long n1 = (long long)P.dim * P.NV;
  const long long n = 2 * n1 + P.NEd;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i < n1) {
    z[i] = TZ((double)r[i] + tau * (double)r[n1 + i] / dv[i]);
  } else if (i < 2 * n1) {
    z[i] = TZ((double)r[i] / dv[i - n1]);
  } else {
    z[i] = TZ((double)r[i] * ime[i - 2 * n1]);
  }
}

// ---- Chebyshev iteration on the velocity Schur block (preconditioner kind 3) -------------
// S = dR_v/dk_v + tau dR_v/dk_x = M_V + tau dF.1/dv + tau^2 dF.1/dx, applied through the
// record J.w to directions [tau d | d | 0]; Jacobi-scaled by D = the clamped diagonal of
// M_V + tau dF/dv (1 on fixed rows).  Vectors are state-shaped; only velocity rows are used.
template <class TR>
__global__ void k_cheb_init(long long n1, const double* __restrict__ dv, const TR* __restrict__ r,
                            float* __restrict__ res, float* __restrict__ d, float* __restrict__ z, float inv_theta) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n1) return;
  const float rv = (float)r[n1 + j];
  const float dj = inv_theta * (float)(rv / dv[j]);
  res[n1 + j] = rv;
  d[n1 + j] = dj;
  z[n1 + j] = dj;
}

__global__ void k_cheb_dir(long long n1, long long n, const float* __restrict__ d, float* __restrict__ w, float tau) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  w[i] = i < n1 ? tau * d[n1 + i] : (i < 2 * n1 ? d[i] : 0.f);
}

__global__ void k_cheb_step(long long n1, const double* __restrict__ dv, const float* __restrict__ jw,
                            float* __restrict__ res, float* __restrict__ d, float* __restrict__ z, float c1, float c2) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n1) return;
  const float rj = res[n1 + j] - jw[n1 + j];
  res[n1 + j] = rj;
  const float dj = c1 * d[n1 + j] + c2 * (float)(rj / dv[j]);
  d[n1 + j] = dj;
  z[n1 + j] += dj;
}

template <class TR, class TZ>
__global__ void k_cheb_out(long long n1, long long n, const double* __restrict__ ime, const TR* __restrict__ r,
                           const float* __restrict__ z, TZ* __restrict__ out, double tau) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i < n1) out[i] = TZ((double)r[i] + tau * (double)z[n1 + i]);
  else if (i < 2 * n1) out[i] = TZ(z[i]);
  else out[i] = TZ((double)r[i] * ime[i - 2 * n1]);
}

// velocity rows only: y_v = D^-1 x_v (the power iteration of the Chebyshev bounds)
__global__ void k_cheb_scale(long long n1, const double* __restrict__ dv, const float* __restrict__ x,
                             float* __restrict__ y) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n1) return;
  y[n1 + j] = (float)(x[n1 + j] / dv[j]);
}

template <class TR>
cudaError_t launch_cheb_init(cudaStream_t s, long long n1, const double* dv, const TR* r, float* res, float* d,
                             float* z, double inv_theta) {
  k_cheb_init<TR><<<nb(n1, 256), 256, 0, s>>>(n1, dv, r, res, d, z, (float)inv_theta);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_cheb_dir(cudaStream_t s, long long n1, long long n, const float* d, float* w, double tau) {
  k_cheb_dir<<<nb(n, 256), 256, 0, s>>>(n1, n, d, w, (float)tau);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_cheb_step(cudaStream_t s, long long n1, const double* dv, const float* jw, float* res, float* d,
                             float* z, double c1, double c2) {
  k_cheb_step<<<nb(n1, 256), 256, 0, s>>>(n1, dv, jw, res, d, z, (float)c1, (float)c2);
  count_launches(1);
  return cudaGetLastError();
}
template <class TR, class TZ>
cudaError_t launch_cheb_out(cudaStream_t s, long long n1, long long n, const double* ime, const TR* r, const float* z,
                            TZ* out, double tau) {
  k_cheb_out<TR, TZ><<<nb(n, 256), 256, 0, s>>>(n1, n, ime, r, z, out, tau);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_cheb_scale(cudaStream_t s, long long n1, const double* dv, const float* x, float* y) {
  k_cheb_scale<<<nb(n1, 256), 256, 0, s>>>(n1, dv, x, y);
  count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_cheb_init<float>(cudaStream_t, long long, const double*, const float*, float*, float*,
                                             float*, double);
template cudaError_t launch_cheb_out<float, float>(cudaStream_t, long long, long long, const double*, const float*,
                                                   const float*, float*, double);
template cudaError_t launch_cheb_out<float, double>(cudaStream_t, long long, long long, const double*, const float*,
                                                    const float*, double*, double);

template <class TR, class TZ>
cudaError_t launch_prec(int kind, cudaStream_t s, const ElemParams& P, const KronPrec& K, const double* diag_mv,
                        const double* inv_me, const TR* r, TZ* z, double tau) {
  if (kind == 1) return kron_apply<TR, TZ>(s, P, K, inv_me, r, z, tau);
  const long long n = 2LL * P.dim * P.NV + P.NEd;
  if (kind == 2) {   // diag_mv is the per-dof velocity diagonal here
    k_precond_dof<TR, TZ><<<nb(n, 256), 256, 0, s>>>(P, diag_mv, inv_me, r, z, tau);
    count_launches(1);
    return cudaGetLastError();
  }
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
