// Device helpers shared by the element kernels (lh_kernels.cu, lh_explicit.cu): the
// per-element shared-memory plan, element and lattice indexing, quadrature-point constants,
// boundary masks, block reductions, the node-centric gather of element rows (G^T of the
// paper's Sec. 2.2, Eq. (8)) and small launch helpers.
#pragma once
#include <atomic>
#include <cfloat>
#include "lh_internal.h"
#include "lh_kernels.h"
#include "lh_qp.cuh"
#include "lh_contract.cuh"

namespace lh {

// Per-element shared-memory plan (units of T): the inputs (NCH H1 fields, NCV H1 fields
// read as values only, NCL L2 fields) and the contraction scratch.  The kernel's forward
// contractions take at most max(NCH, NCV, NCL) fields and its backward ones at most
// max(NCO, 1); the scratch holds the largest need over those counts.
template <int DIM, int K, int NCH, int NCV, int NCL, int NCO, int XL = 0>
struct Plan {
  using C = Cfg<DIM, K>;
  static constexpr int NCF = lay::imax(lay::imax(NCH, NCV), lay::imax(NCL, 1)), NCB = lay::imax(NCO, 1);
  using NF = NeedFMax<DIM, K, NCF>;
  using NB = NeedBMax<DIM, K, NCB>;
  static constexpr int IN = NCH * C::ND + NCV * C::ND + NCL * C::NL;
  static constexpr int T1 = lay::imax(NF::T1, NB::T1);
  static constexpr int T2 = lay::imax(NF::T2, NB::T2);
  static constexpr int SF = NB::SF;
  static constexpr int PER = IN + T1 + T2 + SF + XL;   // XL: extra scratch of a fused kernel
  static constexpr int HEAD = ((Tab<K>::SMEM + C::THREADS + 1) / 2) * 2;   // tables + reduction
  static constexpr size_t bytes(size_t szT) { return szT * (size_t)(HEAD + C::EPB * PER); }
};

struct ElemIdx {
  long long e;
  int ex, ey, ez;
  bool valid;
};

// element of this thread: NTE threads per element, EPB elements per block
template <int DIM, int NTE, int EPB>
__device__ __forceinline__ ElemIdx elem_index_nt(const ElemParams& P) {
  ElemIdx r;
  const int eb = threadIdx.x / NTE;
  r.e = (long long)blockIdx.x * EPB + eb;
  r.valid = r.e < P.NE;
  // 32-bit lattice arithmetic: dim * N_V < 2^31 is checked at mesh creation, so NE fits
  const unsigned e = r.valid ? (unsigned)r.e : 0u, n0 = (unsigned)P.n0, n1 = (unsigned)P.n1;
  const unsigned t = e / n0;
  r.ex = (int)(e - t * n0);
  if constexpr (DIM == 3) {
    const unsigned u = t / n1;
    r.ey = (int)(t - u * n1);
    r.ez = (int)u;
  } else {
    r.ey = (int)(t % n1);
    r.ez = 0;
  }
  return r;
}
template <int DIM, int K>
__device__ __forceinline__ ElemIdx elem_index(const ElemParams& P) {
  return elem_index_nt<DIM, Cfg<DIM, K>::NQ, Cfg<DIM, K>::EPB>(P);
}

// Two quadrature points per thread (the paired element kernels): NT = NQ / 2 threads per
// element, EPB elements per block of at least 128 threads; WARP: the element's threads lie
// within one warp, so a warp barrier orders its shared-memory phases.
template <int DIM, int K>
struct Cfg2 {
  using C = Cfg<DIM, K>;
  static constexpr int NT = C::NQ / 2;
  static constexpr int EPB = NT >= 128 ? 1 : 128 / NT;
  static constexpr int THREADS = EPB * NT;
  static constexpr bool WARP = NT <= 32 && 32 % NT == 0;
};

// global lattice node of local H1 node a of element (ex, ey, ez)
template <int DIM, int K>
__device__ __forceinline__ long long node_of(const ElemParams& P, const ElemIdx& E, int a) {
  constexpr int D = K + 1;
  const int a0 = a % D, a1 = (a / D) % D, a2 = a / (D * D);
  // node indices are below N_V < 2^31 (checked at mesh creation): 32-bit products
  const unsigned i0 = (unsigned)E.ex * K + a0, i1 = (unsigned)E.ey * K + a1;
  if constexpr (DIM == 2) return (long long)(i0 + (unsigned)P.N0 * i1);
  const unsigned i2 = (unsigned)E.ez * K + a2;
  return (long long)(i0 + (unsigned)P.N0 * (i1 + (unsigned)P.N1 * i2));
}

template <int DIM, int K, class T>
__device__ __forceinline__ QpC<T> qp_consts(const ElemParams& P, const ElemIdx& E, const T* sW, int lt) {
  constexpr int Q = 2 * K;
  QpC<T> c;
  const int q0 = lt % Q, q1 = (lt / Q) % Q, q2 = lt / (Q * Q);
  T a = sW[q0] * sW[q1];
  if constexpr (DIM == 3) a *= sW[q2];
  c.alpha = a;
  const double rho0 = E.valid ? P.rho0[E.e] : 1.0;
  const double gam = E.valid ? P.gamma[E.e] : 1.4;
  c.mq = T(rho0 * P.detJ0) * a;
  c.inv_detJ0 = T(1.0 / P.detJ0);
  c.gm1 = T(gam - 1.0);
  c.ggm1 = T(gam * (gam - 1.0));
  c.h0 = T(P.h0);
  c.inv_hc = T(P.inv_hc);
  c.q1 = T(P.q1);
  c.q2 = T(P.q2);
  c.scoef = T(P.scoef);
  c.eps2 = T(P.eps2);
  c.visc = P.visc != 0;
  return c;
}

// true if velocity component comp of lattice node nd is fixed (v.n = 0 on a masked face)
template <int DIM>
__device__ __forceinline__ bool fixed_node(const ElemParams& P, long long nd_, int comp) {
  const int nd = (int)nd_;
  int ic, Nc;
  if (comp == 0) {
    ic = nd % P.N0;
    Nc = P.N0;
  } else if (comp == 1) {
    ic = (nd / P.N0) % P.N1;
    Nc = P.N1;
  } else {
    ic = nd / (P.N0 * P.N1);
    Nc = P.N2;
  }
  const bool lo = ((P.bc >> (2 * comp)) & 1u) && ic == 0;
  const bool hi = ((P.bc >> (2 * comp + 1)) & 1u) && ic == Nc - 1;
  return lo || hi;
}

template <class T>
__device__ __forceinline__ void load_tables(const ElemParams& P, T* s, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = T(P.tab[i]);
}

// min over the block (thread 0 holds the result); red has blockDim.x entries
__device__ __forceinline__ double block_min(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 1; s < (int)blockDim.x; s <<= 1) {
    const int i = threadIdx.x;
    double o = DBL_MAX;
    if ((i % (2 * s)) == 0 && i + s < (int)blockDim.x) o = red[i + s];
    __syncthreads();
    if ((i % (2 * s)) == 0) red[i] = fmin(red[i], o);
    __syncthreads();
  }
  return red[0];
}

template <int DIM, int K, class T>
__device__ __forceinline__ T gather_node_ic(const ElemParams& P, const T* __restrict__ ev, int ncomp, int comp,
                                            const int (&ic)[3]) {
  // 32-bit lattice arithmetic (node counts stay far below 2^31); per axis at most two
  // elements share the node: option 0 (the lower element, or the only one) and option 1
  // (the upper element), summed in the fixed order lower-then-upper per axis
  constexpr int D = K + 1, ND = Cfg<DIM, K>::ND;
  const int nel[3] = {P.n0, P.n1, P.n2};
  int e0[3], l0[3], e1[3], l1[3];
  bool v0[3], v1[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d >= DIM) {
      e0[d] = 0; l0[d] = 0; v0[d] = true; e1[d] = 0; l1[d] = 0; v1[d] = false;
      continue;
    }
    const int q = ic[d] / K, r = ic[d] % K;
    if (r != 0) {
      e0[d] = q; l0[d] = r; v0[d] = true;
      e1[d] = 0; l1[d] = 0; v1[d] = false;
    } else {
      e0[d] = q - 1; l0[d] = K; v0[d] = q >= 1;
      e1[d] = q; l1[d] = 0; v1[d] = q < nel[d];
    }
  }
  T s = T(0);
#pragma unroll
  for (int b2 = 0; b2 < 2; ++b2)
#pragma unroll
    for (int b1 = 0; b1 < 2; ++b1)
#pragma unroll
      for (int b0 = 0; b0 < 2; ++b0) {
        const bool ok = (b0 ? v1[0] : v0[0]) && (b1 ? v1[1] : v0[1]) && (b2 ? v1[2] : v0[2]);
        if (!ok) continue;
        const int ex = b0 ? e1[0] : e0[0], ey = b1 ? e1[1] : e0[1], ez = b2 ? e1[2] : e0[2];
        const int a = (b0 ? l1[0] : l0[0]) + D * ((b1 ? l1[1] : l0[1]) + D * (b2 ? l1[2] : l0[2]));
        const long long e = (long long)((unsigned)ex + (unsigned)P.n0 * ((unsigned)ey + (unsigned)P.n1 * (unsigned)ez));
        s += ev[(e * ncomp + comp) * ND + a];
      }
  return s;
}

template <int DIM, int K, class T>
__device__ __forceinline__ T gather_node(const ElemParams& P, const T* __restrict__ ev, int ncomp, int comp,
                                         long long nd_) {
  const int nd = (int)nd_;
  const int ic[3] = {nd % P.N0, (nd / P.N0) % P.N1, DIM == 3 ? nd / (P.N0 * P.N1) : 0};
  return gather_node_ic<DIM, K>(P, ev, ncomp, comp, ic);
}

// velocity component comp of lattice node (ic) is fixed (v.n = 0 on a masked face)
template <int DIM>
__device__ __forceinline__ bool fixed_node_ic(const ElemParams& P, const int (&ic)[3], int comp) {
  const int Nc = comp == 0 ? P.N0 : comp == 1 ? P.N1 : P.N2;
  const int c = ic[comp];
  return (((P.bc >> (2 * comp)) & 1u) && c == 0) || (((P.bc >> (2 * comp + 1)) & 1u) && c == Nc - 1);
}

// Launch shape of the node-centric assembly kernels: blocks of kAsmX nodes along x, one
// (y, z plane, component) row per block, grid-strided in y and z past the grid limits, so
// that a thread finds its node without integer division.
constexpr int kAsmX = 64;
static inline dim3 asm_grid(const ElemParams& P) {
  const long long zc = (long long)(P.dim == 3 ? P.N2 : 1) * P.dim;
  return dim3((unsigned)((P.N0 + kAsmX - 1) / kAsmX), (unsigned)(P.N1 < 65535 ? P.N1 : 65535),
              (unsigned)(zc < 65535 ? zc : 65535));
}
// f(comp, ic, nd) for every node row this thread owns under asm_grid
template <int DIM, class F>
__device__ __forceinline__ void for_asm_nodes(const ElemParams& P, F&& f) {
  const int ix = (int)blockIdx.x * kAsmX + (int)threadIdx.x;
  if (ix >= P.N0) return;
  const int nz = DIM == 3 ? P.N2 : 1;
  for (int zc = blockIdx.z; zc < nz * DIM; zc += gridDim.z) {
    const int comp = zc / nz, iz = zc - comp * nz;
    for (int iy = blockIdx.y; iy < P.N1; iy += gridDim.y) {
      const int ic[3] = {ix, iy, iz};
      const long long nd = (long long)((unsigned)ix + (unsigned)P.N0 * ((unsigned)iy + (unsigned)P.N1 * (unsigned)iz));
      f(comp, ic, nd);
    }
  }
}

// dynamic shared-memory limit of a kernel, set once per device (a per-device attribute)
template <auto KERN>
static cudaError_t prep(size_t bytes) {
  static std::atomic<unsigned long long> done{0};
  cudaError_t e = fill_const_tables();   // this translation unit's constant tables, once per device
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    done.fetch_or(bit, std::memory_order_release);
  }
  return cudaSuccess;
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

static inline void mark(cudaEvent_t* ev2, int i, cudaStream_t s) {
  if (ev2) cudaEventRecord(ev2[i], s);
}

// out[comp * NV + node] = sum of the element rows of that node (element scratch [e][ncomp][ND])
template <int DIM, int K>
__global__ void k_assemble_sum(ElemParams P, const double* __restrict__ ev, int ncomp, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ncomp * P.NV) return;
  const int comp = (int)(i / P.NV);
  out[i] = gather_node<DIM, K>(P, ev, ncomp, comp, i % P.NV);
}

// smallest singular value of a DIM x DIM matrix (the explicit time-step estimate's
// h_min = sigma_min(J) / K)
template <int DIM>
__device__ __forceinline__ double sigma_min(const double (&J)[DIM][DIM]) {
  // smallest eigenvalue of the symmetric J^T J, then its square root
  double M[DIM][DIM];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) {
      double s = 0;
      for (int r = 0; r < DIM; ++r) s += J[r][i] * J[r][j];
      M[i][j] = s;
    }
  if constexpr (DIM == 2) {
    const double tr = M[0][0] + M[1][1];
    const double dd = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    const double disc = sqrt(fmax(0.25 * tr * tr - dd, 0.0));
    return sqrt(fmax(0.5 * tr - disc, 0.0));
  } else {
    // eigenvalues of a symmetric 3x3 matrix by the trigonometric solution of its
    // characteristic cubic (Smith 1961)
    const double p1 = M[0][1] * M[0][1] + M[0][2] * M[0][2] + M[1][2] * M[1][2];
    const double q = (M[0][0] + M[1][1] + M[2][2]) / 3.0;
    const double p2 = (M[0][0] - q) * (M[0][0] - q) + (M[1][1] - q) * (M[1][1] - q) +
                      (M[2][2] - q) * (M[2][2] - q) + 2.0 * p1;
    const double p = sqrt(p2 / 6.0);
    if (p <= 1e-300) return sqrt(fmax(q, 0.0));
    double Bm[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Bm[i][j] = (M[i][j] - (i == j ? q : 0.0)) / p;
    const double detB = Bm[0][0] * (Bm[1][1] * Bm[2][2] - Bm[1][2] * Bm[2][1]) -
                        Bm[0][1] * (Bm[1][0] * Bm[2][2] - Bm[1][2] * Bm[2][0]) +
                        Bm[0][2] * (Bm[1][0] * Bm[2][1] - Bm[1][1] * Bm[2][0]);
    const double r = fmin(fmax(0.5 * detB, -1.0), 1.0);
    const double phi = acos(r) / 3.0;
    const double lmin = q + 2.0 * p * cos(phi + 2.0 * 3.14159265358979323846 / 3.0);
    return sqrt(fmax(lmin, 0.0));
  }
}

}  // namespace lh
