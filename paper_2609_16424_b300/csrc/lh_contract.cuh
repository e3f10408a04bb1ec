// Sum-factorised basis contractions (the B and B^T operators of paper Sec. 2.2, Eq. (8)).
//
// Tensor-product elements let B act one direction at a time (Sec. 2.2: O(p^{d+1}) work
// per element instead of O(p^{2d})).  One thread per quadrature point; intermediates live
// in shared memory.  Two forms of the same stages:
//  * line form (FP32, whose element kernels are bound by shared-memory instructions):
//    every stage that contracts a direction runs one thread per 1D line of the element
//    (all other indices fixed); the thread loads the line once into registers and forms
//    every output of the line with the 1D table entries as compile-time operands (constant
//    memory), so the only shared-memory traffic is the intermediates themselves.  The last
//    forward stage runs per quadrature point, with this thread's table row taken from
//    shared memory once.  The intermediate layouts are padded so that the lanes of a warp
//    fall into distinct banks (the padding is chosen at compile time by counting banks for
//    the first warp).  The line stages take the element's thread count as a stride (NT:
//    one thread per point, or half of that when each thread holds two points); with two
//    points per thread the per-point stages (s3x2, p0x2) work on the pair (q0, q1, q2),
//    (q0 + 1, q1, q2) in paired FP32 operations.
//  * output-parallel form (FP64 and double-float, bound by arithmetic): the threads of an
//    element stride over the outputs of each stage, which keeps every lane busy (the line
//    counts are not multiples of the warp width).
// Every entry point ends with a barrier so the caller may reuse the scratch at once; the
// stage functions themselves have none.
// In both forms each output is the same sum, in the same order, as the plain definition
// out = sum_a table(q, a) in(a) along each direction, so they give identical results.
//
// Tables (row-major): B[q*D + a] = w_a(z_q), G[q*D + a] = w_a'(z_q) for the H1 basis,
// Bl[q*L + j] = phi_j(z_q) for the L2 basis.
// Element-local layouts: H1 values [c][a2][a1][a0] (a = a0 + D a1 + D^2 a2), L2 values
// [c][j2][j1][j0], quadrature values [q2][q1][q0].
#pragma once
#include <atomic>
#include <type_traits>
#include <mutex>
#include <vector>
#include "lh_common.cuh"
#include "lh_f2.cuh"
#include "lh_internal.h"

namespace lh {

// 1D table layout in the device table buffer (built by the host at mesh creation):
// [B | G | Bl | w | H1 nodes | L2 nodes]
template <int K>
struct Tab {
  static constexpr int D = K + 1, L = K, Q = 2 * K;
  static constexpr int B = 0, G = Q * D, BL = 2 * Q * D, W = 2 * Q * D + Q * L;
  static constexpr int SMEM = 2 * Q * D + Q * L + Q;           // entries staged in shared memory
};

// ---------------------------------------------------------------------------------------
// The tables of orders 1-4 in constant memory: one copy per translation unit, written on
// each device by fill_const_tables() before the first launch there.
template <int K>
struct TabOff {
  static constexpr int v = TabOff<K - 1>::v + Tab<K - 1>::SMEM;
};
template <>
struct TabOff<1> {
  static constexpr int v = 0;
};
constexpr int kTabAll = TabOff<5>::v;

static __constant__ double c_tab_d[kTabAll];
static __constant__ float c_tab_f[kTabAll];     // float(t)
static __constant__ float c_tab_flo[kTabAll];   // float(t - float(t)): DF = (c_tab_f, c_tab_flo)

template <class T>
struct CT;
template <>
struct CT<double> {
  static __device__ __forceinline__ double at(int i) { return c_tab_d[i]; }
};
template <>
struct CT<float> {
  static __device__ __forceinline__ float at(int i) { return c_tab_f[i]; }
};
template <>
struct CT<DF> {
  static __device__ __forceinline__ DF at(int i) { return DF(c_tab_f[i], c_tab_flo[i]); }
};
template <class T, int K>
__device__ __forceinline__ T cB(int q, int a) {
  return CT<T>::at(TabOff<K>::v + Tab<K>::B + q * (K + 1) + a);
}
template <class T, int K>
__device__ __forceinline__ T cG(int q, int a) {
  return CT<T>::at(TabOff<K>::v + Tab<K>::G + q * (K + 1) + a);
}
// the "L2" table of l2_fwd / l2_bwd: the L2 basis (N = K) or the H1 values (N = K + 1)
template <class T, int K, int N>
__device__ __forceinline__ T cL(int q, int j) {
  static_assert(N == K || N == K + 1, "l2 contractions take N = K or K + 1");
  if constexpr (N == K + 1) return cB<T, K>(q, j);
  else return CT<T>::at(TabOff<K>::v + Tab<K>::BL + q * K + j);
}

static inline cudaError_t fill_const_tables() {
  static std::atomic<unsigned long long> done{0};
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  double d[kTabAll];
  float f[kTabAll], flo[kTabAll];
  const int n[4] = {Tab<1>::SMEM, Tab<2>::SMEM, Tab<3>::SMEM, Tab<4>::SMEM};
  int o = 0;
  for (int K = 1; K <= 4; ++K) {
    const std::vector<double> t = host_tables(K);
    if ((int)t.size() < n[K - 1]) return cudaErrorInvalidValue;
    for (int i = 0; i < n[K - 1]; ++i) {
      d[o + i] = t[i];
      f[o + i] = (float)t[i];
      flo[o + i] = (float)(t[i] - (double)f[o + i]);
    }
    o += n[K - 1];
  }
  e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(d));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(f));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tab_flo, flo, sizeof(flo));
  if (e != cudaSuccess) return e;
  done.fetch_or(bit, std::memory_order_release);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------------------
// Intermediate layouts (compile time).  ways() is the largest number of distinct addresses
// that one of the 32 banks receives from a warp's lanes (1 = conflict free, equal
// addresses broadcast); each pick takes the padding with the fewest ways over the stage
// accesses it affects, smallest first.
namespace lay {
constexpr int ways(const int (&a)[32]) {
  int cnt[32] = {};
  int worst = 1;
  for (int l = 0; l < 32; ++l) {
    if (a[l] < 0) continue;
    bool dup = false;
    for (int k = 0; k < l; ++k) dup = dup || a[k] == a[l];
    if (!dup) {
      const int b = a[l] & 31;
      cnt[b] += 1;
      if (cnt[b] > worst) worst = cnt[b];
    }
  }
  return worst;
}
constexpr int lanes(int nq) { return nq < 32 ? nq : 32; }
constexpr int imax(int a, int b) { return a > b ? a : b; }

// forward 3D, N 1D dofs, NC fields:
//   t1[q0][m][a1] (m = c N + a2): a1 stride 1, m stride N1, q0 stride P1
//   t2[q1][q0][m]: m stride 1, (q1 Q + q0) stride MS
struct F3L {
  int N1, P1, MS;
};
constexpr F3L pick_f3(int N, int NC, int Q) {
  const int NM = NC * N, nl = lanes(Q * Q * Q);
  F3L r{N, NM * N, NM};
  int best = 1 << 30;
  for (int n1 = N; n1 < N + 4; ++n1)
    for (int p1 = NM * n1; p1 < NM * n1 + 8; ++p1) {
      int w1[32] = {}, w2[32] = {};
      for (int l = 0; l < 32; ++l) {
        w1[l] = (l < nl && l < NM * N) ? (l / N) * n1 + l % N : -1;            // stage 1 stores
        w2[l] = (l < nl && l < Q * NM) ? (l / NM) * p1 + (l % NM) * n1 : -1;   // stage 2 loads
      }
      const int s = ways(w1) + ways(w2);
      if (s < best) {
        best = s;
        r.N1 = n1;
        r.P1 = p1;
      }
    }
  best = 1 << 30;
  for (int ms = NM; ms < NM + 16; ++ms) {
    int w1[32] = {}, w2[32] = {};
    for (int l = 0; l < 32; ++l) {
      w1[l] = (l < nl && l < Q * NM) ? (l / NM) * ms + l % NM : -1;   // stage 2 stores
      w2[l] = l < nl ? (((l / Q) % Q) * Q + l % Q) * ms : -1;          // stage 3 loads
    }
    const int s = ways(w1) + ways(w2);
    if (s < best) {
      best = s;
      r.MS = ms;
    }
  }
  return r;
}
// forward 2D: t1[q0][r] (r = c N + a1), q0 stride R
constexpr int pick_f2(int N, int NC, int Q) {
  const int NM = NC * N, nl = lanes(Q * Q);
  int r = NM, best = 1 << 30;
  for (int R = NM; R < NM + 33; ++R) {
    int w[32] = {};
    for (int l = 0; l < 32; ++l) w[l] = l < nl ? (l % Q) * R : -1;   // stage 2 loads
    const int s = ways(w);
    if (s < best) {
      best = s;
      r = R;
    }
  }
  return r;
}
// backward 3D, N 1D dofs, NC fields:
//   sf[c][point]: c stride NQp
//   t2[a2][c][q1][q0]: c stride CA, a2 stride SA
//   t1[q0][m][a1] (m = c N + a2): q0 stride RB
struct B3L {
  int NQp, CA, SA, RB;
};
constexpr B3L pick_b3(int N, int NC, int Q) {
  const int QQ = Q * Q, NQ = QQ * Q, NM = NC * N, nl = lanes(NQ);
  B3L r{NQ, QQ, NC * QQ, NM * N};
  int best = 1 << 30;
  for (int v = NQ; v < NQ + 33; ++v) {
    int w[32] = {};
    for (int l = 0; l < 32; ++l) w[l] = (l < nl && l < NC * QQ) ? (l / QQ) * v + l % QQ : -1;   // stage A loads
    const int s = ways(w);
    if (s < best) {
      best = s;
      r.NQp = v;
    }
  }
  best = 1 << 30;
  for (int ca = QQ; ca < QQ + 17; ++ca)
    for (int sa = NC * ca; sa < NC * ca + 8; ++sa) {
      int w1[32] = {}, w2[32] = {};
      for (int l = 0; l < 32; ++l) {
        w1[l] = (l < nl && l < NC * QQ) ? (l / QQ) * ca + l % QQ : -1;                           // stage A stores
        w2[l] = (l < nl && l < NM * Q) ? ((l / Q) % N) * sa + ((l / Q) / N) * ca + l % Q : -1;   // stage B loads
      }
      const int s = ways(w1) + ways(w2);
      if (s < best) {
        best = s;
        r.CA = ca;
        r.SA = sa;
      }
    }
  best = 1 << 30;
  for (int rb = NM * N; rb < NM * N + 33; ++rb) {
    int w[32] = {};
    for (int l = 0; l < 32; ++l) w[l] = (l < nl && l < NM * Q) ? (l % Q) * rb + (l / Q) * N : -1;   // stage B stores
    const int s = ways(w);
    if (s < best) {
      best = s;
      r.RB = rb;
    }
  }
  return r;
}
// backward 2D: sf[c][point] (c stride NQp), t1[q0][r] (r = c N + a1, q0 stride R)
struct B2L {
  int NQp, R;
};
constexpr B2L pick_b2(int N, int NC, int Q) {
  const int NQ = Q * Q, NM = NC * N, nl = lanes(NQ);
  B2L r{NQ, NM};
  int best = 1 << 30;
  for (int v = NQ; v < NQ + 33; ++v) {
    int w[32] = {};
    for (int l = 0; l < 32; ++l) w[l] = (l < nl && l < NC * Q) ? (l / Q) * v + l % Q : -1;   // stage A loads
    const int s = ways(w);
    if (s < best) {
      best = s;
      r.NQp = v;
    }
  }
  best = 1 << 30;
  for (int R = NM; R < NM + 33; ++R) {
    int w[32] = {};
    for (int l = 0; l < 32; ++l) w[l] = (l < nl && l < NC * Q) ? (l % Q) * R + (l / Q) * N : -1;   // stage A stores
    const int s = ways(w);
    if (s < best) {
      best = s;
      r.R = R;
    }
  }
  return r;
}
}  // namespace lay

template <int N, int NC, int Q>
struct F3 {
  static constexpr lay::F3L v = lay::pick_f3(N, NC, Q);
  static constexpr int N1 = v.N1, P1 = v.P1, MS = v.MS;
};
template <int N, int NC, int Q>
struct F2 {
  static constexpr int R = lay::pick_f2(N, NC, Q);
};
template <int N, int NC, int Q>
struct B3 {
  static constexpr lay::B3L v = lay::pick_b3(N, NC, Q);
  static constexpr int NQp = v.NQp, CA = v.CA, SA = v.SA, RB = v.RB;
};
template <int N, int NC, int Q>
struct B2 {
  static constexpr lay::B2L v = lay::pick_b2(N, NC, Q);
  static constexpr int NQp = v.NQp, R = v.R;
};

// Scratch (entries of T) of the forward contractions of NC fields (h1_fwd, and l2_fwd with
// N = K and N = K + 1) and of the backward ones (h1_bwd, l2_bwd with N = K and K + 1).
// Both forms are covered (the plan is sized in entries, whatever T is): the line form's
// padded layouts and the output-parallel form's plain ones (H1: t1 2 NC D^2 Q, t2 3 NC D Q^2,
// sf (DIM + 1) NC NQ in 3D; t1 2 NC D Q, sf (DIM + 1) NC NQ in 2D; L2 needs less).
template <int DIM, int K, int NC>
struct NeedF {
  static constexpr int D = K + 1, Q = 2 * K;
  static constexpr int T1n = DIM == 3 ? lay::imax(2 * Q * F3<D, NC, Q>::P1, Q * F3<K, NC, Q>::P1)
                                      : lay::imax(2 * Q * F2<D, NC, Q>::R, Q * F2<K, NC, Q>::R);
  static constexpr int T2n = DIM == 3 ? lay::imax(3 * Q * Q * F3<D, NC, Q>::MS, Q * Q * F3<K, NC, Q>::MS) : 1;
  static constexpr int T1 = lay::imax(T1n, DIM == 3 ? 2 * NC * D * D * Q : 2 * NC * D * Q);
  static constexpr int T2 = lay::imax(T2n, DIM == 3 ? 3 * NC * D * Q * Q : 1);
};
template <int DIM, int K, int NC>
struct NeedB {
  static constexpr int D = K + 1, Q = 2 * K, NQ = DIM == 3 ? Q * Q * Q : Q * Q;
  static constexpr int SFn = DIM == 3 ? lay::imax(4 * NC * B3<D, NC, Q>::NQp, NC * B3<K, NC, Q>::NQp)
                                      : lay::imax(3 * NC * B2<D, NC, Q>::NQp, NC * B2<K, NC, Q>::NQp);
  static constexpr int T2n = DIM == 3 ? lay::imax(3 * D * B3<D, NC, Q>::SA, K * B3<K, NC, Q>::SA) : 1;
  static constexpr int T1n = DIM == 3 ? lay::imax(2 * Q * B3<D, NC, Q>::RB, Q * B3<K, NC, Q>::RB)
                                      : lay::imax(2 * Q * B2<D, NC, Q>::R, Q * B2<K, NC, Q>::R);
  static constexpr int SF = lay::imax(SFn, (DIM + 1) * NC * NQ);
  static constexpr int T2 = lay::imax(T2n, DIM == 3 ? 3 * NC * D * Q * Q : 1);
  static constexpr int T1 = lay::imax(T1n, DIM == 3 ? 2 * NC * D * D * Q : 2 * NC * D * Q);
};
// the largest need over 1..NC fields (a kernel calls its contractions with up to NC fields)
template <int DIM, int K, int NC>
struct NeedFMax {
  using A = NeedF<DIM, K, NC>;
  using R = NeedFMax<DIM, K, NC - 1>;
  static constexpr int T1 = lay::imax(A::T1, R::T1), T2 = lay::imax(A::T2, R::T2);
};
template <int DIM, int K>
struct NeedFMax<DIM, K, 0> {
  static constexpr int T1 = 0, T2 = 0;
};
template <int DIM, int K, int NC>
struct NeedBMax {
  using A = NeedB<DIM, K, NC>;
  using R = NeedBMax<DIM, K, NC - 1>;
  static constexpr int SF = lay::imax(A::SF, R::SF), T1 = lay::imax(A::T1, R::T1), T2 = lay::imax(A::T2, R::T2);
};
template <int DIM, int K>
struct NeedBMax<DIM, K, 0> {
  static constexpr int SF = 0, T1 = 0, T2 = 0;
};

// ---------------------------------------------------------------------------------------
// Line form (see the header).
namespace ln {

// The line form's stages, one function per stage (no barriers inside); the entry points
// below put __syncthreads() between them, and the fused entry points run the H1 and L2
// stages of one direction in the same barrier phase (disjoint scratch).

// ---- forward, NC H1 fields: values (if VAL) and reference gradients at this point
template <int DIM, int K, int NC, class T, int NT = 0>
struct H1F {
  static constexpr int D = K + 1, Q = 2 * K, NM = NC * D;
  static constexpr int NS = NT ? NT : (DIM == 3 ? Q * Q * Q : Q * Q);   // threads per element
  // a0 -> q0, one thread per line (c, a2, a1) [3D] or (c, a1) [2D]
  static __device__ __forceinline__ void s1(const T* __restrict__ in, T* t1, int lt) {
    if constexpr (DIM == 3) {
      using LY = F3<D, NC, Q>;
      constexpr int N1 = LY::N1, P1 = LY::P1, T1P = Q * P1;
#pragma unroll
      for (int it = 0; it < (NM * D + NS - 1) / NS; ++it) {
        const int r = lt + it * NS;
        if (r >= NM * D) break;
        T u[D];
#pragma unroll
        for (int a0 = 0; a0 < D; ++a0) u[a0] = in[r * D + a0];
        const int o = (r / D) * N1 + r % D;
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) {
          T sb = 0, sg = 0;
#pragma unroll
          for (int a0 = 0; a0 < D; ++a0) {
            sb += cB<T, K>(q0, a0) * u[a0];
            sg += cG<T, K>(q0, a0) * u[a0];
          }
          t1[q0 * P1 + o] = sb;
          t1[T1P + q0 * P1 + o] = sg;
        }
      }
    } else {
      constexpr int R = F2<D, NC, Q>::R, T1P = Q * R;
#pragma unroll
      for (int it = 0; it < (NM + NS - 1) / NS; ++it) {
        const int r = lt + it * NS;
        if (r >= NM) break;
        T u[D];
#pragma unroll
        for (int a0 = 0; a0 < D; ++a0) u[a0] = in[r * D + a0];
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) {
          T sb = 0, sg = 0;
#pragma unroll
          for (int a0 = 0; a0 < D; ++a0) {
            sb += cB<T, K>(q0, a0) * u[a0];
            sg += cG<T, K>(q0, a0) * u[a0];
          }
          t1[q0 * R + r] = sb;
          t1[T1P + q0 * R + r] = sg;
        }
      }
    }
  }
  // a1 -> q1 (3D only), one thread per line (q0, c, a2)
  static __device__ __forceinline__ void s2(const T* t1, T* t2, int lt) {
    if constexpr (DIM == 3) {
      using LY = F3<D, NC, Q>;
      constexpr int N1 = LY::N1, P1 = LY::P1, MS = LY::MS, T1P = Q * P1, T2P = Q * Q * MS;
#pragma unroll
      for (int it = 0; it < (Q * NM + NS - 1) / NS; ++it) {
        const int n = lt + it * NS;
        if (n >= Q * NM) break;
        const int q0 = n / NM, m = n % NM;
        T xb[D], xg[D];
#pragma unroll
        for (int a1 = 0; a1 < D; ++a1) {
          xb[a1] = t1[q0 * P1 + m * N1 + a1];
          xg[a1] = t1[T1P + q0 * P1 + m * N1 + a1];
        }
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) {
          T bb = 0, bg = 0, gb = 0;
#pragma unroll
          for (int a1 = 0; a1 < D; ++a1) {
            const T b = cB<T, K>(q1, a1), g = cG<T, K>(q1, a1);
            bb += b * xb[a1];
            bg += g * xb[a1];
            gb += b * xg[a1];
          }
          const int o = (q1 * Q + q0) * MS + m;
          t2[o] = bb;
          t2[T2P + o] = bg;
          t2[2 * T2P + o] = gb;
        }
      }
    }
  }
  // the last direction at this thread's point (src: t2 in 3D, t1 in 2D); B, G: the tables in
  // shared memory (this thread's row)
  template <bool VAL>
  static __device__ __forceinline__ void s3(const T* src, const T* B, const T* G, int lt, T (&val)[NC],
                                            T (&grad)[NC][DIM]) {
    if constexpr (DIM == 3) {
      using LY = F3<D, NC, Q>;
      constexpr int MS = LY::MS, T2P = Q * Q * MS;
      const int q0 = lt % Q, q1 = (lt / Q) % Q, q2 = lt / (Q * Q);
      T b2[D], g2[D];
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2) {
        b2[a2] = B[q2 * D + a2];
        g2[a2] = G[q2 * D + a2];
      }
      const int pb = (q1 * Q + q0) * MS;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T v = 0, dx = 0, dy = 0, dz = 0;
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) {
          const int o = pb + c * D + a2;
          if constexpr (VAL) v += b2[a2] * src[o];
          dy += b2[a2] * src[T2P + o];
          dx += b2[a2] * src[2 * T2P + o];
          dz += g2[a2] * src[o];
        }
        val[c] = v;
        grad[c][0] = dx;
        grad[c][1] = dy;
        grad[c][2] = dz;
      }
    } else {
      constexpr int R = F2<D, NC, Q>::R, T1P = Q * R;
      const int q0 = lt % Q, q1 = lt / Q;
      T b1[D], g1[D];
#pragma unroll
      for (int a1 = 0; a1 < D; ++a1) {
        b1[a1] = B[q1 * D + a1];
        g1[a1] = G[q1 * D + a1];
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T v = 0, dx = 0, dy = 0;
#pragma unroll
        for (int a1 = 0; a1 < D; ++a1) {
          const int o = q0 * R + c * D + a1;
          v += b1[a1] * src[o];
          dx += b1[a1] * src[T1P + o];
          dy += g1[a1] * src[o];
        }
        val[c] = v;
        grad[c][0] = dx;
        grad[c][1] = dy;
      }
    }
  }
  // Paired form of s3 (T = float): this thread's two points differ in q0 only, (q0, q1, q2)
  // and (q0 + 1, q1, q2) with q0 = 2 (lt % (Q/2)) (pair_points); the last direction's table
  // row is common to both, the intermediates differ.
  template <bool VAL>
  static __device__ __forceinline__ void s3x2(const float* src, const float* B, const float* G, int lt,
                                              float2 (&val)[NC], float2 (&grad)[NC][DIM]) {
    constexpr int QH = Q / 2;
    if constexpr (DIM == 3) {
      using LY = F3<D, NC, Q>;
      constexpr int MS = LY::MS, T2P = Q * Q * MS;
      const int q0 = 2 * (lt % QH), q1 = (lt / QH) % Q, q2 = lt / (QH * Q);
      float2 b2[D], g2[D];
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2) {
        b2[a2] = f2s(B[q2 * D + a2]);
        g2[a2] = f2s(G[q2 * D + a2]);
      }
      const int pa = (q1 * Q + q0) * MS, pb = pa + MS;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float2 v = f2s(0.f), dx = v, dy = v, dz = v;
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) {
          const int o = c * D + a2;
          const float2 s0 = make_float2(src[pa + o], src[pb + o]);
          const float2 s1 = make_float2(src[T2P + pa + o], src[T2P + pb + o]);
          const float2 s2 = make_float2(src[2 * T2P + pa + o], src[2 * T2P + pb + o]);
          if (a2 == 0) {
            if constexpr (VAL) v = f2mul(b2[0], s0);
            dy = f2mul(b2[0], s1);
            dx = f2mul(b2[0], s2);
            dz = f2mul(g2[0], s0);
          } else {
            if constexpr (VAL) v = f2fma(b2[a2], s0, v);
            dy = f2fma(b2[a2], s1, dy);
            dx = f2fma(b2[a2], s2, dx);
            dz = f2fma(g2[a2], s0, dz);
          }
        }
        val[c] = v;
        grad[c][0] = dx;
        grad[c][1] = dy;
        grad[c][2] = dz;
      }
    } else {
      constexpr int R = F2<D, NC, Q>::R, T1P = Q * R;
      const int q0 = 2 * (lt % QH), q1 = lt / QH;
      float2 b1[D], g1[D];
#pragma unroll
      for (int a1 = 0; a1 < D; ++a1) {
        b1[a1] = f2s(B[q1 * D + a1]);
        g1[a1] = f2s(G[q1 * D + a1]);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float2 v = f2s(0.f), dx = v, dy = v;
#pragma unroll
        for (int a1 = 0; a1 < D; ++a1) {
          const int o = q0 * R + c * D + a1;
          const float2 s0 = make_float2(src[o], src[o + R]);
          const float2 s1 = make_float2(src[T1P + o], src[T1P + o + R]);
          if (a1 == 0) {
            v = f2mul(b1[0], s0);
            dx = f2mul(b1[0], s1);
            dy = f2mul(g1[0], s0);
          } else {
            v = f2fma(b1[a1], s0, v);
            dx = f2fma(b1[a1], s1, dx);
            dy = f2fma(g1[a1], s0, dy);
          }
        }
        val[c] = v;
        grad[c][0] = dx;
        grad[c][1] = dy;
      }
    }
  }
};

// ---- forward, NC fields with L 1D dofs: values at this point (table cL<T, K, L>)
template <int DIM, int K, int NC, class T, int L, int NT = 0>
struct L2F {
  static constexpr int Q = 2 * K, NM = NC * L;
  static constexpr int NS = NT ? NT : (DIM == 3 ? Q * Q * Q : Q * Q);
  static __device__ __forceinline__ void s1(const T* __restrict__ in, T* t1, int lt) {
    if constexpr (DIM == 3) {
      using LY = F3<L, NC, Q>;
      constexpr int N1 = LY::N1, P1 = LY::P1;
#pragma unroll
      for (int it = 0; it < (NM * L + NS - 1) / NS; ++it) {
        const int r = lt + it * NS;
        if (r >= NM * L) break;            // j0 -> q0, line (c, j2, j1)
        T u[L];
#pragma unroll
        for (int j0 = 0; j0 < L; ++j0) u[j0] = in[r * L + j0];
        const int o = (r / L) * N1 + r % L;
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) {
          T s = 0;
#pragma unroll
          for (int j0 = 0; j0 < L; ++j0) s += cL<T, K, L>(q0, j0) * u[j0];
          t1[q0 * P1 + o] = s;
        }
      }
    } else {
      constexpr int R = F2<L, NC, Q>::R;
#pragma unroll
      for (int it = 0; it < (NM + NS - 1) / NS; ++it) {
        const int r = lt + it * NS;
        if (r >= NM) break;                // j0 -> q0, line (c, j1)
        T u[L];
#pragma unroll
        for (int j0 = 0; j0 < L; ++j0) u[j0] = in[r * L + j0];
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) {
          T s = 0;
#pragma unroll
          for (int j0 = 0; j0 < L; ++j0) s += cL<T, K, L>(q0, j0) * u[j0];
          t1[q0 * R + r] = s;
        }
      }
    }
  }
  static __device__ __forceinline__ void s2(const T* t1, T* t2, int lt) {
    if constexpr (DIM == 3) {
      using LY = F3<L, NC, Q>;
      constexpr int N1 = LY::N1, P1 = LY::P1, MS = LY::MS;
#pragma unroll
      for (int it = 0; it < (Q * NM + NS - 1) / NS; ++it) {
        const int n = lt + it * NS;
        if (n >= Q * NM) break;            // j1 -> q1, line (q0, c, j2)
        const int q0 = n / NM, m = n % NM;
        T x[L];
#pragma unroll
        for (int j1 = 0; j1 < L; ++j1) x[j1] = t1[q0 * P1 + m * N1 + j1];
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) {
          T s = 0;
#pragma unroll
          for (int j1 = 0; j1 < L; ++j1) s += cL<T, K, L>(q1, j1) * x[j1];
          t2[(q1 * Q + q0) * MS + m] = s;
        }
      }
    }
  }
  // Bl: the table in shared memory (this thread's row)
  static __device__ __forceinline__ void s3(const T* src, const T* Bl, int lt, T (&val)[NC]) {
    if constexpr (DIM == 3) {
      constexpr int MS = F3<L, NC, Q>::MS;
      const int q0 = lt % Q, q1 = (lt / Q) % Q, q2 = lt / (Q * Q);
      T b2[L];
#pragma unroll
      for (int j2 = 0; j2 < L; ++j2) b2[j2] = Bl[q2 * L + j2];
      const int pb = (q1 * Q + q0) * MS;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T s = 0;
#pragma unroll
        for (int j2 = 0; j2 < L; ++j2) s += b2[j2] * src[pb + c * L + j2];
        val[c] = s;
      }
    } else {
      constexpr int R = F2<L, NC, Q>::R;
      const int q0 = lt % Q, q1 = lt / Q;
      T b1[L];
#pragma unroll
      for (int j1 = 0; j1 < L; ++j1) b1[j1] = Bl[q1 * L + j1];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T s = 0;
#pragma unroll
        for (int j1 = 0; j1 < L; ++j1) s += b1[j1] * src[q0 * R + c * L + j1];
        val[c] = s;
      }
    }
  }
  // paired form of s3 (the points of H1F::s3x2)
  static __device__ __forceinline__ void s3x2(const float* src, const float* Bl, int lt, float2 (&val)[NC]) {
    constexpr int QH = Q / 2;
    if constexpr (DIM == 3) {
      constexpr int MS = F3<L, NC, Q>::MS;
      const int q0 = 2 * (lt % QH), q1 = (lt / QH) % Q, q2 = lt / (QH * Q);
      float2 b2[L];
#pragma unroll
      for (int j2 = 0; j2 < L; ++j2) b2[j2] = f2s(Bl[q2 * L + j2]);
      const int pa = (q1 * Q + q0) * MS, pb = pa + MS;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float2 v = f2mul(b2[0], make_float2(src[pa + c * L], src[pb + c * L]));
#pragma unroll
        for (int j2 = 1; j2 < L; ++j2) v = f2fma(b2[j2], make_float2(src[pa + c * L + j2], src[pb + c * L + j2]), v);
        val[c] = v;
      }
    } else {
      constexpr int R = F2<L, NC, Q>::R;
      const int q0 = 2 * (lt % QH), q1 = lt / QH;
      float2 b1[L];
#pragma unroll
      for (int j1 = 0; j1 < L; ++j1) b1[j1] = f2s(Bl[q1 * L + j1]);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int o = q0 * R + c * L;
        float2 v = f2mul(b1[0], make_float2(src[o], src[o + R]));
#pragma unroll
        for (int j1 = 1; j1 < L; ++j1) v = f2fma(b1[j1], make_float2(src[o + j1], src[o + R + j1]), v);
        val[c] = v;
      }
    }
  }
};

// ---- backward, NC H1 fields: out[c][a] = sum_q (fval w_a + fgrad . grad w_a)
template <int DIM, int K, int NC, class T, int NT = 0>
struct H1B {
  static constexpr int D = K + 1, Q = 2 * K, NM = NC * D;
  static constexpr int NS = NT ? NT : (DIM == 3 ? Q * Q * Q : Q * Q);
  // phase 0: the point values into sf
  static __device__ __forceinline__ void p0(const T (&fval)[NC], const T (&fgrad)[NC][DIM], T* sf, int lt) {
    if constexpr (DIM == 3) {
      constexpr int NQp = B3<D, NC, Q>::NQp, SFP = NC * NQp;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        sf[c * NQp + lt] = fval[c];
        sf[SFP + c * NQp + lt] = fgrad[c][0];
        sf[2 * SFP + c * NQp + lt] = fgrad[c][1];
        sf[3 * SFP + c * NQp + lt] = fgrad[c][2];
      }
    } else {
      constexpr int NQp = B2<D, NC, Q>::NQp, SFP = NC * NQp;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        sf[c * NQp + lt] = fval[c];
        sf[SFP + c * NQp + lt] = fgrad[c][0];
        sf[2 * SFP + c * NQp + lt] = fgrad[c][1];
      }
    }
  }
  // paired form of p0 (the points of H1F::s3x2, adjacent in sf: one 8-byte store per value
  // when the row stride is even)
  static __device__ __forceinline__ void p0x2(const float2 (&fval)[NC], const float2 (&fgrad)[NC][DIM], float* sf,
                                              int lt) {
    constexpr int QH = Q / 2;
    constexpr int NQp = DIM == 3 ? B3<D, NC, Q>::NQp : B2<D, NC, Q>::NQp, SFP = NC * NQp;
    const int p = 2 * (lt % QH) + Q * (lt / QH);
    auto st = [&](int o, float2 v) {
      if constexpr (NQp % 2 == 0) {
        *reinterpret_cast<float2*>(sf + o) = v;
      } else {
        sf[o] = v.x;
        sf[o + 1] = v.y;
      }
    };
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      st(c * NQp + p, fval[c]);
#pragma unroll
      for (int d = 0; d < DIM; ++d) st((d + 1) * SFP + c * NQp + p, fgrad[c][d]);
    }
  }
  // phase 1: 3D q2 -> a2 (sf -> t2), line (c, q1, q0); 2D q1 -> a1 (sf -> t1), line (c, q0)
  static __device__ __forceinline__ void p1(const T* sf, T* t1, T* t2, int lt) {
    if constexpr (DIM == 3) {
      constexpr int QQ = Q * Q;
      using LY = B3<D, NC, Q>;
      constexpr int NQp = LY::NQp, CA = LY::CA, SA = LY::SA, SFP = NC * NQp, T2P = D * SA;
#pragma unroll
      for (int it = 0; it < (NC * QQ + NS - 1) / NS; ++it) {
        const int n = lt + it * NS;
        if (n >= NC * QQ) break;
        const int c = n / QQ, p = n % QQ;
        T f0[Q], f1[Q], f2[Q], f3[Q];
#pragma unroll
        for (int q2 = 0; q2 < Q; ++q2) {
          const int o = c * NQp + q2 * QQ + p;
          f0[q2] = sf[o];
          f1[q2] = sf[SFP + o];
          f2[q2] = sf[2 * SFP + o];
          f3[q2] = sf[3 * SFP + o];
        }
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) {
          T zbb = 0, zbg = 0, zgb = 0;
#pragma unroll
          for (int q2 = 0; q2 < Q; ++q2) {
            const T b = cB<T, K>(q2, a2), g = cG<T, K>(q2, a2);
            zgb += b * f1[q2];
            zbg += b * f2[q2];
            zbb += b * f0[q2] + g * f3[q2];
          }
          const int o = a2 * SA + c * CA + p;
          t2[o] = zbb;
          t2[T2P + o] = zbg;
          t2[2 * T2P + o] = zgb;
        }
      }
    } else {
      using LY = B2<D, NC, Q>;
      constexpr int NQp = LY::NQp, R = LY::R, SFP = NC * NQp, T1P = Q * R;
#pragma unroll
      for (int it = 0; it < (NC * Q + NS - 1) / NS; ++it) {
        const int n = lt + it * NS;
        if (n >= NC * Q) break;
        const int c = n / Q, q0 = n % Q;
        T f0[Q], f1[Q], f2[Q];
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) {
          const int o = c * NQp + q1 * Q + q0;
          f0[q1] = sf[o];
          f1[q1] = sf[SFP + o];
          f2[q1] = sf[2 * SFP + o];
        }
#pragma unroll
        for (int a1 = 0; a1 < D; ++a1) {
          T yb = 0, yg = 0;
#pragma unroll
          for (int q1 = 0; q1 < Q; ++q1) {
            const T b = cB<T, K>(q1, a1), g = cG<T, K>(q1, a1);
            yg += b * f1[q1];
            yb += b * f0[q1] + g * f2[q1];
          }
          const int o = q0 * R + c * D + a1;
          t1[o] = yb;
          t1[T1P + o] = yg;
        }
      }
      (void)t2;
    }
  }
  // phase 2: 3D q1 -> a1 (t2 -> t1), line (c, a2, q0); 2D q0 -> a0 (t1 -> out), line (c, a1)
  static __device__ __forceinline__ void p2(T* t1, const T* t2, int lt, T* out) {
    if constexpr (DIM == 3) {
      constexpr int QQ = Q * Q;
      using LY = B3<D, NC, Q>;
      constexpr int CA = LY::CA, SA = LY::SA, RB = LY::RB, T2P = D * SA, T1P = Q * RB;
#pragma unroll
      for (int it = 0; it < (NM * Q + NS - 1) / NS; ++it) {
        const int n = lt + it * NS;
        if (n >= NM * Q) break;
        const int q0 = n % Q, m = n / Q, c = m / D, a2 = m % D;
        T zb[Q], zbg[Q], zgb[Q];
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) {
          const int o = a2 * SA + c * CA + q1 * Q + q0;
          zb[q1] = t2[o];
          zbg[q1] = t2[T2P + o];
          zgb[q1] = t2[2 * T2P + o];
        }
#pragma unroll
        for (int a1 = 0; a1 < D; ++a1) {
          T yb = 0, yg = 0;
#pragma unroll
          for (int q1 = 0; q1 < Q; ++q1) {
            const T b = cB<T, K>(q1, a1), g = cG<T, K>(q1, a1);
            yg += b * zgb[q1];
            yb += g * zbg[q1] + b * zb[q1];
          }
          const int o = q0 * RB + m * D + a1;
          t1[o] = yb;
          t1[T1P + o] = yg;
        }
      }
      (void)out;
    } else {
      using LY = B2<D, NC, Q>;
      constexpr int R = LY::R, T1P = Q * R;
#pragma unroll
      for (int it = 0; it < (NM + NS - 1) / NS; ++it) {
        const int r = lt + it * NS;
        if (r >= NM) break;
        T yb[Q], yg[Q];
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) {
          yb[q0] = t1[q0 * R + r];
          yg[q0] = t1[T1P + q0 * R + r];
        }
#pragma unroll
        for (int a0 = 0; a0 < D; ++a0) {
          T s = 0;
#pragma unroll
          for (int q0 = 0; q0 < Q; ++q0) s += cG<T, K>(q0, a0) * yg[q0] + cB<T, K>(q0, a0) * yb[q0];
          out[r * D + a0] = s;
        }
      }
      (void)t2;
    }
  }
  // phase 3 (3D only): q0 -> a0 (t1 -> out), line (c, a2, a1)
  static __device__ __forceinline__ void p3(const T* t1, int lt, T* out) {
    if constexpr (DIM == 3) {
      constexpr int RB = B3<D, NC, Q>::RB, T1P = Q * RB;
#pragma unroll
      for (int it = 0; it < (NM * D + NS - 1) / NS; ++it) {
        const int r = lt + it * NS;
        if (r >= NM * D) break;
        T yb[Q], yg[Q];
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) {
          yb[q0] = t1[q0 * RB + r];
          yg[q0] = t1[T1P + q0 * RB + r];
        }
#pragma unroll
        for (int a0 = 0; a0 < D; ++a0) {
          T s = 0;
#pragma unroll
          for (int q0 = 0; q0 < Q; ++q0) s += cG<T, K>(q0, a0) * yg[q0] + cB<T, K>(q0, a0) * yb[q0];
          out[r * D + a0] = s;
        }
      }
    }
  }
};

// ---- backward, NC fields with L 1D dofs: out[c][j] = sum_q fval phi_j(q)
template <int DIM, int K, int NC, class T, int L, int NT = 0>
struct L2B {
  static constexpr int Q = 2 * K, NM = NC * L;
  static constexpr int NS = NT ? NT : (DIM == 3 ? Q * Q * Q : Q * Q);
  static __device__ __forceinline__ void p0(const T (&fval)[NC], T* sf, int lt) {
    constexpr int NQp = DIM == 3 ? B3<L, NC, Q>::NQp : B2<L, NC, Q>::NQp;
#pragma unroll
    for (int c = 0; c < NC; ++c) sf[c * NQp + lt] = fval[c];
  }
  static __device__ __forceinline__ void p0x2(const float2 (&fval)[NC], float* sf, int lt) {
    constexpr int QH = Q / 2;
    constexpr int NQp = DIM == 3 ? B3<L, NC, Q>::NQp : B2<L, NC, Q>::NQp;
    const int p = 2 * (lt % QH) + Q * (lt / QH);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if constexpr (NQp % 2 == 0) {
        *reinterpret_cast<float2*>(sf + c * NQp + p) = fval[c];
      } else {
        sf[c * NQp + p] = fval[c].x;
        sf[c * NQp + p + 1] = fval[c].y;
      }
    }
  }
  static __device__ __forceinline__ void p1(const T* sf, T* t1, T* t2, int lt) {
    if constexpr (DIM == 3) {
      constexpr int QQ = Q * Q;
      using LY = B3<L, NC, Q>;
      constexpr int NQp = LY::NQp, CA = LY::CA, SA = LY::SA;
#pragma unroll
      for (int it = 0; it < (NC * QQ + NS - 1) / NS; ++it) {
        const int n = lt + it * NS;
        if (n >= NC * QQ) break;           // q2 -> j2, line (c, q1, q0)
        const int c = n / QQ, p = n % QQ;
        T f[Q];
#pragma unroll
        for (int q2 = 0; q2 < Q; ++q2) f[q2] = sf[c * NQp + q2 * QQ + p];
#pragma unroll
        for (int j2 = 0; j2 < L; ++j2) {
          T s = 0;
#pragma unroll
          for (int q2 = 0; q2 < Q; ++q2) s += cL<T, K, L>(q2, j2) * f[q2];
          t2[j2 * SA + c * CA + p] = s;
        }
      }
      (void)t1;
    } else {
      using LY = B2<L, NC, Q>;
      constexpr int NQp = LY::NQp, R = LY::R;
#pragma unroll
      for (int it = 0; it < (NC * Q + NS - 1) / NS; ++it) {
        const int n = lt + it * NS;
        if (n >= NC * Q) break;            // q1 -> j1, line (c, q0)
        const int c = n / Q, q0 = n % Q;
        T f[Q];
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) f[q1] = sf[c * NQp + q1 * Q + q0];
#pragma unroll
        for (int j1 = 0; j1 < L; ++j1) {
          T s = 0;
#pragma unroll
          for (int q1 = 0; q1 < Q; ++q1) s += cL<T, K, L>(q1, j1) * f[q1];
          t1[q0 * R + c * L + j1] = s;
        }
      }
      (void)t2;
    }
  }
  static __device__ __forceinline__ void p2(T* t1, const T* t2, int lt, T* out) {
    if constexpr (DIM == 3) {
      constexpr int QQ = Q * Q;
      using LY = B3<L, NC, Q>;
      constexpr int CA = LY::CA, SA = LY::SA, RB = LY::RB;
#pragma unroll
      for (int it = 0; it < (NM * Q + NS - 1) / NS; ++it) {
        const int n = lt + it * NS;
        if (n >= NM * Q) break;            // q1 -> j1, line (c, j2, q0)
        const int q0 = n % Q, m = n / Q, c = m / L, j2 = m % L;
        T zz[Q];
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) zz[q1] = t2[j2 * SA + c * CA + q1 * Q + q0];
#pragma unroll
        for (int j1 = 0; j1 < L; ++j1) {
          T s = 0;
#pragma unroll
          for (int q1 = 0; q1 < Q; ++q1) s += cL<T, K, L>(q1, j1) * zz[q1];
          t1[q0 * RB + m * L + j1] = s;
        }
      }
      (void)out;
    } else {
      constexpr int R = B2<L, NC, Q>::R;
#pragma unroll
      for (int it = 0; it < (NM + NS - 1) / NS; ++it) {
        const int r = lt + it * NS;
        if (r >= NM) break;                // q0 -> j0, line (c, j1)
        T y[Q];
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) y[q0] = t1[q0 * R + r];
#pragma unroll
        for (int j0 = 0; j0 < L; ++j0) {
          T s = 0;
#pragma unroll
          for (int q0 = 0; q0 < Q; ++q0) s += cL<T, K, L>(q0, j0) * y[q0];
          out[r * L + j0] = s;
        }
      }
      (void)t2;
    }
  }
  static __device__ __forceinline__ void p3(const T* t1, int lt, T* out) {
    if constexpr (DIM == 3) {
      constexpr int RB = B3<L, NC, Q>::RB;
#pragma unroll
      for (int it = 0; it < (NM * L + NS - 1) / NS; ++it) {
        const int r = lt + it * NS;
        if (r >= NM * L) break;            // q0 -> j0, line (c, j2, j1)
        T y[Q];
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) y[q0] = t1[q0 * RB + r];
#pragma unroll
        for (int j0 = 0; j0 < L; ++j0) {
          T s = 0;
#pragma unroll
          for (int q0 = 0; q0 < Q; ++q0) s += cL<T, K, L>(q0, j0) * y[q0];
          out[r * L + j0] = s;
        }
      }
    }
  }
};

// ---- entry points: the stages with a barrier after each phase
template <int DIM, int K, int NC, class T, bool VAL = true>
__device__ __forceinline__ void h1_fwd(const T* __restrict__ in, T* t1, T* t2, const T* B, const T* G,
                                       int lt, T (&val)[NC], T (&grad)[NC][DIM]) {
  using S = H1F<DIM, K, NC, T>;
  S::s1(in, t1, lt);
  __syncthreads();
  if constexpr (DIM == 3) {
    S::s2(t1, t2, lt);
    __syncthreads();
  }
  S::template s3<VAL>(DIM == 3 ? t2 : t1, B, G, lt, val, grad);
  __syncthreads();
}
template <int DIM, int K, int NC, class T, int L_ = K>
__device__ __forceinline__ void l2_fwd(const T* __restrict__ in, T* t1, T* t2, const T* Bl, int lt, T (&val)[NC]) {
  using S = L2F<DIM, K, NC, T, L_>;
  S::s1(in, t1, lt);
  __syncthreads();
  if constexpr (DIM == 3) {
    S::s2(t1, t2, lt);
    __syncthreads();
  }
  S::s3(DIM == 3 ? t2 : t1, Bl, lt, val);
  __syncthreads();
}
template <int DIM, int K, int NC, class T>
__device__ __forceinline__ void h1_bwd(const T (&fval)[NC], const T (&fgrad)[NC][DIM], T* sf, T* t1, T* t2,
                                       const T* B, const T* G, int lt, T* out) {
  using S = H1B<DIM, K, NC, T>;
  (void)B;
  (void)G;
  S::p0(fval, fgrad, sf, lt);
  __syncthreads();
  S::p1(sf, t1, t2, lt);
  __syncthreads();
  S::p2(t1, t2, lt, out);
  __syncthreads();
  if constexpr (DIM == 3) {
    S::p3(t1, lt, out);
    __syncthreads();
  }
}
template <int DIM, int K, int NC, class T, int L_ = K>
__device__ __forceinline__ void l2_bwd(const T (&fval)[NC], T* sf, T* t1, T* t2, const T* Bl, int lt, T* out) {
  using S = L2B<DIM, K, NC, T, L_>;
  (void)Bl;
  S::p0(fval, sf, lt);
  __syncthreads();
  S::p1(sf, t1, t2, lt);
  __syncthreads();
  S::p2(t1, t2, lt, out);
  __syncthreads();
  if constexpr (DIM == 3) {
    S::p3(t1, lt, out);
    __syncthreads();
  }
}

// H1 and L2 fields together, each phase of both under one barrier; the L2 stages use their
// own scratch (u1, u2, sfl: L2Scratch sizes)
template <int DIM, int K, int NC, int NCL, class T, bool VAL = true>
__device__ __forceinline__ void h1l2_fwd(const T* __restrict__ in, const T* __restrict__ inl, T* t1, T* t2, T* u1,
                                         T* u2, const T* B, const T* G, const T* Bl, int lt, T (&val)[NC],
                                         T (&grad)[NC][DIM], T (&lval)[NCL]) {
  using S = H1F<DIM, K, NC, T>;
  using SL = L2F<DIM, K, NCL, T, K>;
  S::s1(in, t1, lt);
  SL::s1(inl, u1, lt);
  __syncthreads();
  if constexpr (DIM == 3) {
    S::s2(t1, t2, lt);
    SL::s2(u1, u2, lt);
    __syncthreads();
  }
  S::template s3<VAL>(DIM == 3 ? t2 : t1, B, G, lt, val, grad);
  SL::s3(DIM == 3 ? u2 : u1, Bl, lt, lval);
  __syncthreads();
}
template <int DIM, int K, int NC, int NCL, class T>
__device__ __forceinline__ void h1l2_bwd(const T (&fval)[NC], const T (&fgrad)[NC][DIM], const T (&lval)[NCL],
                                         T* sf, T* t1, T* t2, T* sfl, T* u1, T* u2, int lt, T* out, T* outl) {
  using S = H1B<DIM, K, NC, T>;
  using SL = L2B<DIM, K, NCL, T, K>;
  S::p0(fval, fgrad, sf, lt);
  SL::p0(lval, sfl, lt);
  __syncthreads();
  S::p1(sf, t1, t2, lt);
  SL::p1(sfl, u1, u2, lt);
  __syncthreads();
  S::p2(t1, t2, lt, out);
  SL::p2(u1, u2, lt, outl);
  __syncthreads();
  if constexpr (DIM == 3) {
    S::p3(t1, lt, out);
    SL::p3(u1, lt, outl);
    __syncthreads();
  }
}

// Paired fused entry points (T = float, NT threads per element, two points per thread):
// the line stages stride over NT threads; SYNC is the barrier between phases (__syncwarp
// when the element's threads are one warp or part of one, else __syncthreads).
template <bool WARP>
__device__ __forceinline__ void esync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}
template <int DIM, int K, int NC, int NCL, int NT, bool WARP, bool VAL = true>
__device__ __forceinline__ void h1l2_fwd_x2(const float* __restrict__ in, const float* __restrict__ inl, float* t1,
                                            float* t2, float* u1, float* u2, const float* B, const float* G,
                                            const float* Bl, int lt, float2 (&val)[NC], float2 (&grad)[NC][DIM],
                                            float2 (&lval)[NCL]) {
  using S = H1F<DIM, K, NC, float, NT>;
  using SL = L2F<DIM, K, NCL, float, K, NT>;
  S::s1(in, t1, lt);
  SL::s1(inl, u1, lt);
  esync<WARP>();
  if constexpr (DIM == 3) {
    S::s2(t1, t2, lt);
    SL::s2(u1, u2, lt);
    esync<WARP>();
  }
  S::template s3x2<VAL>(DIM == 3 ? t2 : t1, B, G, lt, val, grad);
  SL::s3x2(DIM == 3 ? u2 : u1, Bl, lt, lval);
  esync<WARP>();
}
template <int DIM, int K, int NC, int NCL, int NT, bool WARP>
__device__ __forceinline__ void h1l2_bwd_x2(const float2 (&fval)[NC], const float2 (&fgrad)[NC][DIM],
                                            const float2 (&lval)[NCL], float* sf, float* t1, float* t2, float* sfl,
                                            float* u1, float* u2, int lt, float* out, float* outl) {
  using S = H1B<DIM, K, NC, float, NT>;
  using SL = L2B<DIM, K, NCL, float, K, NT>;
  S::p0x2(fval, fgrad, sf, lt);
  SL::p0x2(lval, sfl, lt);
  esync<WARP>();
  S::p1(sf, t1, t2, lt);
  SL::p1(sfl, u1, u2, lt);
  esync<WARP>();
  S::p2(t1, t2, lt, out);
  SL::p2(u1, u2, lt, outl);
  esync<WARP>();
  if constexpr (DIM == 3) {
    S::p3(t1, lt, out);
    SL::p3(u1, lt, outl);
    esync<WARP>();
  }
}

// L2 scratch of the fused entry points (entries of T): forward t1, t2 and backward sf, t1, t2
// for NCL fields with K 1D dofs
template <int DIM, int K, int NCL>
struct L2Scratch {
  static constexpr int Q = 2 * K;
  static constexpr int U1 = DIM == 3 ? lay::imax(Q * F3<K, NCL, Q>::P1, Q * B3<K, NCL, Q>::RB)
                                     : lay::imax(Q * F2<K, NCL, Q>::R, Q * B2<K, NCL, Q>::R);
  static constexpr int U2 = DIM == 3 ? lay::imax(Q * Q * F3<K, NCL, Q>::MS, K * B3<K, NCL, Q>::SA) : 1;
  static constexpr int SF = NCL * (DIM == 3 ? B3<K, NCL, Q>::NQp : B2<K, NCL, Q>::NQp);
  static constexpr int ALL = U1 + U2 + SF;
};

}  // namespace ln

// ---------------------------------------------------------------------------------------
// Output-parallel form: the threads of an element stride over the outputs of each stage,
// every output reading its table entries from shared memory.
namespace op {

// values (if VAL; 3D only skips them) and reference gradients of NC H1 fields at this
// thread's quadrature point
template <int DIM, int K, int NC, class T, bool VAL = true>
__device__ __forceinline__ void h1_fwd(const T* __restrict__ in, T* t1, T* t2, const T* B, const T* G,
                                       int lt, T (&val)[NC], T (&grad)[NC][DIM]) {
  constexpr int D = K + 1, Q = 2 * K;
  if constexpr (DIM == 3) {
    constexpr int NQ = Q * Q * Q, S1 = NC * D * D * Q, S2 = NC * D * Q * Q;
    for (int i = lt; i < S1; i += NQ) {              // contract a0 -> q0
      const int q0 = i % Q, r = i / Q;
      const T* u = in + r * D;
      T sb = 0, sg = 0;
#pragma unroll
      for (int a0 = 0; a0 < D; ++a0) {
        sb += B[q0 * D + a0] * u[a0];
        sg += G[q0 * D + a0] * u[a0];
      }
      t1[i] = sb;
      t1[S1 + i] = sg;
    }
    __syncthreads();
    for (int i = lt; i < S2; i += NQ) {              // contract a1 -> q1
      const int q0 = i % Q, q1 = (i / Q) % Q, r = i / (Q * Q);
      const T* sb = t1 + r * D * Q + q0;
      const T* sg = t1 + S1 + r * D * Q + q0;
      T bb = 0, bg = 0, gb = 0;
#pragma unroll
      for (int a1 = 0; a1 < D; ++a1) {
        const T b = B[q1 * D + a1], g = G[q1 * D + a1];
        const T xb = sb[a1 * Q], xg = sg[a1 * Q];
        bb += b * xb;
        bg += g * xb;
        gb += b * xg;
      }
      t2[i] = bb;
      t2[S2 + i] = bg;
      t2[2 * S2 + i] = gb;
    }
    __syncthreads();
    const int q0 = lt % Q, q1 = (lt / Q) % Q, q2 = lt / (Q * Q);
#pragma unroll
    for (int c = 0; c < NC; ++c) {                   // contract a2 -> q2
      const int base = c * D * Q * Q + q1 * Q + q0;
      T v = 0, dx = 0, dy = 0, dz = 0;
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2) {
        const T b = B[q2 * D + a2], g = G[q2 * D + a2];
        const int o = base + a2 * Q * Q;
        if constexpr (VAL) v += b * t2[o];
        dy += b * t2[S2 + o];
        dx += b * t2[2 * S2 + o];
        dz += g * t2[o];
      }
      val[c] = v;
      grad[c][0] = dx;
      grad[c][1] = dy;
      grad[c][2] = dz;
    }
    __syncthreads();
  } else {
    constexpr int NQ = Q * Q, S1 = NC * D * Q;
    for (int i = lt; i < S1; i += NQ) {
      const int q0 = i % Q, r = i / Q;
      const T* u = in + r * D;
      T sb = 0, sg = 0;
#pragma unroll
      for (int a0 = 0; a0 < D; ++a0) {
        sb += B[q0 * D + a0] * u[a0];
        sg += G[q0 * D + a0] * u[a0];
      }
      t1[i] = sb;
      t1[S1 + i] = sg;
    }
    __syncthreads();
    const int q0 = lt % Q, q1 = lt / Q;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T v = 0, dx = 0, dy = 0;
#pragma unroll
      for (int a1 = 0; a1 < D; ++a1) {
        const T b = B[q1 * D + a1], g = G[q1 * D + a1];
        const int o = (c * D + a1) * Q + q0;
        v += b * t1[o];
        dx += b * t1[S1 + o];
        dy += g * t1[o];
      }
      val[c] = v;
      grad[c][0] = dx;
      grad[c][1] = dy;
    }
    __syncthreads();
  }
}

// out[c][a] = sum_q ( fval[c] w_a(q) + sum_r fgrad[c][r] d_r w_a(q) )   (B^T and G^T)
template <int DIM, int K, int NC, class T>
__device__ __forceinline__ void h1_bwd(const T (&fval)[NC], const T (&fgrad)[NC][DIM], T* sf, T* t1, T* t2,
                                       const T* B, const T* G, int lt, T* out) {
  constexpr int D = K + 1, Q = 2 * K;
  if constexpr (DIM == 3) {
    constexpr int NQ = Q * Q * Q, S1 = NC * D * D * Q, S2 = NC * D * Q * Q, ND = D * D * D;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      sf[c * NQ + lt] = fval[c];
      sf[(NC + c) * NQ + lt] = fgrad[c][0];
      sf[(2 * NC + c) * NQ + lt] = fgrad[c][1];
      sf[(3 * NC + c) * NQ + lt] = fgrad[c][2];
    }
    __syncthreads();
    for (int i = lt; i < S2; i += NQ) {              // q2 -> a2
      const int q0 = i % Q, q1 = (i / Q) % Q, a2 = (i / (Q * Q)) % D, c = i / (Q * Q * D);
      T zbb = 0, zbg = 0, zgb = 0;
#pragma unroll
      for (int q2 = 0; q2 < Q; ++q2) {
        const T b = B[q2 * D + a2], g = G[q2 * D + a2];
        const int qi = (q2 * Q + q1) * Q + q0;
        zgb += b * sf[(NC + c) * NQ + qi];
        zbg += b * sf[(2 * NC + c) * NQ + qi];
        zbb += b * sf[c * NQ + qi] + g * sf[(3 * NC + c) * NQ + qi];
      }
      t2[i] = zbb;
      t2[S2 + i] = zbg;
      t2[2 * S2 + i] = zgb;
    }
    __syncthreads();
    for (int i = lt; i < S1; i += NQ) {              // q1 -> a1
      const int q0 = i % Q, a1 = (i / Q) % D, r = i / (Q * D);
      T yb = 0, yg = 0;
#pragma unroll
      for (int q1 = 0; q1 < Q; ++q1) {
        const T b = B[q1 * D + a1], g = G[q1 * D + a1];
        const int o = (r * Q + q1) * Q + q0;
        yg += b * t2[2 * S2 + o];
        yb += g * t2[S2 + o] + b * t2[o];
      }
      t1[i] = yb;
      t1[S1 + i] = yg;
    }
    __syncthreads();
    for (int i = lt; i < NC * ND; i += NQ) {         // q0 -> a0
      const int a0 = i % D, r = i / D;
      T s = 0;
#pragma unroll
      for (int q0 = 0; q0 < Q; ++q0) s += G[q0 * D + a0] * t1[S1 + r * Q + q0] + B[q0 * D + a0] * t1[r * Q + q0];
      out[i] = s;
    }
    __syncthreads();
  } else {
    constexpr int NQ = Q * Q, S1 = NC * D * Q, ND = D * D;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      sf[c * NQ + lt] = fval[c];
      sf[(NC + c) * NQ + lt] = fgrad[c][0];
      sf[(2 * NC + c) * NQ + lt] = fgrad[c][1];
    }
    __syncthreads();
    for (int i = lt; i < S1; i += NQ) {              // q1 -> a1
      const int q0 = i % Q, a1 = (i / Q) % D, c = i / (Q * D);
      T yb = 0, yg = 0;
#pragma unroll
      for (int q1 = 0; q1 < Q; ++q1) {
        const T b = B[q1 * D + a1], g = G[q1 * D + a1];
        const int qi = q1 * Q + q0;
        yg += b * sf[(NC + c) * NQ + qi];
        yb += b * sf[c * NQ + qi] + g * sf[(2 * NC + c) * NQ + qi];
      }
      t1[i] = yb;
      t1[S1 + i] = yg;
    }
    __syncthreads();
    for (int i = lt; i < NC * ND; i += NQ) {         // q0 -> a0
      const int a0 = i % D, r = i / D;
      T s = 0;
#pragma unroll
      for (int q0 = 0; q0 < Q; ++q0) s += G[q0 * D + a0] * t1[S1 + r * Q + q0] + B[q0 * D + a0] * t1[r * Q + q0];
      out[i] = s;
    }
    __syncthreads();
  }
}

// values of NC fields with L_ 1D dofs (default: the L2 basis, L_ = K) at this thread's
// quadrature point; with L_ = K + 1 and the H1 table it interpolates H1 values only
template <int DIM, int K, int NC, class T, int L_ = K>
__device__ __forceinline__ void l2_fwd(const T* __restrict__ in, T* t1, T* t2, const T* Bl, int lt, T (&val)[NC]) {
  constexpr int L = L_, Q = 2 * K;
  if constexpr (DIM == 3) {
    constexpr int NQ = Q * Q * Q, S1 = NC * L * L * Q, S2 = NC * L * Q * Q;
    for (int i = lt; i < S1; i += NQ) {
      const int q0 = i % Q, r = i / Q;
      T s = 0;
#pragma unroll
      for (int j0 = 0; j0 < L; ++j0) s += Bl[q0 * L + j0] * in[r * L + j0];
      t1[i] = s;
    }
    __syncthreads();
    for (int i = lt; i < S2; i += NQ) {
      const int q0 = i % Q, q1 = (i / Q) % Q, r = i / (Q * Q);
      T s = 0;
#pragma unroll
      for (int j1 = 0; j1 < L; ++j1) s += Bl[q1 * L + j1] * t1[(r * L + j1) * Q + q0];
      t2[i] = s;
    }
    __syncthreads();
    const int q0 = lt % Q, q1 = (lt / Q) % Q, q2 = lt / (Q * Q);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T s = 0;
#pragma unroll
      for (int j2 = 0; j2 < L; ++j2) s += Bl[q2 * L + j2] * t2[((c * L + j2) * Q + q1) * Q + q0];
      val[c] = s;
    }
    __syncthreads();
  } else {
    constexpr int NQ = Q * Q, S1 = NC * L * Q;
    for (int i = lt; i < S1; i += NQ) {
      const int q0 = i % Q, r = i / Q;
      T s = 0;
#pragma unroll
      for (int j0 = 0; j0 < L; ++j0) s += Bl[q0 * L + j0] * in[r * L + j0];
      t1[i] = s;
    }
    __syncthreads();
    const int q0 = lt % Q, q1 = lt / Q;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T s = 0;
#pragma unroll
      for (int j1 = 0; j1 < L; ++j1) s += Bl[q1 * L + j1] * t1[(c * L + j1) * Q + q0];
      val[c] = s;
    }
    __syncthreads();
  }
}

// out[c][j] = sum_q fval[c] phi_j(q)  (L_ as in l2_fwd)
template <int DIM, int K, int NC, class T, int L_ = K>
__device__ __forceinline__ void l2_bwd(const T (&fval)[NC], T* sf, T* t1, T* t2, const T* Bl, int lt, T* out) {
  constexpr int L = L_, Q = 2 * K;
  if constexpr (DIM == 3) {
    constexpr int NQ = Q * Q * Q, S1 = NC * L * L * Q, S2 = NC * L * Q * Q, NL = L * L * L;
#pragma unroll
    for (int c = 0; c < NC; ++c) sf[c * NQ + lt] = fval[c];
    __syncthreads();
    for (int i = lt; i < S2; i += NQ) {              // q2 -> j2
      const int q0 = i % Q, q1 = (i / Q) % Q, j2 = (i / (Q * Q)) % L, c = i / (Q * Q * L);
      T s = 0;
#pragma unroll
      for (int q2 = 0; q2 < Q; ++q2) s += Bl[q2 * L + j2] * sf[c * NQ + (q2 * Q + q1) * Q + q0];
      t2[i] = s;
    }
    __syncthreads();
    for (int i = lt; i < S1; i += NQ) {              // q1 -> j1
      const int q0 = i % Q, j1 = (i / Q) % L, r = i / (Q * L);
      T s = 0;
#pragma unroll
      for (int q1 = 0; q1 < Q; ++q1) s += Bl[q1 * L + j1] * t2[(r * Q + q1) * Q + q0];
      t1[i] = s;
    }
    __syncthreads();
    for (int i = lt; i < NC * NL; i += NQ) {         // q0 -> j0
      const int j0 = i % L, r = i / L;
      T s = 0;
#pragma unroll
      for (int q0 = 0; q0 < Q; ++q0) s += Bl[q0 * L + j0] * t1[r * Q + q0];
      out[i] = s;
    }
    __syncthreads();
  } else {
    constexpr int NQ = Q * Q, S1 = NC * L * Q, NL = L * L;
#pragma unroll
    for (int c = 0; c < NC; ++c) sf[c * NQ + lt] = fval[c];
    __syncthreads();
    for (int i = lt; i < S1; i += NQ) {
      const int q0 = i % Q, j1 = (i / Q) % L, c = i / (Q * L);
      T s = 0;
#pragma unroll
      for (int q1 = 0; q1 < Q; ++q1) s += Bl[q1 * L + j1] * sf[c * NQ + q1 * Q + q0];
      t1[i] = s;
    }
    __syncthreads();
    for (int i = lt; i < NC * NL; i += NQ) {
      const int j0 = i % L, r = i / L;
      T s = 0;
#pragma unroll
      for (int q0 = 0; q0 < Q; ++q0) s += Bl[q0 * L + j0] * t1[r * Q + q0];
      out[i] = s;
    }
    __syncthreads();
  }
}

}  // namespace op

// ---------------------------------------------------------------------------------------
// Public entry points: FP32 runs the line form (ln, above), whose stages are bound by
// shared-memory instructions; double and double-float run the output-parallel form (op),
// whose stages are bound by arithmetic and keep every lane of a warp busy.
template <class T>
constexpr bool kLines = std::is_same<T, float>::value;

template <int DIM, int K, int NC, class T, bool VAL = true>
__device__ __forceinline__ void h1_fwd(const T* __restrict__ in, T* t1, T* t2, const T* B, const T* G,
                                       int lt, T (&val)[NC], T (&grad)[NC][DIM]) {
  if constexpr (kLines<T>) ln::h1_fwd<DIM, K, NC, T, VAL>(in, t1, t2, B, G, lt, val, grad);
  else op::h1_fwd<DIM, K, NC, T, VAL>(in, t1, t2, B, G, lt, val, grad);
}
template <int DIM, int K, int NC, class T>
__device__ __forceinline__ void h1_bwd(const T (&fval)[NC], const T (&fgrad)[NC][DIM], T* sf, T* t1, T* t2,
                                       const T* B, const T* G, int lt, T* out) {
  if constexpr (kLines<T>) ln::h1_bwd<DIM, K, NC, T>(fval, fgrad, sf, t1, t2, B, G, lt, out);
  else op::h1_bwd<DIM, K, NC, T>(fval, fgrad, sf, t1, t2, B, G, lt, out);
}
template <int DIM, int K, int NC, class T, int L_ = K>
__device__ __forceinline__ void l2_fwd(const T* __restrict__ in, T* t1, T* t2, const T* Bl, int lt, T (&val)[NC]) {
  if constexpr (kLines<T>) ln::l2_fwd<DIM, K, NC, T, L_>(in, t1, t2, Bl, lt, val);
  else op::l2_fwd<DIM, K, NC, T, L_>(in, t1, t2, Bl, lt, val);
}
template <int DIM, int K, int NC, class T, int L_ = K>
__device__ __forceinline__ void l2_bwd(const T (&fval)[NC], T* sf, T* t1, T* t2, const T* Bl, int lt, T* out) {
  if constexpr (kLines<T>) ln::l2_bwd<DIM, K, NC, T, L_>(fval, sf, t1, t2, Bl, lt, out);
  else op::l2_bwd<DIM, K, NC, T, L_>(fval, sf, t1, t2, Bl, lt, out);
}

}  // namespace lh
