// Sum-factorised basis contractions (the B and B^T operators of paper Sec. 2.2, Eq. (8)).
//
// Tensor-product elements let B act one direction at a time (Sec. 2.2: O(p^{d+1}) work
// per element instead of O(p^{2d})).  One thread per quadrature point; the threads of an
// element stride over the intermediate index sets; intermediates live in shared memory.
// Every function ends with __syncthreads() so the caller may reuse the scratch at once.
//
// Tables (row-major, in shared memory): B[q*D + a] = w_a(z_q), G[q*D + a] = w_a'(z_q)
// for the H1 basis, Bl[q*L + j] = phi_j(z_q) for the L2 basis.
// Element-local layouts: H1 values [c][a2][a1][a0] (a = a0 + D a1 + D^2 a2), L2 values
// [c][j2][j1][j0], quadrature values [q2][q1][q0].
#pragma once
#include "lh_common.cuh"

namespace lh {

// 1D table layout in the device table buffer (built by the host at mesh creation):
// [B | G | Bl | w | H1 nodes | L2 nodes]
template <int K>
struct Tab {
  static constexpr int D = K + 1, L = K, Q = 2 * K;
  static constexpr int B = 0, G = Q * D, BL = 2 * Q * D, W = 2 * Q * D + Q * L;
  static constexpr int SMEM = 2 * Q * D + Q * L + Q;           // entries staged in shared memory
};

template <int DIM, int K, int NC>
struct H1Scratch {
  static constexpr int D = K + 1, Q = 2 * K;
  static constexpr int T1 = DIM == 3 ? 2 * NC * D * D * Q : 2 * NC * D * Q;
  static constexpr int T2 = DIM == 3 ? 3 * NC * D * Q * Q : 1;
  static constexpr int SF = (DIM + 1) * NC * (DIM == 3 ? Q * Q * Q : Q * Q);
};

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

}  // namespace lh
