// Vector kernels of the Newton-GMRES driver (paper Sec. 3.5, Eq. (22)): deterministic
// dot products, Gram-Schmidt updates, the block-diagonal preconditioner and precision
// conversions.  All are HBM-bound streaming kernels over the n unknowns.
#include <cfloat>
#include <cstdint>
#include "lh_kernels.h"

namespace lh {

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// s += sum_{j < m} hs[j] v[j * ld4] in the order j = 0, 1, ... (four columns' loads issued
// together)
__device__ __forceinline__ void cols4(float4& s, const float* hs, const float4* v, long long ld4, int m) {
  int j = 0;
  for (; j + 4 <= m; j += 4, v += 4 * ld4) {
    const float4 x0 = v[0], x1 = v[ld4], x2 = v[2 * ld4], x3 = v[3 * ld4];
    const float4 x[4] = {x0, x1, x2, x3};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float c = hs[j + u];
      s.x += c * x[u].x;
      s.y += c * x[u].y;
      s.z += c * x[u].z;
      s.w += c * x[u].w;
    }
  }
  for (; j < m; ++j, v += ld4) {
    const float4 x = *v;
    const float c = hs[j];
    s.x += c * x.x;
    s.y += c * x.y;
    s.z += c * x.z;
    s.w += c * x.w;
  }
}

// Fused deterministic multi-dot: out[j] = V_j . w for j < m, plus out[m] = w . w when
// with_self.  Each block reduces a fixed contiguous chunk of the index range (one pass
// over w for up to 8 vectors at a time, fixed-order warp and block trees) and writes its
// partials; the last block to finish (ticket from an atomic counter) adds the partials of
// every output in block order.  The result depends only on n and the data, not on the
// order in which blocks finish.
// outputs per pass over the chunk: 16 in float, 8 in double (register budget)
template <class T> struct MdotChunk { static constexpr int value = sizeof(T) == sizeof(float) ? 16 : 8; };
constexpr int kChunkMax = 16;

static inline unsigned red_grid(long long n) {
  long long g = (n + 1023) / 1024;
  if (g < 1) g = 1;
  if (g > kRedBlocks) g = kRedBlocks;
  return (unsigned)g;
}

// SUB (float4 form only): the first Gram-Schmidt update fused in front of the multi-dot:
// w' = w - V hsub (the same sums, in the same order, as k_gemv4<true>) is written to wout and
// the outputs are V^T w' (and w'.w').
template <class T, bool VEC4, bool SUB = false>
__global__ void __launch_bounds__(kRedThreads)
k_mdot(const T* __restrict__ V, int m, long long ld, const T* __restrict__ w, long long n, int with_self,
       double* __restrict__ part, unsigned* __restrict__ counter, double* __restrict__ out,
       const int* __restrict__ jdev, const int* __restrict__ gate, const double* __restrict__ hsub = nullptr,
       float* __restrict__ wout = nullptr) {
  // per-thread and warp sums in T (float: a few hundred terms, ~1e-7 relative), block and
  // grid sums in double.  jdev: column count from the device (m = *jdev + 1, at most
  // kArnMax); gate: the launch does nothing unless *gate != 0 (both only inside the
  // device-driven Arnoldi).
  if (gate && *gate == 0) return;
  if (jdev) m = min(*jdev + 1, kArnMax);
  constexpr int kChunk = MdotChunk<T>::value;
  __shared__ double red[kRedThreads / 32][kChunkMax];
  __shared__ bool last;
  __shared__ float hsn[SUB ? 64 : 1];
  static_assert(!SUB || (VEC4 && sizeof(T) == sizeof(float)), "the fused update is float4 only");
  if constexpr (SUB) {
    if ((int)threadIdx.x < m) hsn[threadIdx.x] = -(float)hsub[threadIdx.x];
    __syncthreads();
  }
  const int nout = m + (with_self ? 1 : 0);
  long long chunk = (n + gridDim.x - 1) / gridDim.x;
  if constexpr (VEC4) chunk = (chunk + 3) / 4 * 4;   // chunk boundaries on 16-byte boundaries
  const long long beg = (long long)blockIdx.x * chunk;
  const long long end = beg + chunk < n ? beg + chunk : n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nout; c0 += kChunk) {
    T acc[kChunk];
    const T* vq[kChunk];   // per-vector pointers (no 64-bit index products in the loop)
#pragma unroll
    for (int q = 0; q < kChunk; ++q) {
      acc[q] = T(0);
      vq[q] = c0 + q < m ? V + (long long)(c0 + q) * ld : w;
    }
    const int nq = nout - c0 < kChunk ? nout - c0 : kChunk;
    if constexpr (VEC4) {
      // four consecutive entries per load (ld, n multiples of 4, 16-byte aligned vectors)
      for (long long i = beg + 4 * threadIdx.x; i < end; i += 4 * blockDim.x) {
        float4 wi;
        if constexpr (SUB) {
          if (c0 == 0) {   // w' at this position, kept for the later chunks of outputs
            wi = *reinterpret_cast<const float4*>(w + i);
            cols4(wi, hsn, reinterpret_cast<const float4*>(V + i), ld / 4, m);
            *reinterpret_cast<float4*>(wout + i) = wi;
          } else {
            wi = *reinterpret_cast<const float4*>(wout + i);
          }
        } else {
          wi = w ? *reinterpret_cast<const float4*>(w + i) : make_float4(1.f, 1.f, 1.f, 1.f);
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
          if (q < nq) {
            const float4 v = c0 + q == m ? wi : *reinterpret_cast<const float4*>(vq[q] + i);
            acc[q] += (v.x * wi.x + v.y * wi.y) + (v.z * wi.z + v.w * wi.w);
          }
      }
    } else if (w) {
      for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const T wi = w[i];
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
          if (q < nq) acc[q] += vq[q][i] * wi;
      }
    } else {
      for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) {
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
          if (q < nq) acc[q] += vq[q][i];
      }
    }
    // warp reduce-scatter (fixed butterfly): at each step the lanes with bit o set keep the
    // upper half of their outputs and receive the partner's upper half; after log2(kChunk)
    // halvings every lane holds one output, the remaining steps add the lane pairs.
    // kChunk - 1 + 5 - log2(kChunk) shuffles instead of 5 kChunk.
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int o = 16 >> st;
      const int cnt = kChunk >> st;   // outputs held per lane before this step
      if (cnt >= 2) {
        const int half = cnt / 2;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < kChunk / 2; ++q)
          if (q < half) {
            const T send = up ? acc[q] : acc[q + half];
            const T keep = up ? acc[q + half] : acc[q];
            acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
      } else {
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
      }
    }
    {
      constexpr int shift = kChunk == 16 ? 1 : kChunk == 8 ? 2 : 0;
      static_assert(kChunk == 16 || kChunk == 8, "butterfly layout");
      if ((lane & ((1 << shift) - 1)) == 0) red[warp][lane >> shift] = (double)acc[0];
    }
    __syncthreads();
    if (threadIdx.x < kChunk && c0 + (int)threadIdx.x < nout) {
      double v = 0.0;
      for (int q = 0; q < kRedThreads / 32; ++q) v += red[q][threadIdx.x];
      part[(long long)(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
    }
    __syncthreads();
  }
  __threadfence();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // last block: out[j] = sum over blocks of the partials; kRedThreads / kChunk consecutive
  // threads per output, each summing a fixed strided subset, then a fixed shuffle tree
  constexpr int kPer = kRedThreads / kChunk;
  for (int c0 = 0; c0 < nout; c0 += kChunk) {
    const int q = threadIdx.x / kPer, sub = threadIdx.x % kPer;
    double v = 0.0;
    if (c0 + q < nout)
      for (unsigned b = sub; b < gridDim.x; b += kPer) v += __ldcg(part + (long long)(c0 + q) * gridDim.x + b);
    for (int o = kPer / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, kPer);
    if (sub == 0 && c0 + q < nout) out[c0 + q] = v;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

template <class T>
cudaError_t launch_mdot(cudaStream_t s, const T* V, int m, long long ld, const T* w, long long n, int with_self,
                        double* partials, unsigned* counter, double* out_dev) {
  if (m + (with_self ? 1 : 0) > 72) return cudaErrorInvalidValue;
  const bool vec4 = sizeof(T) == sizeof(float) && n % 4 == 0 && ld % 4 == 0 &&
                    reinterpret_cast<uintptr_t>(V) % 16 == 0 && reinterpret_cast<uintptr_t>(w) % 16 == 0;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (vec4) {
      k_mdot<T, true><<<red_grid(n), kRedThreads, 0, s>>>(V, m, ld, w, n, with_self, partials, counter, out_dev,
                                                           nullptr, nullptr);
      count_launches(1);
      return cudaGetLastError();
    }
  }
  k_mdot<T, false><<<red_grid(n), kRedThreads, 0, s>>>(V, m, ld, w, n, with_self, partials, counter, out_dev,
                                                        nullptr, nullptr);
  count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_mdot<double>(cudaStream_t, const double*, int, long long, const double*, long long, int,
                                         double*, unsigned*, double*);
template cudaError_t launch_mdot<float>(cudaStream_t, const float*, int, long long, const float*, long long, int,
                                        double*, unsigned*, double*);

__global__ void __launch_bounds__(kRedThreads) k_min(const double* __restrict__ v, long long n, double* out) {
  __shared__ double red[kRedThreads];
  double m = DBL_MAX;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, v[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

cudaError_t launch_min(cudaStream_t s, const double* v, long long n, double* out_dev) {
  k_min<<<1, kRedThreads, 0, s>>>(v, n, out_dev);
  count_launches(1);
  return cudaGetLastError();
}

template <class T>
__global__ void k_gemv_sub(const T* __restrict__ V, int m, long long ld, const double* __restrict__ h,
                           T* __restrict__ w, long long n) {
  __shared__ T hs[64];
  if ((int)threadIdx.x < m) hs[threadIdx.x] = T(h[threadIdx.x]);
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T s = w[i];
    const T* v = V + i;
    for (int j = 0; j < m; ++j, v += ld) s -= hs[j] * *v;
    w[i] = s;
  }
}

// float4 forms (n, ld multiples of 4, 16-byte aligned): y = beta y + sign * V h
template <bool SUB>
__global__ void k_gemv4(const float* __restrict__ V, int m, long long ld, const double* __restrict__ h, float beta,
                        float* __restrict__ y, long long n4, const int* __restrict__ jdev = nullptr,
                        const int* __restrict__ gate = nullptr) {
  __shared__ float hs[64];
  if (gate && *gate == 0) return;
  if (jdev) m = min(*jdev + 1, kArnMax);
  if ((int)threadIdx.x < m) hs[threadIdx.x] = SUB ? -(float)h[threadIdx.x] : (float)h[threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (SUB || beta != 0.f) {
      s = reinterpret_cast<const float4*>(y)[i];
      if (!SUB) s = make_float4(beta * s.x, beta * s.y, beta * s.z, beta * s.w);
    }
    const float4* v = reinterpret_cast<const float4*>(V) + i;
    const long long ld4 = ld / 4;
    for (int j = 0; j < m; ++j, v += ld4) {
      const float4 x = *v;
      const float c = hs[j];
      s.x += c * x.x;
      s.y += c * x.y;
      s.z += c * x.z;
      s.w += c * x.w;
    }
    reinterpret_cast<float4*>(y)[i] = s;
  }
}

// second Gram-Schmidt pass fused with the normalisation: y = (w - V h) / hn with
// hn^2 = h[m] - sum_q h[q]^2 (h[m] = w.w from the same multi-dot); y = 0 if hn^2 <= 0
__global__ void k_gemv4_norm(const float* __restrict__ V, int m, long long ld, const double* __restrict__ h,
                             const float* __restrict__ w, float* __restrict__ y, long long n4) {
  __shared__ float hs[64];
  __shared__ float s_inv;
  if (threadIdx.x == 0) {
    double hh = 0.0;
    for (int q = 0; q < m; ++q) hh += h[q] * h[q];
    const double hn2 = h[m] - hh;
    s_inv = hn2 > 0.0 ? (float)(1.0 / sqrt(hn2)) : 0.f;
  }
  if ((int)threadIdx.x < m) hs[threadIdx.x] = -(float)h[threadIdx.x];
  __syncthreads();
  const float inv = s_inv;
  const long long ld4 = ld / 4;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    float4 s = reinterpret_cast<const float4*>(w)[i];
    const float4* v = reinterpret_cast<const float4*>(V) + i;
    for (int j = 0; j < m; ++j, v += ld4) {
      const float4 x = *v;
      const float c = hs[j];
      s.x += c * x.x;
      s.y += c * x.y;
      s.z += c * x.z;
      s.w += c * x.w;
    }
    reinterpret_cast<float4*>(y)[i] = make_float4(s.x * inv, s.y * inv, s.z * inv, s.w * inv);
  }
}

template <class T>
__global__ void k_gemv_norm(const T* __restrict__ V, int m, long long ld, const double* __restrict__ h,
                            const T* __restrict__ w, T* __restrict__ y, long long n) {
  __shared__ T hs[64];
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    double hh = 0.0;
    for (int q = 0; q < m; ++q) hh += h[q] * h[q];
    const double hn2 = h[m] - hh;
    s_inv = hn2 > 0.0 ? 1.0 / sqrt(hn2) : 0.0;
  }
  if ((int)threadIdx.x < m) hs[threadIdx.x] = T(h[threadIdx.x]);
  __syncthreads();
  const T inv = T(s_inv);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T s = w[i];
    const T* v = V + i;
    for (int j = 0; j < m; ++j, v += ld) s -= hs[j] * *v;
    y[i] = s * inv;
  }
}

static bool vec4_ok(const void* a, const void* b, long long ld, long long n) {
  return n % 4 == 0 && ld % 4 == 0 && reinterpret_cast<uintptr_t>(a) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(b) % 16 == 0;
}

template <class T>
cudaError_t launch_gemv_sub(cudaStream_t s, const T* V, int m, long long ld, const double* h, T* w, long long n) {
  if (m > 64) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (vec4_ok(V, w, ld, n)) {
      const long long n4 = n / 4;
      k_gemv4<true><<<nblk(n4, 256) < 4736u ? nblk(n4, 256) : 4736u, 256, 0, s>>>(V, m, ld, h, 1.f, w, n4);
      count_launches(1);
      return cudaGetLastError();
    }
  }
  k_gemv_sub<T><<<nblk(n, 256) < 4736u ? nblk(n, 256) : 4736u, 256, 0, s>>>(V, m, ld, h, w, n);
  count_launches(1);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_gemv_norm(cudaStream_t s, const T* V, int m, long long ld, const double* h, const T* w, T* y,
                             long long n) {
  if (m > 64) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (vec4_ok(V, w, ld, n) && reinterpret_cast<uintptr_t>(y) % 16 == 0) {
      const long long n4 = n / 4;
      k_gemv4_norm<<<nblk(n4, 256) < 4736u ? nblk(n4, 256) : 4736u, 256, 0, s>>>(V, m, ld, h, w, y, n4);
      count_launches(1);
      return cudaGetLastError();
    }
  }
  k_gemv_norm<T><<<nblk(n, 256) < 4736u ? nblk(n, 256) : 4736u, 256, 0, s>>>(V, m, ld, h, w, y, n);
  count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_gemv_norm<double>(cudaStream_t, const double*, int, long long, const double*,
                                              const double*, double*, long long);
template cudaError_t launch_gemv_norm<float>(cudaStream_t, const float*, int, long long, const double*,
                                             const float*, float*, long long);

template cudaError_t launch_gemv_sub<double>(cudaStream_t, const double*, int, long long, const double*, double*,
                                             long long);
template cudaError_t launch_gemv_sub<float>(cudaStream_t, const float*, int, long long, const double*, float*,
                                            long long);

// ---- device-side Arnoldi (FP32 basis) ----
static inline unsigned gemv_grid(long long n4) { return nblk(n4, 256) < 4736u ? nblk(n4, 256) : 4736u; }

cudaError_t launch_mdot_dev(cudaStream_t s, const float* V, const int* jdev, long long ld, const float* w, long long n,
                            int with_self, const int* gate, double* partials, unsigned* counter, double* out_dev) {
  if (!vec4_ok(V, w, ld, n)) return cudaErrorInvalidValue;
  k_mdot<float, true><<<red_grid(n), kRedThreads, 0, s>>>(V, 1, ld, w, n, with_self, partials, counter, out_dev, jdev,
                                                          gate);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mdot_sub(cudaStream_t s, const float* V, int m, const int* jdev, long long ld, const float* w,
                            const double* hsub, float* wout, long long n, double* partials, unsigned* counter,
                            double* out_dev) {
  if (!vec4_ok(V, w, ld, n) || reinterpret_cast<uintptr_t>(wout) % 16 != 0 || m + 1 > 72) return cudaErrorInvalidValue;
  k_mdot<float, true, true><<<red_grid(n), kRedThreads, 0, s>>>(V, m, ld, w, n, 1, partials, counter, out_dev, jdev,
                                                                nullptr, hsub, wout);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gemv_sub_dev(cudaStream_t s, const float* V, const int* jdev, long long ld, const double* h,
                                float* w, long long n, const int* gate) {
  if (!vec4_ok(V, w, ld, n)) return cudaErrorInvalidValue;
  const long long n4 = n / 4;
  k_gemv4<true><<<gemv_grid(n4), 256, 0, s>>>(V, 1, ld, h, 1.f, w, n4, jdev, gate);
  count_launches(1);
  return cudaGetLastError();
}

// as k_gemv4_norm with m = st->j + 1 coefficients; writes column m of V and vin.  Block 0
// also stores hn^2 (Pythagoras) and whether the second pass still cancelled (hn^2 <= 1e-4
// w.w, then the exact norm is taken) in the cycle state and as the IF condition `fix`.
__global__ void k_gemv4_norm_dev(float* V, ArnState* st, long long ld, const double* __restrict__ h,
                                 const float* __restrict__ w, float* __restrict__ vin, long long n4,
                                 cudaGraphConditionalHandle fix) {
  __shared__ float hs[64];
  __shared__ float s_inv;
  const int m = min(st->j + 1, kArnMax);
  if (threadIdx.x == 0) {
    double hh = 0.0;
    for (int q = 0; q < m; ++q) hh += h[q] * h[q];
    const double ww = h[m];
    const double hn2 = ww - hh;
    s_inv = hn2 > 0.0 ? (float)(1.0 / sqrt(hn2)) : 0.f;
    if (blockIdx.x == 0) {
      const int f = hn2 > 1e-4 * ww ? 0 : 1;
      st->hn2 = hn2;
      st->fix = f;
      cudaGraphSetConditional(fix, (unsigned)f);
    }
  }
  if ((int)threadIdx.x < m) hs[threadIdx.x] = -(float)h[threadIdx.x];
  __syncthreads();
  const float inv = s_inv;
  const long long ld4 = ld / 4;
  float4* y = reinterpret_cast<float4*>(V + (long long)m * ld);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    float4 t = reinterpret_cast<const float4*>(w)[i];
    const float4* v = reinterpret_cast<const float4*>(V) + i;
    for (int j = 0; j < m; ++j, v += ld4) {
      const float4 x = *v;
      const float c = hs[j];
      t.x += c * x.x;
      t.y += c * x.y;
      t.z += c * x.z;
      t.w += c * x.w;
    }
    const float4 o = make_float4(t.x * inv, t.y * inv, t.z * inv, t.w * inv);
    y[i] = o;
    reinterpret_cast<float4*>(vin)[i] = o;
  }
}

cudaError_t launch_gemv_norm_dev(cudaStream_t s, float* V, ArnState* st, long long ld, const double* h,
                                 const float* w, float* vin, long long n, cudaGraphConditionalHandle fix) {
  if (!vec4_ok(V, w, ld, n) || reinterpret_cast<uintptr_t>(vin) % 16 != 0) return cudaErrorInvalidValue;
  const long long n4 = n / 4;
  k_gemv4_norm_dev<<<gemv_grid(n4), 256, 0, s>>>(V, st, ld, h, w, vin, n4, fix);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_arn_scale(const ArnState* __restrict__ st, const float* __restrict__ w, float* V, long long ld,
                            float* __restrict__ vin, long long n4) {
  if (st->fix == 0) return;
  const double hn2 = st->hn2;
  if (!(hn2 > 0.0)) return;
  const float a = (float)(1.0 / sqrt(hn2));
  const int m = min(st->j + 1, kArnMax);
  float4* y = reinterpret_cast<float4*>(V + (long long)m * ld);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const float4 x = reinterpret_cast<const float4*>(w)[i];
    const float4 o = make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
    y[i] = o;
    reinterpret_cast<float4*>(vin)[i] = o;
  }
}

cudaError_t launch_arn_scale(cudaStream_t s, const ArnState* st, const float* w, float* V, long long ld, float* vin,
                             long long n) {
  if (!vec4_ok(V, w, ld, n) || reinterpret_cast<uintptr_t>(vin) % 16 != 0) return cudaErrorInvalidValue;
  const long long n4 = n / 4;
  k_arn_scale<<<gemv_grid(n4), 256, 0, s>>>(st, w, V, ld, vin, n4);
  count_launches(1);
  return cudaGetLastError();
}

// One Arnoldi column's bookkeeping, in the order of the host loop: H[i][j] = h1[i] + h2[i]
// (both Gram-Schmidt passes), H[j+1][j] = hn, the previous Givens rotations, the new
// rotation, g, and the stopping test.  The WHILE condition is 1 only while the cycle runs.
__global__ void k_arn_givens(const double* __restrict__ h1, const double* __restrict__ h2, ArnState* st,
                             cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = st->j;
  int stop = 0;
  if (j < 0 || j >= st->mres || j >= kArnMax) {
    stop = 3;   // cannot happen while the host sets mres <= kArnMax; ends the loop regardless
  } else {
    const double hn2 = st->hn2;
    if (!isfinite(hn2)) {
      stop = 5;
    } else {
      double c[kArnMax + 1];
      for (int i = 0; i <= j; ++i) c[i] = h1[i] + h2[i];
      const double hn = sqrt(fmax(hn2, 0.0));
      c[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double a = c[i], b = c[i + 1];
        c[i] = st->cs[i] * a + st->sn[i] * b;
        c[i + 1] = -st->sn[i] * a + st->cs[i] * b;
      }
      const double a = c[j], b = c[j + 1];
      const double rad = hypot(a, b);
      st->cs[j] = rad > 0 ? a / rad : 1.0;
      st->sn[j] = rad > 0 ? b / rad : 0.0;
      c[j] = rad;
      c[j + 1] = 0.0;
      for (int i = 0; i <= j + 1; ++i) st->H[i * kArnMax + j] = c[i];
      const double gj = st->g[j];
      st->g[j + 1] = -st->sn[j] * gj;
      st->g[j] = st->cs[j] * gj;
      st->j = j + 1;
      if (fabs(st->g[j + 1]) <= st->tol || hn == 0.0) stop = 1;
      else if (j + 1 >= st->mres) stop = 3;
      else if (j + 1 >= st->maxit) stop = 4;
    }
  }
  st->stop = stop;
  cudaGraphSetConditional(cond, stop == 0 ? 1u : 0u);
}

cudaError_t launch_arn_givens(cudaStream_t s, const double* h1, const double* h2, ArnState* st,
                              cudaGraphConditionalHandle cond) {
  k_arn_givens<<<1, 32, 0, s>>>(h1, h2, st, cond);
  count_launches(1);
  return cudaGetLastError();
}

template <class T>
__global__ void k_gemv(const T* __restrict__ V, int m, long long ld, const double* __restrict__ h, double beta,
                       T* __restrict__ y, long long n) {
  __shared__ T hs[64];
  if ((int)threadIdx.x < m) hs[threadIdx.x] = T(h[threadIdx.x]);
  __syncthreads();
  const T bt = T(beta);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T s = beta == 0.0 ? T(0) : bt * y[i];
    const T* v = V + i;
    for (int j = 0; j < m; ++j, v += ld) s += hs[j] * *v;
    y[i] = s;
  }
}

template <class T>
cudaError_t launch_gemv(cudaStream_t s, const T* V, int m, long long ld, const double* h, double beta, T* y,
                        long long n) {
  if (m > 64) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (vec4_ok(V, y, ld, n)) {
      const long long n4 = n / 4;
      k_gemv4<false><<<nblk(n4, 256) < 4736u ? nblk(n4, 256) : 4736u, 256, 0, s>>>(V, m, ld, h, (float)beta, y, n4);
      count_launches(1);
      return cudaGetLastError();
    }
  }
  k_gemv<T><<<nblk(n, 256) < 4736u ? nblk(n, 256) : 4736u, 256, 0, s>>>(V, m, ld, h, beta, y, n);
  count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_gemv<double>(cudaStream_t, const double*, int, long long, const double*, double, double*,
                                         long long);
template cudaError_t launch_gemv<float>(cudaStream_t, const float*, int, long long, const double*, double, float*,
                                        long long);

// y = a x (+ b z), with x of type TX, z float (may be NULL), y of type TY
template <class TX, class TY>
__global__ void k_scale(double a, const TX* __restrict__ x, double b, const float* __restrict__ z, TY* __restrict__ y,
                        long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if constexpr (sizeof(TY) == sizeof(float) && sizeof(TX) == sizeof(float)) {
    float v = (float)a * x[i];
    if (z) v += (float)b * z[i];
    y[i] = v;
  } else {
    double v = a * (double)x[i];
    if (z) v += b * (double)z[i];
    y[i] = TY(v);
  }
}

template <class TX, class TY>
cudaError_t launch_scale(cudaStream_t s, double a, const TX* x, double b, const float* z, TY* y, long long n) {
  if (n > 0) {
    k_scale<TX, TY><<<nblk(n, 256), 256, 0, s>>>(a, x, b, z, y, n);
    count_launches(1);
  }
  return cudaGetLastError();
}
template cudaError_t launch_scale<double, float>(cudaStream_t, double, const double*, double, const float*, float*,
                                                 long long);
template cudaError_t launch_scale<float, float>(cudaStream_t, double, const float*, double, const float*, float*,
                                                long long);
template cudaError_t launch_scale<double, double>(cudaStream_t, double, const double*, double, const float*,
                                                  double*, long long);

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

cudaError_t launch_axpby(cudaStream_t s, double a, const double* x, double b, double* y, long long n) {
  if (n > 0) {
    k_axpby<<<nblk(n, 256), 256, 0, s>>>(a, x, b, y, n);
    count_launches(1);
  }
  return cudaGetLastError();
}

// y = x * (1 / scale_dev[0])
// y = w * x elementwise (x may alias y)
template <class T>
__global__ void k_row_mul(const double* __restrict__ w, const T* x, T* y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = T((double)x[i] * w[i]);
}

template <class T>
cudaError_t launch_row_mul(cudaStream_t s, const double* w, const T* x, T* y, long long n) {
  if (n > 0) {
    k_row_mul<T><<<nblk(n, 256), 256, 0, s>>>(w, x, y, n);
    count_launches(1);
  }
  return cudaGetLastError();
}
template cudaError_t launch_row_mul<double>(cudaStream_t, const double*, const double*, double*, long long);
template cudaError_t launch_row_mul<float>(cudaStream_t, const double*, const float*, float*, long long);

__global__ void k_scale_copy(const double* __restrict__ x, const double* __restrict__ sc, double* __restrict__ y,
                             long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] / sc[0];
}

cudaError_t launch_scale_copy(cudaStream_t s, const double* x, const double* scale_dev, double* y, long long n) {
  if (n > 0) {
    k_scale_copy<<<nblk(n, 256), 256, 0, s>>>(x, scale_dev, y, n);
    count_launches(1);
  }
  return cudaGetLastError();
}

__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
__global__ void k_to_f64(const float* __restrict__ x, double* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i];
}
cudaError_t launch_to_f32(cudaStream_t s, const double* x, float* y, long long n) {
  if (n > 0) {
    k_to_f32<<<nblk(n, 256), 256, 0, s>>>(x, y, n);
    count_launches(1);
  }
  return cudaGetLastError();
}
cudaError_t launch_to_f64(cudaStream_t s, const float* x, double* y, long long n) {
  if (n > 0) {
    k_to_f64<<<nblk(n, 256), 256, 0, s>>>(x, y, n);
    count_launches(1);
  }
  return cudaGetLastError();
}

__global__ void k_jacobi_h1(long long nv, int dim, const double* __restrict__ diag, const double* __restrict__ r,
                            double* __restrict__ z) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nv * dim) z[i] = r[i] / diag[i % nv];
}

cudaError_t launch_jacobi_h1(cudaStream_t s, long long nv, int dim, const double* diag, const double* r, double* z) {
  k_jacobi_h1<<<nblk(nv * dim, 256), 256, 0, s>>>(nv, dim, diag, r, z);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_mul(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] * b[i];
}

cudaError_t launch_mul(cudaStream_t s, const double* a, const double* b, double* y, long long n) {
  if (n > 0) {
    k_mul<<<nblk(n, 256), 256, 0, s>>>(a, b, y, n);
    count_launches(1);
  }
  return cudaGetLastError();
}

// ---- FMA throughput probe (roofline denominator of the FP64 / FP32 pipes)
template <class T, int CH>
__global__ void k_fma_probe(T* out, int iters, T a, T b) {
  T acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = T(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = acc[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
static cudaError_t probe(int iters, double* tflops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_probe<T, 8><<<blocks, threads>>>(out, 16, T(0.999), T(0.001));
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_fma_probe<T, 8><<<blocks, threads>>>(out, iters, T(0.999), T(0.001));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return e;
}

cudaError_t launch_probe_fma(int prec, double* tflops) {
  return prec == 0 ? probe<double>(4000, tflops) : probe<float>(40000, tflops);
}

}  // namespace lh
