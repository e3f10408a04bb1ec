// Vector kernels of the Newton-GMRES driver (paper Sec. 3.5, Eq. (22)): deterministic
// dot products, Gram-Schmidt updates, the block-diagonal preconditioner and precision
// conversions.  All are HBM-bound streaming kernels over the n unknowns.
#include <cfloat>
#include "lh_kernels.h"

namespace lh {

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Fused deterministic multi-dot: out[j] = V_j . w for j < m, plus out[m] = w . w when
// with_self.  Each block reduces a fixed contiguous chunk of the index range (one pass
// over w for up to 8 vectors at a time, fixed-order warp and block trees) and writes its
// partials; the last block to finish (ticket from an atomic counter) adds the partials of
// every output in block order.  The result depends only on n and the data, not on the
// order in which blocks finish.
constexpr int kChunk = 8;

static inline unsigned red_grid(long long n) {
  long long g = (n + 1023) / 1024;
  if (g < 1) g = 1;
  if (g > kRedBlocks) g = kRedBlocks;
  return (unsigned)g;
}

__global__ void __launch_bounds__(kRedThreads)
k_mdot(const double* __restrict__ V, int m, long long ld, const double* __restrict__ w, long long n, int with_self,
       double* __restrict__ part, unsigned* __restrict__ counter, double* __restrict__ out) {
  __shared__ double red[kRedThreads / 32][kChunk];
  __shared__ bool last;
  const int nout = m + (with_self ? 1 : 0);
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long beg = (long long)blockIdx.x * chunk;
  const long long end = beg + chunk < n ? beg + chunk : n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nout; c0 += kChunk) {
    double acc[kChunk];
#pragma unroll
    for (int q = 0; q < kChunk; ++q) acc[q] = 0.0;
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) {
      const double wi = w ? w[i] : 1.0;
#pragma unroll
      for (int q = 0; q < kChunk; ++q) {
        const int j = c0 + q;
        if (j < m) acc[q] += V[j * ld + i] * wi;
        else if (j < nout) acc[q] += wi * wi;
      }
    }
#pragma unroll
    for (int q = 0; q < kChunk; ++q) {
      double v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][q] = v;
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
  // last block: out[j] = sum over blocks of the partials, the whole block reducing up to
  // kChunk outputs at a time (coalesced L2 loads, fixed-order trees)
  for (int c0 = 0; c0 < nout; c0 += kChunk) {
    double acc[kChunk];
#pragma unroll
    for (int q = 0; q < kChunk; ++q) {
      acc[q] = 0.0;
      if (c0 + q < nout)
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
          acc[q] += __ldcg(part + (long long)(c0 + q) * gridDim.x + b);
    }
#pragma unroll
    for (int q = 0; q < kChunk; ++q) {
      double v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kChunk && c0 + (int)threadIdx.x < nout) {
      double v = 0.0;
      for (int q = 0; q < kRedThreads / 32; ++q) v += red[q][threadIdx.x];
      out[c0 + threadIdx.x] = v;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *counter = 0u;
}

cudaError_t launch_mdot(cudaStream_t s, const double* V, int m, long long ld, const double* w, long long n,
                        int with_self, double* partials, unsigned* counter, double* out_dev) {
  if (m + (with_self ? 1 : 0) > 72) return cudaErrorInvalidValue;
  k_mdot<<<red_grid(n), kRedThreads, 0, s>>>(V, m, ld, w, n, with_self, partials, counter, out_dev);
  count_launches(1);
  return cudaGetLastError();
}

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

__global__ void k_gemv_sub(const double* __restrict__ V, int m, long long ld, const double* __restrict__ h,
                           double* __restrict__ w, long long n) {
  __shared__ double hs[64];
  if ((int)threadIdx.x < m) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int j = 0; j < m; ++j) s -= hs[j] * V[j * ld + i];
    w[i] = s;
  }
}

cudaError_t launch_gemv_sub(cudaStream_t s, const double* V, int m, long long ld, const double* h, double* w,
                            long long n) {
  if (m > 64) return cudaErrorInvalidValue;
  k_gemv_sub<<<nblk(n, 256) < 4736u ? nblk(n, 256) : 4736u, 256, 0, s>>>(V, m, ld, h, w, n);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_gemv(const double* __restrict__ V, int m, long long ld, const double* __restrict__ h, double beta,
                       double* __restrict__ y, long long n) {
  __shared__ double hs[64];
  if ((int)threadIdx.x < m) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = beta == 0.0 ? 0.0 : beta * y[i];
    for (int j = 0; j < m; ++j) s += hs[j] * V[j * ld + i];
    y[i] = s;
  }
}

cudaError_t launch_gemv(cudaStream_t s, const double* V, int m, long long ld, const double* h, double beta,
                        double* y, long long n) {
  if (m > 64) return cudaErrorInvalidValue;
  k_gemv<<<nblk(n, 256) < 4736u ? nblk(n, 256) : 4736u, 256, 0, s>>>(V, m, ld, h, beta, y, n);
  count_launches(1);
  return cudaGetLastError();
}

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

// velocity rows of the preconditioner: diagonal of M_V, identity on fixed rows
__device__ __forceinline__ double jacobi_v(const ElemParams& P, const double* __restrict__ dmv,
                                           const double* __restrict__ r, long long n1, long long j) {
  const int comp = (int)(j / P.NV);
  const long long nd = j % P.NV;
  long long ic;
  int Nc;
  if (comp == 0) { ic = nd % P.N0; Nc = P.N0; }
  else if (comp == 1) { ic = (nd / P.N0) % P.N1; Nc = P.N1; }
  else { ic = nd / ((long long)P.N0 * P.N1); Nc = P.N2; }
  const bool fixed = (((P.bc >> (2 * comp)) & 1u) && ic == 0) || (((P.bc >> (2 * comp + 1)) & 1u) && ic == Nc - 1);
  return fixed ? r[n1 + j] : r[n1 + j] / dmv[nd];
}

// block upper-triangular preconditioner: z_v = D_V^-1 r_v, z_x = r_x + tau z_v (exact
// elimination of the dR_x/dk_v = -tau I coupling), z_e = M_E^-1 r_e
template <class TZ>
__global__ void k_precond(ElemParams P, const double* __restrict__ dmv, const double* __restrict__ ime,
                          const double* __restrict__ r, TZ* __restrict__ z, double tau) {
  const long long n1 = (long long)P.dim * P.NV;
  const long long n = 2 * n1 + P.NEd;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i < n1) {
    z[i] = TZ(r[i] + tau * jacobi_v(P, dmv, r, n1, i));
  } else if (i < 2 * n1) {
    z[i] = TZ(jacobi_v(P, dmv, r, n1, i - n1));
  } else {
    z[i] = TZ(r[i] * ime[i - 2 * n1]);
  }
}

cudaError_t launch_precond(cudaStream_t s, const ElemParams& P, const double* diag_mv, const double* inv_me,
                           const double* r, double* z, double tau) {
  const long long n = 2LL * P.dim * P.NV + P.NEd;
  k_precond<double><<<nblk(n, 256), 256, 0, s>>>(P, diag_mv, inv_me, r, z, tau);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_precond_f32(cudaStream_t s, const ElemParams& P, const double* diag_mv, const double* inv_me,
                               const double* r, float* z, double tau) {
  const long long n = 2LL * P.dim * P.NV + P.NEd;
  k_precond<float><<<nblk(n, 256), 256, 0, s>>>(P, diag_mv, inv_me, r, z, tau);
  count_launches(1);
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
