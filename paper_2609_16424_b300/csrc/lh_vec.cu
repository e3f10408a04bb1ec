// Vector kernels of the Newton-GMRES driver (paper Sec. 3.5, Eq. (22)): deterministic
// dot products, Gram-Schmidt updates, the block-diagonal preconditioner and precision
// conversions.  All are HBM-bound streaming kernels over the n unknowns.
#include <cfloat>
#include "lh_kernels.h"

namespace lh {

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// block sum in fixed order (tree over shared memory); result in red[0]
__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// partials[j * gridDim.x + b] = sum over this block's contiguous chunk of V_j . w
__global__ void __launch_bounds__(kRedThreads)
k_mdot_part(const double* __restrict__ V, int m, long long ld, const double* __restrict__ w, long long n,
            double* __restrict__ part) {
  __shared__ double red[kRedThreads];
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long beg = (long long)blockIdx.x * chunk;
  const long long end = beg + chunk < n ? beg + chunk : n;
  for (int j = 0; j < m; ++j) {
    const double* v = V + j * ld;
    double s = 0.0;
    if (w) {
      for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) s += v[i] * w[i];
    } else {
      for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) s += v[i];
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(long long)j * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kRedThreads)
k_sum_part(const double* __restrict__ part, int nb, int m, double* __restrict__ out) {
  __shared__ double red[kRedThreads];
  for (int j = 0; j < m; ++j) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(long long)j * nb + b];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[j] = s;
  }
}

cudaError_t launch_mdot(cudaStream_t s, const double* V, int m, long long ld, const double* w, long long n,
                        double* partials, double* out_dev) {
  k_mdot_part<<<kRedBlocks, kRedThreads, 0, s>>>(V, m, ld, w, n, partials);
  k_sum_part<<<1, kRedThreads, 0, s>>>(partials, kRedBlocks, m, out_dev);
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
  return cudaGetLastError();
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

cudaError_t launch_axpby(cudaStream_t s, double a, const double* x, double b, double* y, long long n) {
  if (n > 0) k_axpby<<<nblk(n, 256), 256, 0, s>>>(a, x, b, y, n);
  return cudaGetLastError();
}

// y = x * (1 / scale_dev[0])
__global__ void k_scale_copy(const double* __restrict__ x, const double* __restrict__ sc, double* __restrict__ y,
                             long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] / sc[0];
}

cudaError_t launch_scale_copy(cudaStream_t s, const double* x, const double* scale_dev, double* y, long long n) {
  if (n > 0) k_scale_copy<<<nblk(n, 256), 256, 0, s>>>(x, scale_dev, y, n);
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
  if (n > 0) k_to_f32<<<nblk(n, 256), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}
cudaError_t launch_to_f64(cudaStream_t s, const float* x, double* y, long long n) {
  if (n > 0) k_to_f64<<<nblk(n, 256), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

__global__ void k_precond(ElemParams P, const double* __restrict__ dmv, const double* __restrict__ ime,
                          const double* __restrict__ r, double* __restrict__ z) {
  const long long n1 = (long long)P.dim * P.NV;
  const long long n = 2 * n1 + P.NEd;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i < n1) {
    z[i] = r[i];
  } else if (i < 2 * n1) {
    const long long j = i - n1;
    const int comp = (int)(j / P.NV);
    const long long nd = j % P.NV;
    long long ic;
    int Nc;
    if (comp == 0) { ic = nd % P.N0; Nc = P.N0; }
    else if (comp == 1) { ic = (nd / P.N0) % P.N1; Nc = P.N1; }
    else { ic = nd / ((long long)P.N0 * P.N1); Nc = P.N2; }
    const bool fixed = (((P.bc >> (2 * comp)) & 1u) && ic == 0) || (((P.bc >> (2 * comp + 1)) & 1u) && ic == Nc - 1);
    z[i] = fixed ? r[i] : r[i] / dmv[nd];
  } else {
    z[i] = r[i] * ime[i - 2 * n1];
  }
}

cudaError_t launch_precond(cudaStream_t s, const ElemParams& P, const double* diag_mv, const double* inv_me,
                           const double* r, double* z) {
  const long long n = 2LL * P.dim * P.NV + P.NEd;
  k_precond<<<nblk(n, 256), 256, 0, s>>>(P, diag_mv, inv_me, r, z);
  return cudaGetLastError();
}

__global__ void k_jacobi_h1(long long nv, int dim, const double* __restrict__ diag, const double* __restrict__ r,
                            double* __restrict__ z) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nv * dim) z[i] = r[i] / diag[i % nv];
}

cudaError_t launch_jacobi_h1(cudaStream_t s, long long nv, int dim, const double* diag, const double* r, double* z) {
  k_jacobi_h1<<<nblk(nv * dim, 256), 256, 0, s>>>(nv, dim, diag, r, z);
  return cudaGetLastError();
}

__global__ void k_mul(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] * b[i];
}

cudaError_t launch_mul(cudaStream_t s, const double* a, const double* b, double* y, long long n) {
  if (n > 0) k_mul<<<nblk(n, 256), 256, 0, s>>>(a, b, y, n);
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
