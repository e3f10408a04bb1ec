// Learned Newton initial guess: a per-element MLP trained and evaluated on the GPU.
//
// The paper initialises each stage solve from the previous increment (Sec. 3.5 leaves the
// initial guess open).  This addition predicts the correction k^n - k^{n-1} per element
// from the element dofs of the last two increments and dt; the element predictions are
// averaged onto the shared H1 nodes.
//
// Network: Linear -> GELU -> ... -> Linear, exact GELU z Phi(z), mean-squared-error loss,
// Adam with bias correction.  Matrix products run on the 5th-generation tensor cores
// (tcgen05.mma kind::f16 issued by one thread, operands rounded to BF16 and staged in shared
// memory, FP32 accumulators in tensor memory read back by tcgen05.ld for the bias / GELU
// epilogue); master weights, biases, activations and the optimiser state are FP32.  Every
// reduction has a fixed order (deterministic).
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "lh_internal.h"
#include "lh_kernels.h"
#include "lh_tc.cuh"

namespace {

// tile of one CTA: 128 rows (tensor-memory lanes) x 64 columns, K staged 64 at a time
constexpr int kTM = 128, kTN = 64, kTK = 64;
constexpr uint32_t kSboA = (uint32_t)(kTK / 8) * 128u;   // bytes between 8-row groups (K-major interleaved)
constexpr uint32_t kWaitPolls = 1u << 22;                 // mbarrier polls before giving up

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// C[m][n] (=|+=) act( sum_k A(m,k) B(k,n) + bias[n] ), A(m,k) = A[m*lam + k*lak],
// B(k,n) = B[k*lbk + n*lbn]; Z (optional) receives the pre-activation.  act: 0 none, 1 GELU.
// Block 128 threads; tile kTM x kTN.  The threads stage A and B as BF16 in the K-major
// interleaved layout (8-row x 16-byte core matrices; the staging loop runs along whichever
// index has unit stride, so either operand may be K- or MN-major in memory); thread 0
// issues four K = 16 MMAs per stage into the FP32 accumulator in tensor memory and commits
// to an mbarrier that every thread waits on (bounded: after a timeout the tile's outputs are
// NaN and *err is set).  Each warp reads its 32 accumulator lanes for the epilogue.
__global__ void __launch_bounds__(128)
k_gemm_tc(int M, int N, int K, const float* __restrict__ A, long long lam, long long lak,
          const float* __restrict__ B, long long lbk, long long lbn, const float* __restrict__ bias, int act,
          float* __restrict__ Z, float* __restrict__ C, long long ldc, int accumulate, int* __restrict__ err) {
  using namespace lh;
  __shared__ __align__(1024) unsigned char sA[kTM * kTK * 2];
  __shared__ __align__(1024) unsigned char sB[kTN * kTK * 2];
  __shared__ uint64_t mbar, mdrain;
  __shared__ uint32_t taddr;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(&taddr, kTN);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_init(&mdrain, 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = taddr;
  const uint32_t idesc = tc::instr_desc(tc::KIND_BF16, kTM, kTN);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < K; k0 += kTK) {
    // stage A [kTM x kTK] and B [kTN x kTK] (rows m resp. n, K index c)
    const bool a_k_fast = lak == 1;
    for (int idx = tid; idx < kTM * kTK; idx += 128) {
      const int r = a_k_fast ? idx / kTK : idx % kTM, c = a_k_fast ? idx % kTK : idx / kTM;
      const int gm = m0 + r, gk = k0 + c;
      const float v = (gm < M && gk < K) ? A[gm * lam + gk * lak] : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(sA + tc::off_il(r, c, 2, 128u, kSboA)) = __float2bfloat16_rn(v);
    }
    const bool b_k_fast = lbk == 1;
    for (int idx = tid; idx < kTN * kTK; idx += 128) {
      const int r = b_k_fast ? idx / kTK : idx % kTN, c = b_k_fast ? idx % kTK : idx / kTN;
      const int gn = n0 + r, gk = k0 + c;
      const float v = (gn < N && gk < K) ? B[gk * lbk + gn * lbn] : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(sB + tc::off_il(r, c, 2, 128u, kSboA)) = __float2bfloat16_rn(v);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    tc::fence_after_sync();
    if (!ok) break;
    if (tid == 0) {
#pragma unroll
      for (int j = 0; j < kTK / 16; ++j) {
        const uint32_t ko = (uint32_t)(j * 2) * 128u;   // two core matrices (16 K entries) per MMA
        tc::mma<tc::KIND_BF16>(tm, tc::smem_desc(tc::smem_u32(sA) + ko, 128u, kSboA, tc::SW_NONE),
                               tc::smem_desc(tc::smem_u32(sB) + ko, 128u, kSboA, tc::SW_NONE), idesc,
                               k0 > 0 || j > 0);
      }
      tc::commit(&mbar);
    }
    ok = tc::mbar_wait(&mbar, phase, kWaitPolls);   // the stage is read: shared memory reusable
    phase ^= 1u;
  }
  tc::fence_before_sync();
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  tc::fence_after_sync();
  if (!ok && tid == 0) {   // record the timeout, let issued MMAs drain before releasing tensor memory
    atomicExch(err, 1);
    tc::commit(&mdrain);
    tc::mbar_wait(&mdrain, 0, kWaitPolls);
  }
  const int r = m0 + 32 * warp + lane;
#pragma unroll 1
  for (int ch = 0; ch < kTN / 8; ++ch) {
    float v[8];
    if (ok) {
      tc::tmem_ld8(tm + ((uint32_t)(32 * warp) << 16) + (uint32_t)(8 * ch), v);
      tc::tmem_wait_ld();
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = n0 + 8 * ch + t;
      if (r >= M || c >= N) continue;
      float z = ok ? v[t] + (bias ? bias[c] : 0.f) : __int_as_float(0x7fc00000);
      if (Z) Z[r * ldc + c] = z;
      const float y = act == 1 ? gelu(z) : z;
      if (accumulate) C[r * ldc + c] += y;
      else C[r * ldc + c] = y;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tm, kTN);
}

// dZ = dH * GELU'(Z)
__global__ void k_gelu_back(const float* __restrict__ dH, const float* __restrict__ Z, float* __restrict__ dZ,
                            long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dZ[i] = dH[i] * gelu_grad(Z[i]);
}

// R = Y - T, dY = 2 R / (M N), per-block partial sums of R^2 (fixed partition)
__global__ void __launch_bounds__(256)
k_mse(const float* __restrict__ Y, const float* __restrict__ T, long long n, float* __restrict__ dY,
      double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  const float sc = 2.f / (float)n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = Y[i] - T[i];
    dY[i] = sc * r;
    s += (double)r * r;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// db[n] = sum_m dZ[m][n]  (one block per column, fixed-order tree)
__global__ void __launch_bounds__(256)
k_colsum(const float* __restrict__ dZ, int M, int N, float* __restrict__ db) {
  __shared__ float red[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int m = threadIdx.x; m < M; m += blockDim.x) s += dZ[(long long)m * N + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = red[0];
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---- features and the nodal average of element predictions --------------------------------
// element e, local H1 node a -> global lattice node
__device__ __forceinline__ long long elem_node(const lh::ElemParams& P, long long e, int a) {
  const int D = P.K + 1;
  const long long ex = e % P.n0, ey = (e / P.n0) % P.n1, ez = e / ((long long)P.n0 * P.n1);
  const int a0 = a % D, a1 = (a / D) % D, a2 = a / (D * D);
  const long long i0 = ex * P.K + a0, i1 = ey * P.K + a1, i2 = P.dim == 3 ? ez * P.K + a2 : 0;
  return i0 + (long long)P.N0 * (i1 + (long long)P.N1 * i2);
}

// X[e][f]: f < F1: element dofs of k1 = [x (dim*ND) | v (dim*ND) | e (NL)] scaled by
// 1/scale[group]; then the same for k2; last feature dt / scale[3].
__global__ void k_features(lh::ElemParams P, int ND, int NL, const double* __restrict__ k1,
                           const double* __restrict__ k2, double dt, const float* __restrict__ scale,
                           float* __restrict__ X, int F) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.NE * F) return;
  const long long e = t / F;
  const int f = (int)(t % F);
  const int F1 = 2 * P.dim * ND + NL;
  float v;
  if (f == 2 * F1) {
    v = (float)(dt / scale[3]);
  } else {
    const double* k = f < F1 ? k1 : k2;
    const int g = f % F1;
    if (g < 2 * P.dim * ND) {
      const int comp = g / ND, a = g % ND;   // comp < dim: x rows, else v rows
      v = (float)(k[comp * P.NV + elem_node(P, e, a)] / scale[comp < P.dim ? 0 : 1]);
    } else {
      v = (float)(k[2 * P.dim * P.NV + e * NL + (g - 2 * P.dim * ND)] / scale[2]);
    }
  }
  X[t] = v;
}

// Initial guess from element predictions Y [NE][F2], F2 = dim ND + NL (v rows, then e rows,
// scaled by scale[1] / scale[2]):
//   v rows: k0_v = k1_v + average over the elements sharing the node; 0 on fixed rows;
//   e rows: k0_e = k1_e + the element's own prediction;
//   x rows: k0_x = u_v + tau k0_v, which solves R_x = k_x - u_v - tau k_v = 0 exactly.
// One thread per node and velocity component (writes its v and x entries) or per L2 dof;
// the elements around a node are visited in a fixed order.
__global__ void k_scatter_pred(lh::ElemParams P, int ND, int NL, const double* __restrict__ u, double tau,
                               const double* __restrict__ k1, const float* __restrict__ Y, int F2,
                               const float* __restrict__ scale, double* __restrict__ k0) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n1 = (long long)P.dim * P.NV;
  if (i >= n1 + P.NEd) return;
  if (i >= n1) {
    const long long j = i - n1, e = j / NL;
    k0[2 * n1 + j] = k1[2 * n1 + j] + (double)Y[e * F2 + P.dim * ND + j % NL] * scale[2];
    return;
  }
  const int comp = (int)(i / P.NV);
  const long long nd = i % P.NV;
  const int D = P.K + 1;
  const long long ic[3] = {nd % P.N0, (nd / P.N0) % P.N1, nd / ((long long)P.N0 * P.N1)};
  const int nel[3] = {P.n0, P.n1, P.n2};
  const int Nn[3] = {P.N0, P.N1, P.N2};
  const bool fixed = (((P.bc >> (2 * comp)) & 1u) && ic[comp] == 0) ||
                     (((P.bc >> (2 * comp + 1)) & 1u) && ic[comp] == Nn[comp] - 1);
  double kv = 0.0;
  if (!fixed) {
    int el[3][2], loc[3][2], cnt[3];
    for (int d = 0; d < 3; ++d) {
      cnt[d] = 0;
      if (d >= P.dim) {
        el[d][0] = 0;
        loc[d][0] = 0;
        cnt[d] = 1;
        continue;
      }
      const int q = (int)(ic[d] / P.K), r = (int)(ic[d] % P.K);
      if (r == 0) {
        if (q >= 1) { el[d][cnt[d]] = q - 1; loc[d][cnt[d]] = P.K; ++cnt[d]; }
        if (q < nel[d]) { el[d][cnt[d]] = q; loc[d][cnt[d]] = 0; ++cnt[d]; }
      } else {
        el[d][0] = q;
        loc[d][0] = r;
        cnt[d] = 1;
      }
    }
    double s = 0.0;
    int c = 0;
    for (int a2 = 0; a2 < cnt[2]; ++a2)
      for (int a1 = 0; a1 < cnt[1]; ++a1)
        for (int a0 = 0; a0 < cnt[0]; ++a0) {
          const long long e = el[0][a0] + (long long)P.n0 * (el[1][a1] + (long long)P.n1 * el[2][a2]);
          const int a = loc[0][a0] + D * (loc[1][a1] + D * loc[2][a2]);
          s += (double)Y[e * F2 + comp * ND + a];
          ++c;
        }
    kv = k1[n1 + i] + s / c * scale[1];
  }
  k0[n1 + i] = kv;
  k0[i] = u[n1 + i] + tau * kv;
}

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct lh_mlp {
  int n_in = 0, hidden = 0, layers = 0, n_out = 0;
  long long n_params = 0;
  cudaStream_t stream = nullptr;
  float* d_w = nullptr;      // parameters, flat: W_1 [h][in], b_1 [h], ...
  float* d_g = nullptr;      // gradients (same layout)
  float* d_m = nullptr;      // Adam first moments
  float* d_v = nullptr;      // Adam second moments
  int t = 0;                 // Adam step count
  float* d_act = nullptr;    // activations / pre-activations workspace
  long long act_cap = 0;
  double* d_part = nullptr;  // loss partials
  int* d_err = nullptr;      // set by a tensor-core GEMM whose bounded wait timed out
  std::string err;
  std::vector<long long> woff, boff;   // parameter offsets per layer
  std::vector<int> din, dout;          // layer shapes
};

namespace {

lh_status mfail(lh_mlp* m, lh_status st, const std::string& msg) {
  if (m) m->err = msg;
  return lh::set_global_error(st, msg);
}

#define MLP_CK(m, call)                                                                    \
  do {                                                                                     \
    cudaError_t e__ = (call);                                                              \
    if (e__ != cudaSuccess) return mfail(m, LH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
  } while (0)

// the flag of the tensor-core GEMMs' bounded waits (synchronises; clears the flag)
lh_status check_tc(lh_mlp* m) {
  int flag = 0;
  MLP_CK(m, cudaMemcpyAsync(&flag, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  MLP_CK(m, cudaStreamSynchronize(m->stream));
  if (!flag) return LH_OK;
  MLP_CK(m, cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream));
  return mfail(m, LH_ECUDA, "MLP: a bounded wait on the tensor cores timed out (results are NaN)");
}

cudaError_t gemm(cudaStream_t s, int M, int N, int K, const float* A, long long lam, long long lak, const float* B,
                 long long lbk, long long lbn, const float* bias, int act, float* Z, float* C, long long ldc,
                 int accumulate, int* err) {
  dim3 grid(nb(N, kTN), nb(M, kTM));
  k_gemm_tc<<<grid, 128, 0, s>>>(M, N, K, A, lam, lak, B, lbk, lbn, bias, act, Z, C, ldc, accumulate, err);
  lh::count_launches(1);
  return cudaGetLastError();
}

// activations workspace for a batch of M rows: per layer l the input H_l [M][din_l] and the
// pre-activation Z_l [M][dout_l]; plus dY / dH / dZ scratch [M][max dim] x 2
lh_status ensure_act(lh_mlp* m, int M) {
  long long need = 0;
  for (size_t l = 0; l < m->din.size(); ++l) need += (long long)M * (m->din[l] + m->dout[l]);
  int mx = std::max(m->n_in, std::max(m->hidden, m->n_out));
  need += 2LL * M * mx + (long long)M * m->n_out;
  if (need <= m->act_cap) return LH_OK;
  if (m->d_act) cudaFree(m->d_act);
  m->d_act = nullptr;
  if (cudaMalloc(&m->d_act, sizeof(float) * need) != cudaSuccess) return mfail(m, LH_ENOMEM, "MLP workspace");
  m->act_cap = need;
  return LH_OK;
}

// forward over M rows; H_0 = X (copied), returns pointer to Y (= Z of the last layer)
lh_status forward(lh_mlp* m, const float* X, int M, float** Hs, float** Zs) {
  cudaStream_t s = m->stream;
  float* p = m->d_act;
  const int L = (int)m->din.size();
  for (int l = 0; l < L; ++l) {
    Hs[l] = p;
    p += (long long)M * m->din[l];
    Zs[l] = p;
    p += (long long)M * m->dout[l];
  }
  MLP_CK(m, cudaMemcpyAsync(Hs[0], X, sizeof(float) * (size_t)M * m->n_in, cudaMemcpyDeviceToDevice, s));
  for (int l = 0; l < L; ++l) {
    const bool last = l == L - 1;
    float* out = last ? Zs[l] : Hs[l + 1];
    MLP_CK(m, gemm(s, M, m->dout[l], m->din[l], Hs[l], m->din[l], 1, m->d_w + m->woff[l], 1, m->din[l],
                   m->d_w + m->boff[l], last ? 0 : 1, last ? nullptr : Zs[l], out, m->dout[l], 0, m->d_err));
  }
  return LH_OK;
}

}  // namespace

extern "C" {

lh_status lh_mlp_create(int n_in, int hidden, int layers, int n_out, const float* init_params, void* stream,
                        lh_mlp** out) {
  if (!out) return mfail(nullptr, LH_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_in < 1 || hidden < 1 || layers < 1 || n_out < 1 || layers > 16)
    return mfail(nullptr, LH_EINVAL, "lh_mlp_create: bad shape");
  lh_mlp* m = new (std::nothrow) lh_mlp();
  if (!m) return mfail(nullptr, LH_ENOMEM, "host allocation failed");
  m->n_in = n_in;
  m->hidden = hidden;
  m->layers = layers;
  m->n_out = n_out;
  m->stream = reinterpret_cast<cudaStream_t>(stream);
  std::vector<int> dims{n_in};
  for (int l = 0; l < layers; ++l) dims.push_back(hidden);
  dims.push_back(n_out);
  long long o = 0;
  for (size_t l = 0; l + 1 < dims.size(); ++l) {
    m->din.push_back(dims[l]);
    m->dout.push_back(dims[l + 1]);
    m->woff.push_back(o);
    o += (long long)dims[l + 1] * dims[l];
    m->boff.push_back(o);
    o += dims[l + 1];
  }
  m->n_params = o;
  const size_t bytes = sizeof(float) * o;
  if (cudaMalloc(&m->d_w, bytes) != cudaSuccess || cudaMalloc(&m->d_g, bytes) != cudaSuccess ||
      cudaMalloc(&m->d_m, bytes) != cudaSuccess || cudaMalloc(&m->d_v, bytes) != cudaSuccess ||
      cudaMalloc(&m->d_part, sizeof(double) * 1024) != cudaSuccess ||
      cudaMalloc(&m->d_err, sizeof(int)) != cudaSuccess || cudaMemset(m->d_err, 0, sizeof(int)) != cudaSuccess) {
    lh_mlp_destroy(m);
    return mfail(nullptr, LH_ENOMEM, "lh_mlp_create: device allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(m->d_m, 0, bytes, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_v, 0, bytes, m->stream);
  if (e == cudaSuccess && init_params)
    e = cudaMemcpyAsync(m->d_w, init_params, bytes, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess && !init_params) e = cudaMemsetAsync(m->d_w, 0, bytes, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    lh_mlp_destroy(m);
    return mfail(nullptr, LH_ECUDA, std::string("lh_mlp_create: ") + cudaGetErrorString(e));
  }
  *out = m;
  return LH_OK;
}

lh_status lh_mlp_destroy(lh_mlp* m) {
  if (!m) return LH_OK;
  float* bufs[] = {m->d_w, m->d_g, m->d_m, m->d_v, m->d_act};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (m->d_part) cudaFree(m->d_part);
  if (m->d_err) cudaFree(m->d_err);
  delete m;
  return LH_OK;
}

long long lh_mlp_num_params(const lh_mlp* m) { return m ? m->n_params : 0; }

lh_status lh_mlp_params(lh_mlp* m, float* host_out) {
  if (!m || !host_out) return mfail(m, LH_EINVAL, "NULL argument to lh_mlp_params");
  MLP_CK(m, cudaMemcpyAsync(host_out, m->d_w, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, m->stream));
  MLP_CK(m, cudaStreamSynchronize(m->stream));
  return check_tc(m);
}

lh_status lh_mlp_forward(lh_mlp* m, const float* X, int M, float* Y) {
  if (!m || !X || !Y || M < 1) return mfail(m, LH_EINVAL, "bad argument to lh_mlp_forward");
  lh_status st = ensure_act(m, M);
  if (st != LH_OK) return st;
  std::vector<float*> Hs(m->din.size()), Zs(m->din.size());
  if ((st = forward(m, X, M, Hs.data(), Zs.data())) != LH_OK) return st;
  MLP_CK(m, cudaMemcpyAsync(Y, Zs.back(), sizeof(float) * (size_t)M * m->n_out, cudaMemcpyDeviceToDevice,
                            m->stream));
  return LH_OK;
}

lh_status lh_mlp_grad(lh_mlp* m, const float* X, const float* T, int M, float* grad_out, double* loss) {
  if (!m || !X || !T || M < 1) return mfail(m, LH_EINVAL, "bad argument to lh_mlp_grad");
  lh_status st = ensure_act(m, M);
  if (st != LH_OK) return st;
  const int L = (int)m->din.size();
  std::vector<float*> Hs(L), Zs(L);
  if ((st = forward(m, X, M, Hs.data(), Zs.data())) != LH_OK) return st;
  cudaStream_t s = m->stream;
  float* scratch = Zs[L - 1] + (long long)M * m->dout[L - 1];
  const int mx = std::max(m->n_in, std::max(m->hidden, m->n_out));
  float* dA = scratch;                      // dZ of the current layer
  float* dB = scratch + (long long)M * mx;  // dH of the layer below
  const long long ny = (long long)M * m->n_out;
  const int pb = 592;
  k_mse<<<pb, 256, 0, s>>>(Zs[L - 1], T, ny, dA, m->d_part);
  lh::count_launches(1);
  MLP_CK(m, cudaGetLastError());
  for (int l = L - 1; l >= 0; --l) {
    const int N = m->dout[l], K = m->din[l];
    // dW_l = dZ^T H_l  ([N][K], reduction over the M rows), db_l = column sums of dZ
    MLP_CK(m, gemm(s, N, K, M, dA, 1, N, Hs[l], K, 1, nullptr, 0, nullptr, m->d_g + m->woff[l], K, 0, m->d_err));
    k_colsum<<<N, 256, 0, s>>>(dA, M, N, m->d_g + m->boff[l]);
    lh::count_launches(1);
    if (l == 0) break;
    // dH_l = dZ W_l ([M][K]); dZ_{l-1} = dH_l * GELU'(Z_{l-1})
    MLP_CK(m, gemm(s, M, K, N, dA, N, 1, m->d_w + m->woff[l], K, 1, nullptr, 0, nullptr, dB, K, 0, m->d_err));
    k_gelu_back<<<nb((long long)M * K, 256), 256, 0, s>>>(dB, Zs[l - 1], dA, (long long)M * K);
    lh::count_launches(1);
    MLP_CK(m, cudaGetLastError());
  }
  if (loss) {
    std::vector<double> part(pb);
    MLP_CK(m, cudaMemcpyAsync(part.data(), m->d_part, sizeof(double) * pb, cudaMemcpyDeviceToHost, s));
    MLP_CK(m, cudaStreamSynchronize(s));
    double sum = 0.0;
    for (int i = 0; i < pb; ++i) sum += part[i];
    *loss = sum / (double)ny;
    if ((st = check_tc(m)) != LH_OK) return st;
  }
  if (grad_out)
    MLP_CK(m, cudaMemcpyAsync(grad_out, m->d_g, sizeof(float) * m->n_params, cudaMemcpyDeviceToDevice, s));
  return LH_OK;
}

lh_status lh_mlp_train_step(lh_mlp* m, const float* X, const float* T, int M, float lr, double* loss) {
  lh_status st = lh_mlp_grad(m, X, T, M, nullptr, loss);
  if (st != LH_OK) return st;
  ++m->t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)m->t), c2 = 1.f - std::pow(b2, (float)m->t);
  k_adam<<<nb(m->n_params, 256), 256, 0, m->stream>>>(m->d_w, m->d_g, m->d_m, m->d_v, m->n_params, lr, b1, b2,
                                                      1e-8f, c1, c2);
  lh::count_launches(1);
  MLP_CK(m, cudaGetLastError());
  return LH_OK;
}

const char* lh_mlp_last_error(const lh_mlp* m) { return m ? m->err.c_str() : ""; }

lh_status lh_mlp_features(lh_mesh* mesh, const double* k1, const double* k2, double dt, const float* scale,
                          float* X) {
  if (!mesh || !k1 || !k2 || !scale || !X) return lh::set_global_error(LH_EINVAL, "NULL argument to lh_mlp_features");
  const lh::ElemParams& P = mesh->P;
  int ND = 1, NL = 1;
  for (int c = 0; c < P.dim; ++c) {
    ND *= P.K + 1;
    NL *= P.K;
  }
  const int F = 2 * (2 * P.dim * ND + NL) + 1;
  k_features<<<nb(P.NE * F, 256), 256, 0, mesh->stream>>>(P, ND, NL, k1, k2, dt, scale, X, F);
  lh::count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LH_OK : lh::set_global_error(LH_ECUDA, cudaGetErrorString(e));
}

lh_status lh_mlp_apply_prediction(lh_mesh* mesh, const double* u, double tau, const double* k1, const float* Y,
                                  const float* scale, double* k0) {
  if (!mesh || !u || !k1 || !Y || !scale || !k0)
    return lh::set_global_error(LH_EINVAL, "NULL argument to lh_mlp_apply_prediction");
  const lh::ElemParams& P = mesh->P;
  int ND = 1, NL = 1;
  for (int c = 0; c < P.dim; ++c) {
    ND *= P.K + 1;
    NL *= P.K;
  }
  const int F2 = P.dim * ND + NL;
  const long long nthreads = (long long)P.dim * P.NV + P.NEd;
  k_scatter_pred<<<nb(nthreads, 256), 256, 0, mesh->stream>>>(P, ND, NL, u, tau, k1, Y, F2, scale, k0);
  lh::count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LH_OK : lh::set_global_error(LH_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
