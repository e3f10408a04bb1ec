// Tensor-core Jacobian action from the linearisation record (mixed precision J.w inside
// GMRES; the tangent of paper Sec. 3.1, Eq. (10), with the element operator B of Sec. 2.2,
// Eq. (8), applied on the 5th-generation tensor cores).
//
// The element interpolation of a batch of EB = 16 elements is a dense MMA per sub-chunk of
// QS = 16 quadrature points (the next sub-chunk's MMA runs while this one is processed):
//   D_f[(c, e)][(q, r)] = sum_k U[(c, e)][k] Bf[(q, r)][k]
// rows (c, e) = component c of the direction (dk_x, dk_v, dk_e) of element e (M = 128:
// 8 component slots x 16 elements), K = element dofs (H1 then L2), columns (q, r) = value
// (r = 0) and reference derivatives (r = 1..dim) at quadrature point q.  The transposed
// operator B^T is a second MMA per sub-chunk of 16 quadrature points, accumulated over
// the sub-chunks:
//   D_b[(c', e)][a] += sum_(q, r) F[(c', e)][(q, r)] Bb[a][(q, r)]
// with F = (m_q dv_q, S-tangent) for the H1 rows c' < dim and (g_q, 0, ..) for the L2 row
// c' = dim.  Operands are TF32 or BF16 in shared memory, accumulators FP32 in tensor
// memory.  Between the two MMAs the linearised point map of Eqs. (11)-(20), read from the
// linearisation record the FP64 residual wrote, is applied in FP32 on the CUDA cores, one
// thread per (element, quadrature point).
//
// Dense element operators are (Q^d x 4) x (D^d + L^d) entries; they fit in shared memory
// for 2D k <= 4 and 3D k <= 2.  Persistent CTAs (two per SM with BF16 operands, one with
// TF32 by shared memory) each own 256 tensor-memory columns for the whole launch.
#include <atomic>
#include <cfloat>
#include <mutex>
#include "lh_internal.h"
#include "lh_kernels.h"
#include "lh_qp.cuh"
#include "lh_contract.cuh"
#include "lh_tc.cuh"

namespace lh {

namespace {

constexpr int EB = 16;    // elements per batch
constexpr int QS = 16;    // quadrature points per sub-chunk
constexpr int NTH = EB * QS;
constexpr uint32_t kWaitPolls = 1u << 22;   // default mbarrier polls before giving up
std::atomic<uint32_t> g_wait_polls{kWaitPolls};

__host__ __device__ constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int pow2_cols(int x) {
  return x <= 32 ? 32 : x <= 64 ? 64 : x <= 128 ? 128 : x <= 256 ? 256 : 512;
}

template <int DIM, int K, tc::Kind KIND>
struct TcPlan {
  using C = Cfg<DIM, K>;
  static constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ;
  static constexpr int NQP = rup(NQ, QS);          // padded quadrature points
  static constexpr int NSUB = NQP / QS;
  static constexpr int NF = 4 * NQP;               // forward N = TMEM columns of D_f
  static constexpr int MK = tc::mma_k(KIND);
  static constexpr int ESZ = tc::elem_bytes(KIND);
  static constexpr int T = 16 / ESZ;               // entries per 16-byte core row
  static constexpr int KF = rup(ND + NL, MK);      // forward K
  static constexpr int NB = rup(ND + NL, 16);      // backward N
  static constexpr int KB = 4 * NQP;               // backward K (all sub-chunks)
  static constexpr int KBC = 4 * QS;               // backward K per sub-chunk
  static constexpr int NCF = 2 * DIM + 1;          // forward component slots used
  static constexpr int NCB = DIM + 1;              // backward component slots used
  static constexpr int NCOLS = pow2_cols(2 * 4 * QS + NB);   // TMEM: two forward buffers + D_b
  // shared memory (bytes): A_b first (128-byte swizzle wants 1024-byte alignment)
  static constexpr uint32_t AB_ASTRIDE = 16u * 1024u;                 // 128 rows / 8 x 1024
  static constexpr uint32_t SZ_AB = 128u * KBC * ESZ;
  static constexpr uint32_t SBO_F = (uint32_t)(KF / T) * 128u;        // A_f and B_f row-group stride
  static constexpr uint32_t SBO_B = (uint32_t)(KB / T) * 128u;        // B_b row-group stride
  static constexpr uint32_t O_AB = 0;
  static constexpr uint32_t O_BF = O_AB + SZ_AB;
  static constexpr uint32_t O_BB = O_BF + (uint32_t)NF * KF * ESZ;
  static constexpr uint32_t O_AF = O_BB + (uint32_t)NB * KB * ESZ;
  static constexpr uint32_t O_X = O_AF + 128u * KF * ESZ;
  static constexpr uint32_t SZ_X = (uint32_t)EB * QS * 32 * 4;
  static constexpr uint32_t O_W = O_X + SZ_X;                          // 1D weights (float, 8)
  static constexpr uint32_t O_BAR = O_W + 32;                          // 3 mbarriers + taddr
  static constexpr uint32_t BYTES = O_BAR + 32 + 1024;                 // + alignment slack
  static_assert(NF <= 256 && NF % 16 == 0, "forward N out of range");
  static_assert(NB <= 256 && NB % 16 == 0, "backward N out of range");
  static_assert(2 * 4 * QS + NB <= 256, "tensor memory: two CTAs per SM");
  static_assert(KBC * ESZ % 128 == 0, "sub-chunk K must fill 128-byte atoms");
  static_assert((uint32_t)EB * (DIM * ND + NL) * 4 <= SZ_X, "output staging");
  static_assert(NCF <= 8 && NCB <= 4, "component slots");
  static_assert(BYTES <= 227u * 1024u, "shared memory");
};

// entry of the dense element operator: basis function idx (H1 node a < ND, else L2 dof
// ND + j) at quadrature point q, value (r = 0) or reference derivative r - 1
template <int DIM, int K>
__device__ __forceinline__ float basis_entry(const double* __restrict__ tab, int q, int r, int idx) {
  using C = Cfg<DIM, K>;
  constexpr int D = C::D, L = C::L, Q = C::Q;
  if (q >= C::NQ || r > DIM || idx >= C::ND + C::NL) return 0.f;
  int qd[3] = {q % Q, (q / Q) % Q, q / (Q * Q)};
  double v = 1.0;
  if (idx < C::ND) {
    const int ad[3] = {idx % D, (idx / D) % D, idx / (D * D)};
#pragma unroll
    for (int d = 0; d < DIM; ++d)
      v *= (r == d + 1) ? tab[Tab<K>::G + qd[d] * D + ad[d]] : tab[Tab<K>::B + qd[d] * D + ad[d]];
  } else {
    if (r != 0) return 0.f;
    const int j = idx - C::ND;
    const int jd[3] = {j % L, (j / L) % L, j / (L * L)};
#pragma unroll
    for (int d = 0; d < DIM; ++d) v *= tab[Tab<K>::BL + qd[d] * L + jd[d]];
  }
  return (float)v;
}

template <tc::Kind KIND>
__device__ __forceinline__ void put1(unsigned char* base, uint32_t off, float x) {
  if constexpr (KIND == tc::KIND_TF32) *reinterpret_cast<uint32_t*>(base + off) = tc::to_tf32(x);
  else *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(x);
}

// four consecutive K entries of one row (16 bytes of TF32 or 8 bytes of BF16)
template <tc::Kind KIND>
__device__ __forceinline__ void put4(unsigned char* base, uint32_t off, float a, float b, float c, float d) {
  if constexpr (KIND == tc::KIND_TF32) {
    *reinterpret_cast<uint4*>(base + off) = make_uint4(tc::to_tf32(a), tc::to_tf32(b), tc::to_tf32(c), tc::to_tf32(d));
  } else {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t*>(&lo);
    v.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(base + off) = v;
  }
}

__device__ __forceinline__ void cta_sync() {
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

// barrier that also makes the wait status uniform over the CTA: after one thread's wait has
// given up, every thread skips the remaining waits and MMA issues of the launch
__device__ __forceinline__ bool cta_sync_and(bool ok) {
  tc::fence_before_sync();
  const bool all = __syncthreads_and(ok ? 1 : 0) != 0;
  tc::fence_after_sync();
  return all;
}

template <int DIM, int K>
__device__ __forceinline__ long long node_lattice(const ElemParams& P, long long e, int a) {
  constexpr int D = K + 1;
  const int ex = (int)(e % P.n0), ey = (int)((e / P.n0) % P.n1);
  const int a0 = a % D, a1 = (a / D) % D;
  const long long i0 = (long long)ex * K + a0, i1 = (long long)ey * K + a1;
  if constexpr (DIM == 2) return i0 + (long long)P.N0 * i1;
  const int ez = (int)(e / ((long long)P.n0 * P.n1));
  const long long i2 = (long long)ez * K + a / (D * D);
  return i0 + (long long)P.N0 * (i1 + (long long)P.N1 * i2);
}

}  // namespace

template <int DIM, int K, tc::Kind KIND, class TO>
__global__ void __launch_bounds__(NTH, 2)
k_jvp_tc(ElemParams P, const float* __restrict__ rec, float tau, const float* __restrict__ dk,
         float* __restrict__ ev, TO* __restrict__ oute, int* __restrict__ err, uint32_t polls) {
  using PL = TcPlan<DIM, K, KIND>;
  using C = Cfg<DIM, K>;
  constexpr int ND = C::ND, NL = C::NL, NQ = C::NQ, Q = C::Q;
  constexpr int NR = lin_len<DIM>();
  constexpr int ESZ = PL::ESZ, MK = PL::MK;
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned base (the launch adds 1024 bytes of slack)
  unsigned char* sm = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sAb = sm + PL::O_AB;
  unsigned char* sBf = sm + PL::O_BF;
  unsigned char* sBb = sm + PL::O_BB;
  unsigned char* sAf = sm + PL::O_AF;
  float* sX = reinterpret_cast<float*>(sm + PL::O_X);
  float* sW = reinterpret_cast<float*>(sm + PL::O_W);
  uint64_t* mbf = reinterpret_cast<uint64_t*>(sm + PL::O_BAR);
  uint64_t* mbb = mbf + 1;
  uint64_t* mbd = mbf + 2;                 // drain barrier: used once, after a failed wait
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(mbf + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- set-up: tensor memory, barriers, constant operands, zeroed padding
  if (warp == 0) {
    tc::tmem_alloc(s_taddr, PL::NCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(mbf, 1);
    tc::mbar_init(mbb, 1);
    tc::mbar_init(mbd, 1);
    tc::fence_mbar_init();
  }
  for (uint32_t i = tid; i < PL::O_X / 16; i += NTH) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (tid < Q) sW[tid] = (float)P.tab[Tab<K>::W + tid];
  __syncthreads();
  for (int i = tid; i < PL::NF * PL::KF; i += NTH) {          // Bf[(q, r)][k]
    const int n = i / PL::KF, k = i % PL::KF;
    put1<KIND>(sBf, tc::off_il(n, k, ESZ, 128u, PL::SBO_F), basis_entry<DIM, K>(P.tab, n >> 2, n & 3, k));
  }
  for (int i = tid; i < PL::NB * PL::KB; i += NTH) {          // Bb[a][(q, r)]
    const int n = i / PL::KB, k = i % PL::KB;
    put1<KIND>(sBb, tc::off_il(n, k, ESZ, 128u, PL::SBO_B), basis_entry<DIM, K>(P.tab, k >> 2, k & 3, n));
  }
  tc::fence_proxy_async();
  cta_sync();
  const uint32_t tm = *s_taddr;
  // forward accumulators: two buffers of one sub-chunk (4 QS columns) each; then D_b
  const uint32_t tmf = tm, tmb = tm + 2 * PL::KBC;
  const uint32_t id_f = tc::instr_desc(KIND, 128, PL::KBC), id_b = tc::instr_desc(KIND, 128, PL::NB);
  // forward MMA of sub-chunk s: rows [KBC s, KBC (s + 1)) of Bf into buffer s & 1
  auto issue_fwd = [&](int s) {
    const uint32_t rowoff = (uint32_t)(PL::KBC * s / 8) * PL::SBO_F;
#pragma unroll
    for (int j = 0; j < PL::KF / MK; ++j) {
      const uint32_t ko = (uint32_t)(j * MK / PL::T) * 128u;
      tc::mma<KIND>(tmf + (uint32_t)((s & 1) * PL::KBC),
                    tc::smem_desc(tc::smem_u32(sAf) + ko, 128u, PL::SBO_F, tc::SW_NONE),
                    tc::smem_desc(tc::smem_u32(sBf) + rowoff + ko, 128u, PL::SBO_F, tc::SW_NONE), id_f, j > 0);
    }
    tc::commit(mbf);
  };
  uint32_t ph_f = 0, ph_b = 0;
  bool ok = true;


  const long long nbatch = (P.NE + EB - 1) / EB;
  for (long long b = blockIdx.x; b < nbatch; b += gridDim.x) {
    const long long e0 = b * EB;
    // ---- 1. gather the direction into A_f (rows c*16 + e)
    constexpr int PER_E = 2 * DIM * ND + NL;
    for (int i = tid; i < EB * PER_E; i += NTH) {
      const int e = i / PER_E, w = i % PER_E;
      const long long eg = e0 + e;
      const bool valid = eg < P.NE;
      float v = 0.f;
      int row, k;
      if (w < 2 * DIM * ND) {
        const int comp = w / ND, a = w % ND;
        row = comp * EB + e;
        k = a;
        if (valid) v = dk[comp * P.NV + node_lattice<DIM, K>(P, eg, a)];
      } else {
        const int j = w - 2 * DIM * ND;
        row = 2 * DIM * EB + e;
        k = ND + j;
        if (valid) v = dk[2 * DIM * P.NV + eg * NL + j];
      }
      put1<KIND>(sAf, tc::off_il(row, k, ESZ, 128u, PL::SBO_F), v);
    }
    tc::fence_proxy_async();
    cta_sync();
    // ---- 2. forward MMA of the first sub-chunk: D_f = U Bf^T (its 4 QS columns)
    if (tid == 0 && ok) issue_fwd(0);

    bool pending_b = false;
    for (int s = 0; s < PL::NSUB; ++s) {
      // the record of this thread's (element, point) does not depend on the MMA: issue its
      // loads first so their latency overlaps the transposition below
      const int e = tid / QS, ql = tid % QS;
      const int q = QS * s + ql;
      const long long eg = e0 + e;
      const bool valid = eg < P.NE && q < NQ;
      float Lr[NR];
      {
        const float* rq = rec + (valid ? eg * NR * NQ + q : 0);
#pragma unroll
        for (int f = 0; f < NR; ++f) Lr[f] = valid ? rq[f * NQ] : 0.f;
      }
      if (ok) ok = tc::mbar_wait(mbf, ph_f, polls);   // forward MMA of this sub-chunk
      ph_f ^= 1u;
      tc::fence_after_sync();
      // ---- 3. D_f columns of this sub-chunk -> sX[e][q][slot][r] (slot = c ^ e ^ q, 16 B)
      if (__syncthreads_or(ok ? 0 : 1) == 0) {
        const int quarter = warp & 3, half = warp >> 2;
        const int row = 32 * quarter + lane;
        const int cc = row / EB, er = row % EB;
        float v[16];
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const int col = (s & 1) * PL::KBC + 32 * half + 16 * part;
          tc::tmem_ld16(tmf + ((uint32_t)(32 * quarter) << 16) + (uint32_t)col, v);
          tc::tmem_wait_ld();
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int qw = 8 * half + 4 * part + t;
            const int slot = cc ^ (er & 7) ^ (qw & 7);
            *reinterpret_cast<float4*>(sX + ((er * QS + qw) * 8 + slot) * 4) =
                make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
          }
        }
      }
      ok = cta_sync_and(ok);
      // next sub-chunk's forward MMA, into the other buffer (read in the previous sub-chunk).
      // Issued only after this barrier: every thread has then finished its wait on the
      // current phase of mbf, so that barrier cannot run a phase ahead of a waiting thread.
      if (tid == 0 && ok && s + 1 < PL::NSUB) issue_fwd(s + 1);
      // ---- 4. quadrature-point tangent, thread = (e, ql)
      float fval[DIM], fgrad[DIM][DIM], g = 0.f;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        fval[i] = 0.f;
#pragma unroll
        for (int r = 0; r < DIM; ++r) fgrad[i][r] = 0.f;
      }
      if (valid) {
        float hv[2 * DIM + 1], hg[2 * DIM][DIM];
#pragma unroll
        for (int cc = 0; cc <= 2 * DIM; ++cc) {
          const int slot = cc ^ (e & 7) ^ (ql & 7);
          const float4 x = *reinterpret_cast<const float4*>(sX + ((e * QS + ql) * 8 + slot) * 4);
          hv[cc] = x.x;
          if (cc < 2 * DIM) {
            hg[cc][0] = x.y;
            hg[cc][1] = x.z;
            if constexpr (DIM == 3) hg[cc][2] = x.w;
          }
        }
        const int q0 = q % Q, q1 = (q / Q) % Q, q2 = q / (Q * Q);
        float a = sW[q0] * sW[q1];
        if constexpr (DIM == 3) a *= sW[q2];
        const float mq = P.fmq0[eg] * a;
        float dJ[DIM][DIM], dGv[DIM][DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
          for (int r = 0; r < DIM; ++r) {
            dJ[i][r] = tau * hg[i][r];
            dGv[i][r] = tau * hg[DIM + i][r];
          }
        const float lq = hv[2 * DIM];
        float dEo, dW;
        qp_tangent_lin<DIM>(Lr, dJ, dGv, tau * lq, P.fq1, P.fq2, P.visc != 0, fgrad, dEo, dW);
#pragma unroll
        for (int i = 0; i < DIM; ++i) fval[i] = mq * hv[DIM + i];
        g = mq * lq - dEo;
        if constexpr (DIM == 2) {
          if (P.tg) {   // d(W s(x_q)) = dW s + W grad s . dx
            constexpr int O = 2 * DIM * DIM;
            g -= dW * Lr[O + LF_TGS] + Lr[O + LF_W] * (Lr[O + LF_TGX] * tau * hv[0] + Lr[O + LF_TGY] * tau * hv[1]);
          }
        }
      }
      // ---- 5. F into A_b (the previous backward MMA must have finished reading it)
      if (pending_b) {
        if (ok) ok = tc::mbar_wait(mbb, ph_b, polls);
        ph_b ^= 1u;
        pending_b = false;
      }
#pragma unroll
      for (int i = 0; i < DIM; ++i)
        put4<KIND>(sAb, tc::off_sw128(i * EB + e, 4 * ql, ESZ, PL::AB_ASTRIDE), fval[i], fgrad[i][0], fgrad[i][1],
                   DIM == 3 ? fgrad[i][DIM - 1] : 0.f);
      put4<KIND>(sAb, tc::off_sw128(DIM * EB + e, 4 * ql, ESZ, PL::AB_ASTRIDE), g, 0.f, 0.f, 0.f);
      tc::fence_proxy_async();
      ok = cta_sync_and(ok);
      // ---- 6. backward MMA of this sub-chunk: D_b += F Bb^T (K slice of the sub-chunk)
      if (tid == 0 && ok) {
#pragma unroll
        for (int j = 0; j < PL::KBC / MK; ++j) {
          const int k0 = j * MK;
          const uint32_t ao = (uint32_t)(k0 * ESZ / 128) * PL::AB_ASTRIDE + (uint32_t)(k0 * ESZ % 128);
          const uint32_t bo = (uint32_t)((PL::KBC * s + k0) / PL::T) * 128u;
          tc::mma<KIND>(tmb, tc::smem_desc(tc::smem_u32(sAb) + ao, 16u, 1024u, tc::SW_128),
                        tc::smem_desc(tc::smem_u32(sBb) + bo, 128u, PL::SBO_B, tc::SW_NONE), id_b, s > 0 || j > 0);
        }
        tc::commit(mbb);
      }
      pending_b = ok;
    }
    // ---- 7. D_b -> staging (rows c'*16 + e in lanes 0..63) -> global
    if (ok) ok = tc::mbar_wait(mbb, ph_b, polls);
    ph_b ^= 1u;
    ok = cta_sync_and(ok);
    float* yh = sX;                         // [EB][DIM][ND]
    float* yl = sX + EB * DIM * ND;         // [EB][NL]
    {
      const int quarter = warp & 3, half = warp >> 2;
      if (quarter < 2) {
        const int row = 32 * quarter + lane;
        const int cc = row / EB, e = row % EB;
        for (int ch = half; ch < PL::NB / 8; ch += 2) {
          float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          if (ok) {
            tc::tmem_ld8(tmb + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(8 * ch), v);
            tc::tmem_wait_ld();
          }
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int a = 8 * ch + t;
            if (cc < DIM && a < ND) yh[(e * DIM + cc) * ND + a] = ok ? v[t] : __int_as_float(0x7fc00000);
            if (cc == DIM && a >= ND && a < ND + NL) yl[e * NL + a - ND] = ok ? v[t] : __int_as_float(0x7fc00000);
          }
        }
      }
    }
    cta_sync();
    {
      const long long nvalid = (P.NE - e0) < EB ? (P.NE - e0) : EB;
      float* evb = ev + e0 * (DIM * ND);
      for (int i = tid; i < nvalid * DIM * ND; i += NTH) evb[i] = yh[i];
      TO* ob = oute + e0 * NL;
      for (int i = tid; i < nvalid * NL; i += NTH) ob[i] = TO(yl[i]);
    }
    // the next batch's sub-chunk 3 overwrites sX only after the sync that follows its gather
  }
  if (!ok) {
    // a wait gave up: record it, then let the MMAs this CTA issued drain (a commit tracks
    // all of the issuing thread's earlier tcgen05 operations; bounded wait) before the
    // tensor memory is released
    if (tid == 0) {
      atomicExch(err, 1);
      tc::commit(mbd);
      tc::mbar_wait(mbd, 0, kWaitPolls);
    }
  }
  cta_sync();
  if (warp == 0) tc::tmem_dealloc(tm, PL::NCOLS);
}

namespace {

template <int DIM, int K, tc::Kind KIND, class TO>
cudaError_t run_tc(const ElemParams& P, cudaStream_t s, const float* rec, double tau, const float* dk, float* ev,
                   TO* out, int* err, cudaEvent_t* ev2) {
  using PL = TcPlan<DIM, K, KIND>;
  auto kern = k_jvp_tc<DIM, K, KIND, TO>;
  // launch shape per device (the shared-memory attribute is a per-device setting)
  constexpr int kMaxDev = 64;
  static int grids[kMaxDev] = {};
  static size_t bytes_of[kMaxDev] = {};
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  int& grid = grids[dev];
  size_t& bytes = bytes_of[dev];
  if (grid == 0) {
    // keep the CTAs that can share an SM within its 512 tensor-memory columns: pad the
    // shared-memory request so that at most 512 / NCOLS CTAs are resident per SM
    int nsm = 0;
    size_t smem_sm = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int v = 0;
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
    smem_sm = (size_t)v;
    const int max_by_tmem = 512 / PL::NCOLS;
    bytes = PL::BYTES;
    const size_t floor_bytes = smem_sm / (size_t)(max_by_tmem + 1) + 1024;
    if (bytes < floor_bytes) bytes = floor_bytes;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess)
      return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTH, bytes)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (per_sm > max_by_tmem) per_sm = max_by_tmem;
    grid = nsm * per_sm;
  }
  const long long nbatch = (P.NE + EB - 1) / EB;
  const int g = (int)(nbatch < grid ? nbatch : grid);
  if (ev2) cudaEventRecord(ev2[0], s);
  kern<<<g, NTH, bytes, s>>>(P, rec, (float)tau, dk, ev, out + 2 * DIM * P.NV, err,
                             g_wait_polls.load(std::memory_order_relaxed));
  if (ev2) cudaEventRecord(ev2[1], s);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_assemble_jvp<TO>(P, s, dk, tau, ev, out);
}

template <int DIM, int K, class TO>
cudaError_t run_tc_kind(const ElemParams& P, cudaStream_t s, int kind, const float* rec, double tau,
                        const float* dk, float* ev, TO* out, int* err, cudaEvent_t* ev2) {
  if (kind == 0) return run_tc<DIM, K, tc::KIND_TF32, TO>(P, s, rec, tau, dk, ev, out, err, ev2);
  return run_tc<DIM, K, tc::KIND_BF16, TO>(P, s, rec, tau, dk, ev, out, err, ev2);
}

}  // namespace

unsigned set_tc_wait_polls(unsigned polls) { return g_wait_polls.exchange(polls, std::memory_order_relaxed); }

bool jvp_tc_supported(int dim, int k) { return (dim == 2 && k >= 1 && k <= 4) || (dim == 3 && k >= 1 && k <= 2); }

template <class TO>
cudaError_t launch_jvp_tc(const ElemParams& P, cudaStream_t s, int kind, const float* rec, double tau,
                          const float* dk, float* ev, TO* out, int* err, cudaEvent_t* ev2) {
  switch (P.dim * 10 + P.K) {
    case 21: return run_tc_kind<2, 1, TO>(P, s, kind, rec, tau, dk, ev, out, err, ev2);
    case 22: return run_tc_kind<2, 2, TO>(P, s, kind, rec, tau, dk, ev, out, err, ev2);
    case 23: return run_tc_kind<2, 3, TO>(P, s, kind, rec, tau, dk, ev, out, err, ev2);
    case 24: return run_tc_kind<2, 4, TO>(P, s, kind, rec, tau, dk, ev, out, err, ev2);
    case 31: return run_tc_kind<3, 1, TO>(P, s, kind, rec, tau, dk, ev, out, err, ev2);
    case 32: return run_tc_kind<3, 2, TO>(P, s, kind, rec, tau, dk, ev, out, err, ev2);
    default: return cudaErrorNotSupported;
  }
}

template cudaError_t launch_jvp_tc<float>(const ElemParams&, cudaStream_t, int, const float*, double, const float*,
                                          float*, float*, int*, cudaEvent_t*);
template cudaError_t launch_jvp_tc<double>(const ElemParams&, cudaStream_t, int, const float*, double,
                                           const float*, float*, double*, int*, cudaEvent_t*);

}  // namespace lh
