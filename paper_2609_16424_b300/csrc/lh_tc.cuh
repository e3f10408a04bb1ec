// 5th-generation tensor-core helpers (tcgen05, sm_100a-family, here sm_103a): tensor-memory
// allocation, shared-memory matrix descriptors, single-thread MMA issue and commit,
// mbarrier waits with an iteration limit, tensor-memory loads.  Inline PTX only.
//
// Operand layouts are K-major (each row of A [M x K] and of B [N x K] holds its K entries),
// D[m][n] = sum_k A[m][k] B[n][k], accumulated in FP32 in tensor memory: row m of a
// M = 128 tile is TMEM lane m, column n is TMEM column (base + n).
//
// Two shared-memory layouts are used:
//   interleaved (no swizzle): 8-row x 16-byte core matrices stored as 128 contiguous bytes;
//     the core matrix of row group g and K group j starts at g*SBO + j*LBO.
//   128-byte swizzle: 8-row x 128-byte atoms (1024 bytes, 1024-byte aligned); row r of an
//     atom at r*128; its 16-byte chunk c stored at chunk position c ^ r.  Atoms of
//     consecutive row groups are SBO apart; an MMA step selects its 32-byte K slice by
//     adding the slice offset to the start address.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace lh {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- shared-memory matrix descriptor (64 bit)
//   [0,14) start address >> 4, [16,30) leading byte offset >> 4, [32,46) stride byte
//   offset >> 4, [46,48) descriptor version 1, [49,52) base offset 0, [52] relative LBO,
//   [61,64) swizzle: 0 none, 2 128-byte.
enum Swizzle : uint32_t { SW_NONE = 0, SW_128 = 2 };

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, Swizzle sw) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)sw << 61;
  return d;
}

// ---- instruction descriptor for kind::tf32 / kind::f16 with FP32 accumulation, both
// operands K-major: [4,6) D format (1 = F32), [7,10) A format, [10,13) B format
// (kind::f16: 1 = BF16; kind::tf32: 2 = TF32), [15] A MN-major, [16] B MN-major,
// [17,23) N >> 3, [24,29) M >> 4.
enum Kind : int { KIND_TF32 = 0, KIND_BF16 = 1 };

__host__ __device__ constexpr uint32_t instr_desc(Kind kind, int M, int N) {
  const uint32_t ab = kind == KIND_TF32 ? 2u : 1u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// K entries consumed by one MMA instruction (32 bytes of each operand row)
__host__ __device__ constexpr int mma_k(Kind kind) { return kind == KIND_TF32 ? 8 : 16; }
__host__ __device__ constexpr int elem_bytes(Kind kind) { return kind == KIND_TF32 ? 4 : 2; }

// ---- tensor memory allocation (one full warp executes alloc / dealloc)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               :: "r"(smem_u32(dst_smem)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

// ---- ordering between thread barriers and tensor-core operations
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- MMA issue (a single thread), D (+)= A B^T
template <Kind KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool accum) {
  const uint32_t acc = accum ? 1u : 0u;
  if constexpr (KIND == KIND_TF32) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc) : "memory");
  } else {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc) : "memory");
  }
}

// arrive on the mbarrier once all previously issued MMAs of this thread have completed
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}

// ---- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also announces `bytes` of asynchronous copies completing on this phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
// bulk copy global -> this CTA's shared memory (both 16-byte aligned, bytes a multiple of
// 16), completing `bytes` on mbar's current phase
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}
// wait for completion of the phase with the given parity; gives up after max_iter polls
// or about 2^31 SM clock cycles (~1 s), whichever comes first, and returns false (the
// caller records the failure and poisons dependent results)
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_iter) {
  const uint32_t a = smem_u32(mbar);
  const long long t0 = clock64();
  for (uint32_t it = 0; it < max_iter && clock64() - t0 < (1ll << 31); ++it) {
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

// ---- tensor memory -> registers: warp w reads lanes [32 (w % 4), 32 (w % 4) + 32);
// thread i gets lane 32 (w % 4) + i, registers = N consecutive columns from taddr's column
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
               "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- operand element conversion (round to nearest)
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// ---- layout offsets (bytes)
// interleaved: row m, K index k, T = 16 / esz entries per core row
__host__ __device__ __forceinline__ uint32_t off_il(int m, int k, int esz, uint32_t lbo, uint32_t sbo) {
  const int T = 16 / esz;
  return (uint32_t)(m >> 3) * sbo + (uint32_t)(k / T) * lbo + (uint32_t)(m & 7) * 16u + (uint32_t)(k % T) * esz;
}
// 128-byte swizzle: K atoms of 128 bytes; atom a of row group g at a * astride + g * 1024
__host__ __device__ __forceinline__ uint32_t off_sw128(int m, int k, int esz, uint32_t astride) {
  const int per_atom = 128 / esz, T = 16 / esz;
  const int a = k / per_atom, kk = k % per_atom;
  const int chunk = kk / T, r = m & 7;
  return (uint32_t)a * astride + (uint32_t)(m >> 3) * 1024u + (uint32_t)r * 128u +
         (uint32_t)(chunk ^ r) * 16u + (uint32_t)(kk % T) * esz;
}

}  // namespace tc
}  // namespace lh
