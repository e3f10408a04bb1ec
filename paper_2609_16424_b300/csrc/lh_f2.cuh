// Paired FP32 arithmetic (the f32x2 add, multiply and fused multiply-add of sm_100 and
// later: two independent float operations per instruction, each rounded exactly as the
// scalar operation).  The element kernels that give each thread two quadrature points use
// it for every per-point operation, so one instruction serves both points.
#pragma once
#include <cuda_runtime.h>

namespace lh {

__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

}  // namespace lh
