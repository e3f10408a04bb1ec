// Double-word ("double-float") arithmetic for the FP64-accurate quadrature-point kernel of
// the residual, run on the FP32 pipe (B300's FP64 rate is about 1/61 of its FP32 rate).
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2 (about 48
// significant bits; FP64 has 53).  Building blocks, all published error-free
// transformations or their standard compositions:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971), TwoProd by one fused
//   multiply-add; the double-word sum, product and quotient of Joldes, Muller and Popescu,
//   "Tight and rigorous error bounds for basic building blocks of double-word arithmetic",
//   ACM TOMS 44 (2017) (sum with both words, relative error <= 3u^2; product <= 5u^2;
//   quotient by one correction of the float quotient);
//   square root and cube root by one Newton step from the float root (Karp and Markstein
//   1997 for the square root);
//   exp by range reduction x = n ln 2 + r (ln 2 in three floats) and the Taylor polynomial
//   of degree 12 on |r| <= ln(2)/2 (truncation below 2^-48), then exact scaling by 2^n;
//   tanh(z) = sign(z) (1 - E) / (1 + E), E = exp(-2 |z|).
// u = 2^-24.  Host and device: the host instantiation checks it against double math.
#pragma once
#include <cmath>
#include <cuda_runtime.h>
#include "lh_common.cuh"

namespace lh {

struct DD {
  float hi, lo;
  __host__ __device__ __forceinline__ DD() {}
  __host__ __device__ __forceinline__ constexpr DD(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ constexpr DD(float a) : hi(a), lo(0.f) {}
  __host__ __device__ __forceinline__ constexpr DD(int a) : hi((float)a), lo(0.f) {}
  // exact split of a double (only for constants and set-up: uses FP64 conversions)
  __host__ __device__ __forceinline__ constexpr DD(double a) : hi((float)a), lo((float)(a - (double)(float)a)) {}
};

__host__ __device__ __forceinline__ double to_double(const DD& a) { return (double)a.hi + (double)a.lo; }

namespace dd {
__host__ __device__ __forceinline__ float fma_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
__host__ __device__ __forceinline__ DD two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  return DD(s, (a - (s - v)) + (b - v));
}
__host__ __device__ __forceinline__ DD fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = a + b;
  return DD(s, b - (s - a));
}
__host__ __device__ __forceinline__ DD two_prod(float a, float b) {
  const float p = a * b;
  return DD(p, fma_(a, b, -p));
}
}  // namespace dd

__host__ __device__ __forceinline__ DD operator+(const DD& x, const DD& y) {
  const DD s = dd::two_sum(x.hi, y.hi);
  const DD t = dd::two_sum(x.lo, y.lo);
  const DD v = dd::fast_two_sum(s.hi, s.lo + t.hi);
  return dd::fast_two_sum(v.hi, t.lo + v.lo);
}
__host__ __device__ __forceinline__ DD operator-(const DD& x) { return DD(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ DD operator-(const DD& x, const DD& y) { return x + (-y); }
__host__ __device__ __forceinline__ DD operator*(const DD& x, const DD& y) {
  const DD c = dd::two_prod(x.hi, y.hi);
  const float t = dd::fma_(x.lo, y.hi, x.hi * y.lo);
  return dd::fast_two_sum(c.hi, c.lo + t);
}
__host__ __device__ __forceinline__ DD operator/(const DD& x, const DD& y) {
  const float q = x.hi / y.hi;                    // float quotient
  const DD r = x - y * DD(q);                     // remainder in double-word
  const float c = r.hi / y.hi;                    // its float correction
  return dd::fast_two_sum(q, c);
}
__host__ __device__ __forceinline__ DD& operator+=(DD& a, const DD& b) { return a = a + b; }
__host__ __device__ __forceinline__ bool operator<(const DD& a, const DD& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__host__ __device__ __forceinline__ bool operator>=(const DD& a, const DD& b) { return !(a < b); }

// square root: s = sqrt(hi) in float, then s + (x - s^2) / (2 s)
__host__ __device__ __forceinline__ DD lsqrt(const DD& x) {
  if (!(x.hi > 0.f)) return DD(0.f);
  const float s = sqrtf(x.hi);
  const DD e = x - dd::two_prod(s, s);
  return dd::fast_two_sum(s, e.hi / (2.f * s));
}

// cube root of x > 0: y = cbrt(hi) in float, then y + (x - y^3) / (3 y^2)
__host__ __device__ __forceinline__ DD lcbrt(const DD& x) {
  if (!(x.hi > 0.f)) return DD(0.f);
  const float y = cbrtf(x.hi);
  const DD y2 = dd::two_prod(y, y);
  const DD e = x - y2 * DD(y);
  return dd::fast_two_sum(y, e.hi / (3.f * y2.hi));
}

// exp(x) for x <= 0 (the only use here), down to the float range; 0 below
__host__ __device__ __forceinline__ DD exp_nonpos(const DD& x) {
  if (x.hi < -87.f) return DD(0.f);
  constexpr double L2 = 0.6931471805599453094;                 // ln 2 to double precision
  constexpr float L2a = (float)L2;
  constexpr float L2b = (float)(L2 - (double)L2a);
  constexpr float L2c = (float)(L2 - (double)L2a - (double)L2b);
  const float n = rintf(x.hi * 1.4426950408889634f);          // nearest integer to x / ln 2
  // r = x - n ln 2 exactly in the first two words (n, the L2 words have few significant bits
  // in their products, so each product is exact or carried by TwoProd)
  DD r = x - dd::two_prod(n, L2a);
  r = r - dd::two_prod(n, L2b);
  r = r - DD(n * L2c);
  // Taylor polynomial sum_{j<=12} r^j / j!, Horner in double-word
  constexpr double f[13] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320,
                            1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600};
  DD p = DD(f[12]);
#pragma unroll
  for (int j = 11; j >= 0; --j) p = p * r + DD(f[j]);
  const int ni = (int)n;
#ifdef __CUDA_ARCH__
  return DD(ldexpf(p.hi, ni), ldexpf(p.lo, ni));
#else
  return DD(std::ldexp(p.hi, ni), std::ldexp(p.lo, ni));
#endif
}

__host__ __device__ __forceinline__ DD ltanh(const DD& z) {
  const bool neg = z.hi < 0.f;
  const DD a = neg ? -z : z;
  const DD E = exp_nonpos(DD(-2.f) * a);
  const DD t = (DD(1.f) - E) / (DD(1.f) + E);
  return neg ? -t : t;
}

__host__ __device__ __forceinline__ DD value_of(const DD& a) { return a; }

// the contraction type DF (lh_common.cuh) holds the same (hi, lo) pair
__host__ __device__ __forceinline__ DD dd_of(const DF& a) { return DD(a.hi, a.lo); }
__device__ __forceinline__ DF df_of(const DD& a) { return DF(a.hi, a.lo); }

}  // namespace lh
