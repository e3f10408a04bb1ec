// Common device helpers: element configuration, forward-mode dual numbers.
#pragma once
#include <cuda_runtime.h>
#include <cmath>

namespace lh {

// Element configuration for dimension DIM and H1 order K (paper Sec. 2.1: Q_K for x, v
// and discontinuous Q_{K-1} for e), Gauss quadrature with 2K points per direction.
template <int DIM, int K>
struct Cfg {
  static constexpr int D = K + 1;                 // H1 1D dofs
  static constexpr int L = K;                     // L2 1D dofs
  static constexpr int Q = 2 * K;                 // 1D quadrature points
  static constexpr int ND = DIM == 2 ? D * D : D * D * D;
  static constexpr int NL = DIM == 2 ? L * L : L * L * L;
  static constexpr int NQ = DIM == 2 ? Q * Q : Q * Q * Q;
  // elements per thread block: one thread per quadrature point, >= 128 threads
  static constexpr int EPB = NQ >= 128 ? 1 : 128 / NQ;
  static constexpr int THREADS = EPB * NQ;
};

// ---------------------------------------------------------------------------------------
// Forward-mode dual number: value and one directional derivative.  The tangent kernels
// run the same quadrature-point code on Dual<T> that the residual runs on T, so the
// derivative is that of the exact discrete residual (paper Sec. 3.1, Eq. (10)).
template <class T>
struct Dual {
  T v, d;
  __host__ __device__ __forceinline__ Dual() {}
  __host__ __device__ __forceinline__ Dual(T a) : v(a), d(T(0)) {}
  __host__ __device__ __forceinline__ Dual(T a, T b) : v(a), d(b) {}
};

template <class T> __host__ __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T> __host__ __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator+(T a, Dual<T> b) { return {a + b.v, b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return {a.v - b, a.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return {a - b.v, -b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator/(Dual<T> a, T b) { return {a.v / b, a.d / b}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator/(T a, Dual<T> b) {
  T q = a / b.v;
  return {q, -q * b.d / b.v};
}
template <class T> __host__ __device__ __forceinline__ Dual<T>& operator+=(Dual<T>& a, Dual<T> b) { a.v += b.v; a.d += b.d; return a; }

// scalar math, overloaded for T and Dual<T>
__host__ __device__ __forceinline__ double lsqrt(double a) { return ::sqrt(a); }
__host__ __device__ __forceinline__ float lsqrt(float a) { return ::sqrtf(a); }
__host__ __device__ __forceinline__ double ltanh(double a) { return ::tanh(a); }
__host__ __device__ __forceinline__ float ltanh(float a) { return ::tanhf(a); }
__host__ __device__ __forceinline__ double lcbrt(double a) { return ::cbrt(a); }
__host__ __device__ __forceinline__ float lcbrt(float a) { return ::cbrtf(a); }
__host__ __device__ __forceinline__ double lcos(double a) { return ::cos(a); }
__host__ __device__ __forceinline__ float lcos(float a) { return ::cosf(a); }
__host__ __device__ __forceinline__ double lsin(double a) { return ::sin(a); }
__host__ __device__ __forceinline__ float lsin(float a) { return ::sinf(a); }

template <class T> __host__ __device__ __forceinline__ Dual<T> lsqrt(Dual<T> a) {
  T s = lsqrt(a.v);
  return {s, a.d * (T(0.5) / s)};
}
template <class T> __host__ __device__ __forceinline__ Dual<T> ltanh(Dual<T> a) {
  T t = ltanh(a.v);
  return {t, a.d * (T(1) - t * t)};
}
template <class T> __host__ __device__ __forceinline__ Dual<T> lcbrt(Dual<T> a) {
  T c = lcbrt(a.v);
  return {c, a.d * c / (T(3) * a.v)};
}
template <class T> __host__ __device__ __forceinline__ Dual<T> lcos(Dual<T> a) { return {lcos(a.v), -lsin(a.v) * a.d}; }

// x^(1/DIM) for the volume-scaled length of Eq. (14)
template <int DIM, class S> __host__ __device__ __forceinline__ S root_dim(S x) {
  if constexpr (DIM == 2) return lsqrt(x); else return lcbrt(x);
}

template <class T> __host__ __device__ __forceinline__ T value_of(T a) { return a; }
template <class T> __host__ __device__ __forceinline__ T value_of(Dual<T> a) { return a.v; }

// ---------------------------------------------------------------------------------------
// Double-float arithmetic for the FP64 residual's element contractions: a value is an
// unevaluated sum hi + lo of two floats (about 48 significant bits), built from the
// error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971)
// and TwoProduct through a fused multiply-add.  Each multiply-add costs about fifteen FP32
// instructions, which on this GPU's FP32 pipe is several times cheaper than one FP64 FMA on
// its FP64 pipe; relative error per operation about 2^-46.
struct DFProd {   // a product hi * hi' with its rounding error and the cross terms, not normalised
  float p, e;
};
struct DF {
  float hi, lo;
  __device__ __forceinline__ DF() {}
  __device__ __forceinline__ DF(int a) : hi((float)a), lo(0.f) {}
  __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit DF(double a) {
    hi = (float)a;
    lo = (float)(a - (double)hi);
  }
};
__device__ __forceinline__ double to_double(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return DF(s, b - (s - a));
}
__device__ __forceinline__ DFProd operator*(DF a, DF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);           // exact error of the leading product
  return DFProd{p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e))};
}
__device__ __forceinline__ DF operator+(DFProd a, DFProd b) {
  float s, t;
  two_sum(a.p, b.p, s, t);
  return fast_two_sum(s, t + (a.e + b.e));
}
__device__ __forceinline__ DF& operator+=(DF& acc, DFProd a) {
  float s, t;
  two_sum(acc.hi, a.p, s, t);
  acc = fast_two_sum(s, t + (acc.lo + a.e));
  return acc;
}
__device__ __forceinline__ DF& operator+=(DF& acc, DF a) {
  float s, t;
  two_sum(acc.hi, a.hi, s, t);
  acc = fast_two_sum(s, t + (acc.lo + a.lo));
  return acc;
}

}  // namespace lh
