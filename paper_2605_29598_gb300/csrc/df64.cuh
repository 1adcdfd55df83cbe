// FP64-class arithmetic on the FP32 pipe: a value is the unevaluated sum of
// two FP32 numbers, hi + lo with |lo| <= ulp(hi) / 2 ("double-float",
// about 48 significant bits, FP32's exponent range).  GB300 issues FP32 at
// about 60 times its FP64 rate, so the cell kernels of the Schur vmult,
// which the FP64 pipe binds, run faster in this form at about 1e-14
// relative accuracy per operation (not IEEE FP64: the DG_PAIRS precision
// mode of the library).
//
// The operations are the classical error-free transformations:
//  - TwoSum (Knuth): s = a + b, e = (a - (s - v)) + (b - v), v = s - a, so
//    that s + e = a + b exactly;
//  - TwoProduct with a fused multiply-add (Dekker's product without
//    splitting): p = a b, e = fma(a, b, -p) = a b - p exactly;
//  - Fast2Sum renormalisation (|s| >= |e|): hi = s + e, lo = e - (hi - s);
// and the quotient by one Newton-type correction of the FP32 quotient.
#pragma once

#include <cuda_runtime.h>

namespace dg {

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_renorm(float s, float e) {
  const float h = s + e;
  return df64(h, e - (h - s));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  const float e = (a.hi - (s - v)) + (b.hi - v);
  return df_renorm(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_renorm(p, e);
}
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float q1 = a.hi / b.hi;
  const df64 r = a - b * df64(q1, 0.0f);
  const float q2 = r.hi / b.hi;
  return df_renorm(q1, q2);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
// (the other types keep the CUDA math overloads)
using ::fabs;
using ::fmax;
__device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f) ? -a : a; }
__device__ __forceinline__ df64 fmax(df64 a, df64 b) { return a < b ? b : a; }
// read-only load of a pair (the other types keep CUDA's __ldg)
using ::__ldg;
__device__ __forceinline__ df64 __ldg(const df64* p) {
  const float2 v = ::__ldg(reinterpret_cast<const float2*>(p));
  return df64(v.x, v.y);
}

}  // namespace dg
