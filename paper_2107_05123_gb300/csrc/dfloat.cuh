// Double-float arithmetic for the element kernels of the FP64 refinement loop.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, giving
// about 48 significant bits (Dekker 1971; the double-double algorithms of Hida, Li and Bailey,
// 2001, with float components). GB300 issues FP64 instructions at a small fraction of its FP32
// rate, so the element kernels whose FP64 arithmetic bounds them (right-hand sides, residuals)
// compute in this type: about ten to twenty FP32 instructions per FP64 operation, each pipelined
// at the full FP32 rate. Values are loaded from and stored to FP64 arrays.
//
// Building blocks: two_sum (exact sum of two floats as s + e), quick_two_sum (the same when
// |a| >= |b|), two_prod (exact product by one FMA); the accurate addition renormalises after
// adding both components, so that cancellation keeps the relative accuracy of the result.
// Division and the reciprocal square root refine the FP32 hardware estimate by one Newton step
// carried out in double-float.
#pragma once

#include <cuda_runtime.h>

namespace chns {

struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
  // from a double: the nearest float and the float nearest to the remainder
  __host__ __device__ explicit DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit DF(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ explicit DF(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return DF(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ DF df_quick_two_sum(float a, float b) {
  const float s = a + b;
  return DF(s, b - (s - a));
}
__device__ __forceinline__ DF operator+(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  const DF t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df_quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}
// 1/b: r = 1/b.hi in FP32, then r + r (1 - b r) in double-float
__device__ __forceinline__ DF df_recip(DF b) {
  const float r = 1.0f / b.hi;
  const DF rr(r, 0.0f);
  const DF e = DF(1.0f) - b * rr;
  return rr + rr * e;
}
__device__ __forceinline__ DF operator/(DF a, DF b) { return a * df_recip(b); }
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }
__device__ __forceinline__ DF& operator*=(DF& a, DF b) { return a = a * b; }
__device__ __forceinline__ bool operator<(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(DF a, DF b) { return b < a; }
__device__ __forceinline__ bool operator<=(DF a, DF b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(DF a, DF b) { return !(a < b); }
__device__ __forceinline__ bool operator==(DF a, DF b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(DF a, DF b) { return !(a == b); }
// 1/sqrt(x) for x > 0: y = rsqrt(x.hi) in FP32, then y + y (1 - x y^2) / 2 in double-float
// (beside the float and double overloads, which the templated kernels call by the same name)
using ::rsqrt;
__device__ __forceinline__ DF rsqrt(DF x) {
  const float y = rsqrtf(x.hi);
  const DF yy(y, 0.0f);
  const DF e = DF(1.0f) - x * (yy * yy);
  return yy + yy * (e * DF(0.5f));
}

}  // namespace chns
