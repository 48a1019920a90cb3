// Double-float arithmetic on the FP32 pipe (sm_103a).
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2,
// a 48-bit significand in FP32's exponent range (Dekker 1971, "A floating-point
// technique for extending the available precision"; the error-free sum is Knuth's
// TwoSum, the error-free product uses the fused multiply-add).  B300 issues FP64 at
// 1/64 of the FP32 rate, so an amplitude evaluated in pairs of FP32 numbers, at
// 7 to 15 FP32 operations per FP64 one, runs faster than the same code in FP64 at a
// unit roundoff of about 2^-48 instead of 2^-53.
//
// Every FP32 operation is a round-to-nearest intrinsic, which the compiler never
// contracts or reassociates: the error-free transformations depend on each
// operation rounding exactly once.
//   sum      TwoSum of the high parts, the low parts added to its error, then a
//            renormalisation (FastTwoSum): 10 operations.  The error bound is
//            relative to |a| + |b| (Dekker's sum), which the amplitude code's
//            cancellations keep within its 1e-12 tolerance (measured against an
//            extended-precision evaluation).
//   product  TwoProduct of the high parts with one FMA, the cross terms folded in
//            with two more, then FastTwoSum: 7 operations.
//   fma      the exact product of the high parts enters TwoSum with c: 15.
//   divide   two FP32 quotient digits with a double-float remainder.
//   sqrt     one Newton correction of the FP32 square root.
#pragma once
#include <cuda_runtime.h>

namespace rex {

// the FP32 and FP64 overloads stay visible beside the double-float ones below
using ::fma;
using ::rsqrt;
using ::sqrt;

struct df64 {
  float hi, lo;
  df64() = default;   // trivial: shared-memory arrays of it need no constructor
  __device__ __forceinline__ df64(int i) : hi((float)i), lo(0.f) {}
  __device__ __forceinline__ df64(float f) : hi(f), lo(0.f) {}
  __device__ __forceinline__ df64(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df64_make(float hi, float lo) {
  df64 r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// FastTwoSum (|a| >= |b| or a == 0): a + b = s + e exactly
__device__ __forceinline__ df64 df64_renorm(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df64_renorm(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64_make(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df64_renorm(p, e);
}
// a * b + c with the product's high part exact
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  const float s = __fadd_rn(p, c.hi);
  const float bb = __fsub_rn(s, p);
  float e = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df64_renorm(s, e);
}
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df64 r = a - b * df64(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return df64_renorm(q1, q2);
}
__device__ __forceinline__ df64 sqrt(df64 a) {
  if (!(a.hi > 0.f)) return df64_make(a.hi == 0.f ? 0.f : __fsqrt_rn(a.hi), 0.f);   // 0, or NaN below 0
  const float x = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(x, x);
  const float pe = __fmaf_rn(x, x, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);   // a - x^2, to first order
  return df64_renorm(x, __fdiv_rn(r, __fmul_rn(2.f, x)));
}
__device__ __forceinline__ df64 rsqrt(df64 a) { return df64(1) / sqrt(a); }

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

__device__ __forceinline__ bool operator>(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return b > a; }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(a > b); }

// lane exchange of a warp (both parts)
__device__ __forceinline__ df64 shfl_xor(df64 v, int off) {
  return df64_make(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

}  // namespace rex
