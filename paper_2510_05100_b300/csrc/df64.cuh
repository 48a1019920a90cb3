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

#include "helas.cuh"

namespace rex {

// the FP32 and FP64 overloads stay visible beside the double-float ones below
using ::abs;
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

template <>
struct expensive_arith<df64> {
  static constexpr bool value = true;
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
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }

// out += sum of three products, each product's high part exact and added with one
// TwoSum, the low parts gathered in c, one renormalisation at the end (12 operations
// per product instead of the 15 of a double-float FMA)
__device__ __forceinline__ void df64_acc_term(float& s, float& c, df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  const float t = __fadd_rn(s, p);
  const float bb = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, pe));
  c = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, c));
}
__device__ __forceinline__ df64 df64_acc3(df64 out, df64 a1, df64 b1, df64 a2, df64 b2, df64 a3, df64 b3) {
  float s = out.hi, c = out.lo;
  df64_acc_term(s, c, a3, b3);
  df64_acc_term(s, c, a2, b2);
  df64_acc_term(s, c, a1, b1);
  return df64_renorm(s, c);
}

// slash_acc of helas.cuh for double-float values: out += s (gamma . a) psi, where s is
// +1 or -1 (its only values in the amplitude code) and enters as a sign, each output
// component accumulated with df64_acc3
__device__ __forceinline__ void slash_acc(df64 s, const df64* a, const cx<df64>* psi, cx<df64>* out) {
  const bool neg = s.hi < 0.f;
  df64 am = a[0] - a[3], ap = a[0] + a[3], a1 = a[1], a2 = a[2];
  if (neg) {
    am = -am;
    ap = -ap;
    a1 = -a1;
    a2 = -a2;
  }
  out[0].re = df64_acc3(out[0].re, am, psi[2].re, -a1, psi[3].re, -a2, psi[3].im);
  out[0].im = df64_acc3(out[0].im, am, psi[2].im, -a1, psi[3].im, a2, psi[3].re);
  out[1].re = df64_acc3(out[1].re, ap, psi[3].re, -a1, psi[2].re, a2, psi[2].im);
  out[1].im = df64_acc3(out[1].im, ap, psi[3].im, -a1, psi[2].im, -a2, psi[2].re);
  out[2].re = df64_acc3(out[2].re, ap, psi[0].re, a1, psi[1].re, a2, psi[1].im);
  out[2].im = df64_acc3(out[2].im, ap, psi[0].im, a1, psi[1].im, -a2, psi[1].re);
  out[3].re = df64_acc3(out[3].re, am, psi[1].re, a1, psi[0].re, -a2, psi[0].im);
  out[3].im = df64_acc3(out[3].im, am, psi[1].im, a1, psi[0].im, a2, psi[0].re);
}

// exact scaling by 2
__device__ __forceinline__ df64 df64_twice(df64 a) { return df64_make(__fmul_rn(2.f, a.hi), __fmul_rn(2.f, a.lo)); }

// sum of N products from zero, each added with one TwoSum, one renormalisation
template <int N>
__device__ __forceinline__ df64 df64_dot(const df64 (&a)[N], const df64 (&b)[N]) {
  float s = 0.f, c = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) df64_acc_term(s, c, a[i], b[i]);
  return df64_renorm(s, c);
}

// the Minkowski product of helas.cuh (mdot) for double-float vectors
__device__ __forceinline__ df64 df64_mdot(const df64* a, const df64* b) {
  const df64 x[4] = {a[0], -a[1], -a[2], -a[3]}, y[4] = {b[0], b[1], b[2], b[3]};
  return df64_dot(x, y);
}

// ubar_dot of helas.cuh: conj(u_L) . x_R + conj(u_R) . x_L, real and imaginary parts
// each one eight-product sum
__device__ __forceinline__ cx<df64> ubar_dot(const cx<df64>* u, const cx<df64>* x) {
  const cx<df64> b0 = x[2], b1 = x[3], b2 = x[0], b3 = x[1];
  const df64 ar[8] = {u[0].re, u[0].im, u[1].re, u[1].im, u[2].re, u[2].im, u[3].re, u[3].im};
  const df64 br[8] = {b0.re, b0.im, b1.re, b1.im, b2.re, b2.im, b3.re, b3.im};
  const df64 ai[8] = {u[0].re, -u[0].im, u[1].re, -u[1].im, u[2].re, -u[2].im, u[3].re, -u[3].im};
  const df64 bi[8] = {b0.im, b0.re, b1.im, b1.re, b2.im, b2.re, b3.im, b3.re};
  return cx<df64>{df64_dot(ar, br), df64_dot(ai, bi)};
}

// Minkowski product of complex 4-vectors without conjugation (cdotm of the q q~ g
// amplitudes): real and imaginary parts each one eight-product sum
__device__ __forceinline__ cx<df64> cdotm(const cx<df64>* a, const cx<df64>* b) {
  const df64 ar[8] = {a[0].re, -a[0].im, -a[1].re, a[1].im, -a[2].re, a[2].im, -a[3].re, a[3].im};
  const df64 br[8] = {b[0].re, b[0].im, b[1].re, b[1].im, b[2].re, b[2].im, b[3].re, b[3].im};
  const df64 ai[8] = {a[0].re, a[0].im, -a[1].re, -a[1].im, -a[2].re, -a[2].im, -a[3].re, -a[3].im};
  const df64 bi[8] = {b[0].im, b[0].re, b[1].im, b[1].re, b[2].im, b[2].re, b[3].im, b[3].re};
  return cx<df64>{df64_dot(ar, br), df64_dot(ai, bi)};
}

// vvv_acc of helas.cuh (s = +-1 as a sign):
// out += s [ (X.Y)(PY - PX) - (X.(PX + 2 PY)) Y + (Y.(2 PX + PY)) X ]
__device__ __forceinline__ void vvv_acc(df64 s, const df64* jx, const df64* px, const df64* jy, const df64* py,
                                        df64* out) {
  df64 a[4], b[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    a[m] = px[m] + df64_twice(py[m]);
    b[m] = df64_twice(px[m]) + py[m];
  }
  df64 xy = df64_mdot(jx, jy), xa = df64_mdot(jx, a), yb = df64_mdot(jy, b);
  if (s.hi < 0.f) {
    xy = -xy;
    xa = -xa;
    yb = -yb;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) out[m] = df64_acc3(out[m], xy, py[m] - px[m], -xa, jy[m], yb, jx[m]);
}

// vvvv_acc of helas.cuh (s = +-1 as a sign): out += s [ (X.Y) Z + (Y.Z) X - 2 (X.Z) Y ]
__device__ __forceinline__ void vvvv_acc(df64 s, const df64* jx, const df64* jy, const df64* jz, df64* out) {
  df64 xy = df64_mdot(jx, jy), yz = df64_mdot(jy, jz), xz2 = -df64_twice(df64_mdot(jx, jz));
  if (s.hi < 0.f) {
    xy = -xy;
    yz = -yz;
    xz2 = -xz2;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) out[m] = df64_acc3(out[m], xy, jz[m], yz, jx[m], xz2, jy[m]);
}

__device__ __forceinline__ df64 abs(df64 a) { return a.hi < 0.f ? -a : a; }

// lane exchange of a warp: any shuffled type, and double-float values in both parts
template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int off) {
  return __shfl_xor_sync(0xffffffffu, v, off);
}
__device__ __forceinline__ df64 shfl_xor(df64 v, int off) {
  return df64_make(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

}  // namespace rex
