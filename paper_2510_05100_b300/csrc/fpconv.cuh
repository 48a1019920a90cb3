// FP64 <-> FP32 conversions on the integer ALUs (IEEE-754 bit fields).  B300
// issues FP64 instructions, conversions included, at 1/64 of the FP32 rate, so the
// mixed-precision kernels convert their momenta and weights here instead.
#pragma once
#include <cuda_runtime.h>

namespace rex {

// FP64 -> FP32 on integer ALUs (selects, no branches): round to nearest even;
// magnitudes below the FP32 normal range become a signed zero, above it infinity;
// NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_alu(double x) {
  const unsigned long long d = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(d >> 32), lo = (unsigned)d;
  const unsigned sign = hi & 0x80000000u, ahi = hi & 0x7fffffffu;
  // rebias the exponent by 1023 - 127 = 896 and keep 23 mantissa bits
  unsigned f = ((ahi - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;   // the 29 dropped mantissa bits
  f += (rem > 0x10000000u) | ((rem == 0x10000000u) & f);
  const unsigned big = (ahi > 0x7ff00000u || (ahi == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : 0x7f800000u;
  f = ahi < (897u << 20) ? 0u : f;         // |x| < 2^-126
  f = ahi >= (1151u << 20) ? big : f;      // |x| >= 2^128, infinity or NaN
  return __uint_as_float(f | sign);
}

// FP32 -> FP64 on integer ALUs (selects): exact for normal numbers, zeros,
// infinities and NaN (FP32 subnormals, which the conversion above never
// produces, become zero).
__device__ __forceinline__ double f32_to_f64_alu(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u, a = b & 0x7fffffffu;
  const bool small = a < 0x00800000u, special = a >= 0x7f800000u;
  unsigned hi = (a >> 3) + (896u << 20);
  hi = special ? (0x7ff00000u | ((a & 0x7fffffu) >> 3)) : hi;
  hi = small ? 0u : hi;
  const unsigned lo = small ? 0u : a << 29;
  return __hiloint2double((int)(hi | sign), (int)lo);
}

// FP64 -> FP32 on integer ALUs for finite inputs, rounding to nearest even
// (magnitudes below 2^-126 give a signed zero); the caller checks finiteness
// once per event with the largest |x|'s high word, ahi_max (>= 1151 << 20:
// infinite, NaN or beyond the FP32 range).
__device__ __forceinline__ float f64_to_f32_alu_finite(double x, unsigned& ahi_max) {
  const unsigned long long d = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(d >> 32), lo = (unsigned)d;
  const unsigned ahi = hi & 0x7fffffffu;
  ahi_max = max(ahi_max, ahi);
  unsigned f = __funnelshift_l(lo, ahi - (896u << 20), 3);
  // round half to even on the 29 dropped bits: up if bit 28 is set and (bits 0..27
  // are not all zero or the kept value is odd)
  f += (lo >> 28) & 1u & ((lo & 0x0fffffffu) != 0u | f);
  f = ahi < (897u << 20) ? 0u : f;
  return __uint_as_float(f | (hi & 0x80000000u));
}

}  // namespace rex
