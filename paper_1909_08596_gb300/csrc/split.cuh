// Conversions between FP64 and the split-BF16 operand form that avoid the FP64 pipe.
//
// GB300 issues FP64 arithmetic at 1/64 of its FP32 rate, so the operand splitting works on
// an unevaluated two-float form (hi + lo) of each value:
//  * d2ff: a double becomes hi = its 24 leading significant bits (exact truncation, by
//    reassembling the bit fields) and lo = the remaining bits rounded to FP32 (an integer to
//    float conversion and an exact power-of-two scaling), ~48 bits together;
//  * split3f: hi + lo becomes three bf16 slices x0 + x1 + x2, each the round-to-nearest bf16
//    of what the previous slices left (hi - x0 is exact by Sterbenz's lemma), so the slices
//    carry the value to ~2^-26 relative;
//  * f2d: a float widened to double exactly by reassembling the bit fields.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace dmet {

__device__ __forceinline__ float2 d2ff(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long mant = b & ((1ull << 52) - 1);
  if (e == 0x7ff) {  // inf or nan
    return make_float2(__uint_as_float(sign | 0x7f800000u | (mant ? 0x400000u : 0u)), 0.f);
  }
  const int E = e - 1023;
  if (e == 0 || E < -126) return make_float2(__uint_as_float(sign), 0.f);  // below FP32's normal range
  if (E > 127) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const float hi = __uint_as_float(sign | ((unsigned int)(E + 127) << 23) | (unsigned int)(mant >> 29));
  const unsigned int rem = (unsigned int)(mant & ((1u << 29) - 1));
  // rem * 2^(E - 52); the scale is built from its exponent field while it stays normal.
  float lo = (float)rem;
  const int es = E - 52;
  lo = es >= -126 ? lo * __uint_as_float((unsigned int)(es + 127) << 23) : ldexpf(lo, es);
  return make_float2(hi, sign ? -lo : lo);
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xff;
  if (e == 0 || e == 0xff) return (double)f;  // zero, subnormal, inf, nan: rare
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long exp = (unsigned long long)(e - 127 + 1023) << 52;
  const unsigned long long man = (unsigned long long)(b & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | exp | man));
}

__device__ __forceinline__ void split3f(float hi, float lo, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(hi);
  const float r = (hi - __bfloat162float(a)) + lo;
  b = __float2bfloat16_rn(r);
  c = __float2bfloat16_rn(r - __bfloat162float(b));
}

// split3f on two values at once, with paired conversions (bit-identical to two split3f calls):
// .x of each result slice comes from (h0, l0), .y from (h1, l1).
__device__ __forceinline__ void split3f2(float h0, float l0, float h1, float l1, __nv_bfloat162& a,
                                         __nv_bfloat162& b, __nv_bfloat162& c) {
  a = __floats2bfloat162_rn(h0, h1);
  const float2 af = __bfloat1622float2(a);
  const float r0 = (h0 - af.x) + l0, r1 = (h1 - af.y) + l1;
  b = __floats2bfloat162_rn(r0, r1);
  const float2 bf = __bfloat1622float2(b);
  c = __floats2bfloat162_rn(r0 - bf.x, r1 - bf.y);
}

__device__ __forceinline__ void split3d(double x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  const float2 p = d2ff(x);
  split3f(p.x, p.y, a, b, c);
}

}  // namespace dmet
