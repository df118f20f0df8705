// Operand precisions of the tensor-core path: how an FP32 two-float value (hi + lo, ~48 bits) is
// split into slices that the tensor cores multiply exactly, and which slice products are issued.
//
//   BF16x3  three bf16 slices (8 significant bits each), the six products s + t <= 2 (~2^-24
//           relative per product; FP32's exponent range, so no scaling).
//   FP16x2  two fp16 slices (11 significant bits each) of the value times a power-of-two scale,
//           the three products s + t <= 1 (~2^-22 relative): half the products of BF16x3 at the
//           same tensor rate. FP16's exponent range is narrow (normal numbers 2^-14 .. 2^16), so
//           every operand is scaled by a power of two that puts a rigorous bound on its magnitude
//           at 2^14 (scales are computed on the device from the inputs' maxima; a scale is exact,
//           so the product is unchanged and the scaling is undone exactly in the epilogue). Below
//           2^-14 the low slice becomes subnormal: its absolute error stays under 2^-25, i.e.
//           2^-39 of the bound.
//   TF32    one TF32 slice (11 significant bits, FP32 exponent range), one product (~2^-11).
//   TF32x3  two TF32 slices, three products (~2^-22), at half the rate of the 16-bit kinds.
//
// A slice is the round-to-nearest of what the previous slices left over; the leftover after a
// rounding to fewer bits of the same exponent range is exact in FP32 (Sterbenz), so the slices sum
// to the value up to the last slice's rounding.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace dmet {
namespace tc {

enum MmaKind { kKindF16 = 0, kKindTF32 = 1 };

// Round-to-nearest (ties away) to TF32: an FP32 bit pattern whose low 13 mantissa bits are zero.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct PrecBF16x3 {
  using T = __nv_bfloat16;
  static constexpr int kSlices = 3;
  static constexpr int kProducts = 6;
  static constexpr int kKind = kKindF16;
  static constexpr uint32_t kFormat = 1;  // instruction-descriptor A/B type: BF16
  static constexpr bool kScaled = false;
  // product p multiplies slice prod_a(p) of A by slice prod_b(p) of B (product 0 is the leading one)
  __host__ __device__ static constexpr int prod_a(int p) { return p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0); }
  __host__ __device__ static constexpr int prod_b(int p) { return p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0); }
  __device__ __forceinline__ static void split(float hi, float lo, T* s) {
    s[0] = __float2bfloat16_rn(hi);
    const float r = (hi - __bfloat162float(s[0])) + lo;
    s[1] = __float2bfloat16_rn(r);
    s[2] = __float2bfloat16_rn(r - __bfloat162float(s[1]));
  }
};

struct PrecFP16x2 {
  using T = __half;
  static constexpr int kSlices = 2;
  static constexpr int kProducts = 3;
  static constexpr int kKind = kKindF16;
  static constexpr uint32_t kFormat = 0;  // F16
  static constexpr bool kScaled = true;
  __host__ __device__ static constexpr int prod_a(int p) { return p == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int prod_b(int p) { return p == 1 ? 1 : 0; }
  __device__ __forceinline__ static void split(float hi, float lo, T* s) {
    s[0] = __float2half_rn(hi);
    s[1] = __float2half_rn((hi - __half2float(s[0])) + lo);
  }
};

struct PrecTF32 {
  using T = float;
  static constexpr int kSlices = 1;
  static constexpr int kProducts = 1;
  static constexpr int kKind = kKindTF32;
  static constexpr uint32_t kFormat = 2;  // TF32
  static constexpr bool kScaled = false;
  __host__ __device__ static constexpr int prod_a(int) { return 0; }
  __host__ __device__ static constexpr int prod_b(int) { return 0; }
  __device__ __forceinline__ static void split(float hi, float lo, T* s) { s[0] = tf32_rna(hi + lo); }
};

struct PrecTF32x3 {
  using T = float;
  static constexpr int kSlices = 2;
  static constexpr int kProducts = 3;
  static constexpr int kKind = kKindTF32;
  static constexpr uint32_t kFormat = 2;
  static constexpr bool kScaled = false;
  __host__ __device__ static constexpr int prod_a(int p) { return p == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int prod_b(int p) { return p == 1 ? 1 : 0; }
  __device__ __forceinline__ static void split(float hi, float lo, T* s) {
    s[0] = tf32_rna(hi);
    s[1] = tf32_rna((hi - s[0]) + lo);
  }
};

// Elements of one 64-byte K block (a K-major row of a swizzled shared-memory tile).
template <class PREC>
constexpr int kblock_elems() {
  return 64 / (int)sizeof(typename PREC::T);
}

}  // namespace tc
}  // namespace dmet
