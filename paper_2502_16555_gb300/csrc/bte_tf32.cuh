// Split of an FP32 value into a TF32 head (round-to-nearest) and its exact FP32 remainder, the
// operand form of the three-product TF32 GEMM (a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi).
#pragma once
#include <cstdint>

namespace bte {
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}
}  // namespace bte
