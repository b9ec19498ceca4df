// BF16 tensor-core helpers shared by the tensor-core tangent and the warm-start network:
// mma.sync m16n8k16 with BF16 operands and FP32 accumulation, BF16 pair packing, and the split of
// FP32 values into sums of BF16 values (Henry, Tang & Heinecke, "Leveraging the bfloat16
// artificial intelligence datatype for higher-precision computations", 2019): x = h + m + l with
// h = bf16(x), m = bf16(x - h), l = bf16(x - h - m) represents x to about 2^-24 |x|, and a product
// of a split operand with a BF16 operand is summed from one MMA per term.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace vms {

#if defined(__CUDACC__)
// two FP32 values rounded to a BF16 pair: `lo` in the low half (the smaller column or K index)
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float2 bf16x2_value(uint32_t w) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
}
// (x, y) = h + l (two terms: |x - h - l| <= 2^-16 |x|)
__device__ __forceinline__ void bf16x2_split2(float x, float y, uint32_t& h, uint32_t& l) {
  h = bf16x2(x, y);
  const float2 hv = bf16x2_value(h);
  l = bf16x2(x - hv.x, y - hv.y);
}
// (x, y) = h + m + l (three terms)
__device__ __forceinline__ void bf16x2_split3(float x, float y, uint32_t& h, uint32_t& m, uint32_t& l) {
  h = bf16x2(x, y);
  const float2 hv = bf16x2_value(h);
  const float rx = x - hv.x, ry = y - hv.y;
  m = bf16x2(rx, ry);
  const float2 mv = bf16x2_value(m);
  l = bf16x2(rx - mv.x, ry - mv.y);
}
// d += a b for a 16x16 row-major A fragment and a 16x8 column-major B fragment
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
#endif

}  // namespace vms
