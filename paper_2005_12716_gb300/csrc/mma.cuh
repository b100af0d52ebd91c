// BF16 tensor-core helpers shared by the MLP and the split-BF16 direct sum: packing, the hi + lo
// split of FP32 values, and the m16n8k16 warp MMA with FP32 accumulation.
//
// Fragment layout of mma.sync.m16n8k16 (PTX ISA, "Matrix fragments for mma.m16n8k16"), with
// g = lane / 4 and q = lane % 4:
//   A (16 x 16, row-major)   a0: (g, 2q..2q+1)  a1: (g+8, 2q..2q+1)  a2: (g, 2q+8..)  a3: (g+8, 2q+8..)
//   B (16 x 8, column-major) b0: rows 2q..2q+1 of column g   b1: rows 2q+8..2q+9 of column g
//   C (16 x 8)               c0, c1: (g, 2q), (g, 2q+1)   c2, c3: (g+8, 2q), (g+8, 2q+1)
// Each 32-bit register holds two BF16 values, the lower column (or row) in the low half.
#pragma once

#include <cuda_bf16.h>

namespace swense {

__device__ __forceinline__ unsigned bf2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}

// hi + lo split of a pair: hi = bf16(x), lo = bf16(x - hi), both round-to-nearest. The hi halves
// are widened back to FP32 exactly by placing their bits in the upper half of a word.
__device__ __forceinline__ void bf2_split(float a, float b, unsigned& hi, unsigned& lo) {
  hi = bf2(a, b);
  const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xffff0000u);
  lo = bf2(a - ha, b - hb);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16-byte global -> shared asynchronous copy (src_bytes < 16 zero-fills the rest).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

}  // namespace swense
