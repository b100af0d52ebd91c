// Fifth-generation tensor-core (tcgen05) building blocks for sm_100-family GPUs, written as
// inline PTX from the PTX ISA ("Tensor Memory", "tcgen05 instructions", "Matrix descriptors",
// "Instruction descriptor"): tensor-memory allocation, the single-thread MMA with FP32
// accumulators in tensor memory, commit to an mbarrier, and the warp-wide loads and stores
// between registers and tensor memory.
//
// Tensor memory (TMEM) is 128 lanes x 512 columns of 32 bits per SM. An address is
// (lane << 16) | column. A warp reaches only the 32 lanes of its quarter, lanes
// 32 (warp % 4) .. 32 (warp % 4) + 31; with the .32x32b shape thread t of the warp moves lane
// 32 (warp % 4) + t, columns col .. col + x - 1.
#pragma once

#include <cstdint>

namespace swense {
namespace tc {

// ---------------------------------------------------------------- allocation (one warp)
// Allocates `ncols` columns (a power of two, 32..512) and writes the base address to *dst
// (shared memory). Every allocation must be released with dealloc before the CTA exits.
__device__ __forceinline__ void alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// The same for a CTA pair (cta_group::2, a cluster of two CTAs): one warp of each CTA executes
// it; the pair's tensor memory is allocated at the same columns in both CTAs.
__device__ __forceinline__ void alloc2(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void relinquish2() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc2(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------- ordering
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------- descriptors
// Shared-memory matrix descriptor, K-major operand without swizzling ("interleaved" layout): the
// matrix is tiled into core matrices of 8 rows x 16 bytes (8 BF16 along K), each stored as 128
// contiguous bytes (row r at 16 r). lbo = byte distance between core matrices adjacent along K,
// sbo = byte distance between core matrices adjacent along M or N. Bits 46..48 hold the fixed
// value 0b001 of this descriptor version; base offset, stride mode and swizzle are zero.
__device__ __forceinline__ uint64_t smem_desc(const void* base, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(base));
  uint64_t d = 0;
  d |= uint64_t((a >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulation, both operands
// K-major, dense, no negation: D format at bits 4..5 (1 = F32), A and B formats at 7..9 and
// 10..12 (1 = BF16), N >> 3 at 17..22, M >> 4 at 24..28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// ---------------------------------------------------------------- MMA (issued by one thread)
// D[tmem] (+)= A[tmem] x B[smem]: A is M x 16 in tensor memory (lane = row, column c holds K
// elements 2c and 2c + 1), B is described by b_desc (N x 16, K-major). accumulate = 0
// overwrites D.
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The same with A in shared memory (a_desc, M x 16, K-major).
__device__ __forceinline__ void mma_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// CTA-pair MMA (issued by one thread of the pair's even CTA): D (M = 256) += A x B with A's rows
// 0..127 in the even CTA's tensor memory and 128..255 in the odd CTA's (same columns), B's
// columns 0..N/2-1 in the even CTA's shared memory and N/2..N-1 in the odd CTA's (same
// offsets, each half in the K-major core-matrix layout of b_desc), D's rows in each CTA's own
// tensor memory at d_tmem.
__device__ __forceinline__ void mma2_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The same with A in shared memory: a_desc describes each CTA's 128 rows (same offset in both).
__device__ __forceinline__ void mma2_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The mbarrier at the same offset in every CTA of cta_mask receives one arrival when every
// earlier tcgen05 operation of the pair issued by this thread has completed.
__device__ __forceinline__ void commit2(uint64_t* bar, uint16_t cta_mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          static_cast<unsigned>(__cvta_generic_to_shared(bar))),
      "h"(cta_mask)
      : "memory");
}

// The mbarrier receives one arrival when every earlier tcgen05 operation of this thread has
// completed (a CTA's own shared address is a valid shared::cluster address).
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   static_cast<unsigned>(__cvta_generic_to_shared(bar)))
               : "memory");
}

// ---------------------------------------------------------------- registers <-> tensor memory
__device__ __forceinline__ void ld_x16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void ld_x8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void st_x16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace tc
}  // namespace swense
