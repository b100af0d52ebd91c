// The learned-correction network shared by the training kernels and the fused gather: sizes,
// parameter offsets, the BF16 packed weight layout, GELU, and the per-warp layer step on
// m16n8k16 fragments (see mlp.cu for the network's definition).
#pragma once

#include <cuda_bf16.h>

#include <cstddef>

#include "internal.cuh"
#include "mma.cuh"

namespace swense {
namespace mlpnet {

constexpr int NIN = 67, KIN = 80, NH = 64, NOUT = 4, NO = 8, XLD = 68;
constexpr int OFF_W1 = 0, OFF_B1 = NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NOUT * NH, NPARAM = OFF_B3 + NOUT;
static_assert(NPARAM == SWENSE_MLP_NPARAM, "parameter count");

// BF16 copies of the weights in the layouts the MMAs read, plus FP32 biases. The forward part
// comes first (PackedFwd is a prefix of Packed), so inference kernels copy only that.
struct Packed {
  __nv_bfloat16 w1[NH][KIN];    // B of layer 1: [n = hidden][k = input], inputs 67..79 zero
  __nv_bfloat16 w2[NH][NH];     // B of layer 2: [n][k]
  __nv_bfloat16 w3[NO][NH];     // B of layer 3: rows 4..7 zero
  float b1[NH], b2[NH], b3[NO];
  float out_scale;              // inference output multiplier (training targets were divided by it)
  float pad_[3];
  __nv_bfloat16 w2t[NH][NH];    // W2 transposed (backward)
  __nv_bfloat16 w3t[NH][16];    // W3 transposed, k padded to 16 (backward)
};
struct PackedFwd {
  __nv_bfloat16 w1[NH][KIN];
  __nv_bfloat16 w2[NH][NH];
  __nv_bfloat16 w3[NO][NH];
  float b1[NH], b2[NH], b3[NO];
  float out_scale;
  float pad_[3];
};
static_assert(offsetof(Packed, w2t) == sizeof(PackedFwd) && offsetof(Packed, out_scale) == offsetof(PackedFwd, out_scale) &&
              offsetof(Packed, b1) == offsetof(PackedFwd, b1), "PackedFwd is a prefix of Packed");
static_assert(sizeof(PackedFwd) % 16 == 0, "forward part is copied in 16-byte words");
static_assert(sizeof(Packed) <= SWENSE_MLP_PACKED_BYTES, "packed weight size");
static_assert(sizeof(Packed) % 16 == 0, "packed weight size must be a multiple of 16 bytes");

__device__ __forceinline__ unsigned ld_u32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const unsigned*>(p);
}

// GELU, tanh form: 0.5 x (1 + tanh(u)), u = sqrt(2/pi) (x + 0.044715 x^3), with
// tanh(u) = 1 - 2 / (1 + e^{2u}) (saturates correctly at both ends; absolute error ~1e-7 near
// u = 0, far below the BF16 operands it feeds).
__device__ __forceinline__ float gelu_tanh_u(float x) {
  const float c = 0.7978845608028654f;
  const float u = c * fmaf(0.044715f * x, x * x, x);
  return 1.f - __fdividef(2.f, 1.f + __expf(2.f * u));
}
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + gelu_tanh_u(x)); }
__device__ __forceinline__ float gelu_grad(float x) {
  const float c = 0.7978845608028654f;
  const float t = gelu_tanh_u(x);
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * c * fmaf(3.f * 0.044715f, x * x, 1.f);
}

// ------------------------------------------------------------------------------ forward
// Layer with K = 16 * KS inputs held as A fragments (hi and optional lo), N = 8 * NT outputs.
template <int KS, int NT, bool SPLIT>
__device__ __forceinline__ void layer(float (&z)[NT][4], const unsigned (&ahi)[KS][4],
                                      const unsigned (&alo)[KS][4], const __nv_bfloat16* W, int ldw,
                                      const float* bias, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const float bb0 = bias[8 * nt + 2 * t], bb1 = bias[8 * nt + 2 * t + 1];
    z[nt][0] = bb0;
    z[nt][1] = bb1;
    z[nt][2] = bb0;
    z[nt][3] = bb1;
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      const __nv_bfloat16* wr = W + (8 * nt + g) * ldw + 16 * kk + 2 * t;
      const unsigned b0 = ld_u32(wr), b1 = ld_u32(wr + 8);
      mma16816(z[nt], ahi[kk], b0, b1);
      if (SPLIT) mma16816(z[nt], alo[kk], b0, b1);
    }
  }
}

// Accumulator fragments (16 x 8*NT, FP32) -> A fragments (16 x 16*NT/2) after GELU.
template <int NT, bool SPLIT>
__device__ __forceinline__ void to_a(const float (&z)[NT][4], unsigned (&ahi)[NT / 2][4],
                                     unsigned (&alo)[NT / 2][4]) {
#pragma unroll
  for (int kk = 0; kk < NT / 2; ++kk) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float* c = z[2 * kk + h];
      const float g0 = gelu(c[0]), g1 = gelu(c[1]), g2 = gelu(c[2]), g3 = gelu(c[3]);
      if (SPLIT) {
        bf2_split(g0, g1, ahi[kk][2 * h], alo[kk][2 * h]);
        bf2_split(g2, g3, ahi[kk][2 * h + 1], alo[kk][2 * h + 1]);
      } else {
        ahi[kk][2 * h] = bf2(g0, g1);
        ahi[kk][2 * h + 1] = bf2(g2, g3);
      }
    }
  }
}


}  // namespace mlpnet
}  // namespace swense
