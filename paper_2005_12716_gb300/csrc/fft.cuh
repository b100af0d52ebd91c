// Shared-memory inverse DFT (sign +, unnormalised) used by the grid reconstruction kernels.
//
// Iterative Cooley-Tukey decimation in time, in place: the caller scatters each length-n input
// into bit-reversed positions; the stages then combine sub-transforms of length h into 4h
// (two radix-2 stages fused in registers, three twiddle products), preceded by one radix-2 stage
// when log2(n) is odd. Output is in natural order. `batch` arrays of length n lie back to back.
#pragma once

#include "internal.cuh"

namespace swense {

// tw[j] = e^{+2 pi i j / SWENSE_MAX_FFT}
__device__ __forceinline__ void fft_inv_inplace(float2* data, int n, int log2n, int batch,
                                                const float2* __restrict__ tw) {
  const int nthr = blockDim.x;
  int h = 1;
  if (log2n & 1) {
    const int half = n >> 1;
    for (int t = threadIdx.x; t < batch * half; t += nthr) {
      const int b = t / half, j = t - b * half;
      float2* a = data + size_t(b) * n + 2 * j;
      const float2 x0 = a[0], x1 = a[1];
      a[0] = cadd(x0, x1);
      a[1] = csub(x0, x1);
    }
    h = 2;
    __syncthreads();
  }
  const int quarter = n >> 2;
  for (; h < n; h <<= 2) {
    const int s1 = SWENSE_MAX_FFT / (2 * h);  // twiddle stride of the length-2h stage
    const int s2 = s1 >> 1;                   // ... of the length-4h stage
    for (int t = threadIdx.x; t < batch * quarter; t += nthr) {
      const int b = t / quarter, r = t - b * quarter;
      const int g = r / h, j = r - g * h;
      float2* a = data + size_t(b) * n + g * 4 * h + j;
      const float2 w1 = __ldg(&tw[j * s1]);
      const float2 w2 = __ldg(&tw[j * s2]);
      const float2 x0 = a[0], x1 = a[h], x2 = a[2 * h], x3 = a[3 * h];
      const float2 t1 = cmul(w1, x1);
      const float2 a0 = cadd(x0, t1), a1 = csub(x0, t1);
      const float2 t3 = cmul(w1, x3);
      const float2 a2 = cadd(x2, t3), a3 = csub(x2, t3);
      const float2 t2 = cmul(w2, a2);
      const float2 u = cmul_i(cmul(w2, a3));
      a[0] = cadd(a0, t2);
      a[2 * h] = csub(a0, t2);
      a[h] = cadd(a1, u);
      a[3 * h] = csub(a1, u);
    }
    __syncthreads();
  }
}

// Depth factors of the spectral decomposition at vertical position z for |k| = k:
//   finite depth h > 0: F = cosh(k(z+h))/cosh(kh), S = sinh(k(z+h))/cosh(kh), written as
//     (e^{kz} +- e^{-k(z+2h)}) / (1 + e^{-2kh}) so that no term overflows;
//   deep water (h <= 0): F = S = e^{kz}.
// k*z is formed as an unevaluated sum hi + lo (fma residual) so the factor keeps FP32 accuracy
// for the large |k z| of the levels above z = 0.
__device__ __forceinline__ void depth_factors(float k, float z, float h, float& F, float& S) {
  const float kz = k * z;
  const float kz_lo = fmaf(k, z, -kz);
  float e1 = expf(kz);
  e1 = fmaf(e1, kz_lo, e1);
  if (h <= 0.f) {
    F = e1;
    S = e1;
    return;
  }
  const float e2 = expf(-k * (z + 2.f * h));
  const float d = 1.f + expf(-2.f * k * h);
  F = (e1 + e2) / d;
  S = (e1 - e2) / d;
}

}  // namespace swense
