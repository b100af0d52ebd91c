// Internal helpers shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "swense.h"

namespace swense {

// ---------------------------------------------------------------- error reporting (host)
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SWENSE_CUDA_TRY(call)                                   \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::swense::cuda_fail(e_, #call); \
  } while (0)

// ---------------------------------------------------------------- per-device scratch
// Returns a device pointer to at least `bytes` bytes of scratch (256-byte aligned), growing the
// device's workspace if needed. Growing synchronises the device and is refused during capture.
int workspace(size_t bytes, cudaStream_t stream, void** out);

// Twiddle array: the plain table e^{+2 pi i j / SWENSE_MAX_FFT}, j < SWENSE_MAX_FFT, followed by
// the Stockham passes' pass-major tables (fft.cuh, stk_twp). The first call on a device fills it
// with a kernel on `stream` and waits for it (refused during stream capture).
int twiddles(cudaStream_t stream, const float2** out);

// Counts kernel launches made by the library (reported by swense_launches()).
void count_launches(int n);

// Device-side error flags of bounded waits, one per translation unit that has such waits: read
// (and cleared when reset) on the current device; *was_set != 0 when a wait gave up.
int grid_async_flag(bool reset, int* was_set);
int direct_async_flag(bool reset, int* was_set);

// Near-body direct sums (direct.cu, direct_tc.cu). direct_tc: the tensor-core split-BF16 path;
// direct_split_sorted: the per-pair split-BF16 kernel over points sorted by the tensor-core path
// (srt, perm: sorted coordinates and sorted -> caller index), restricted to the tiles of
// `tile_pts` sorted points that tile_bad marks.
int direct_tc(const swense_modes* md, double t, const float* pts, int64_t np, float* eta, float* u,
              float* v, float* w, float* p, int32_t p_mode, double rho, double grav, cudaStream_t stream);
// Grid reconstruction with caller-supplied scratch (grid_ifft.cu), for concurrent batches.
int grid_scratch(const swense_modes* md, int32_t n_tl, const double* t, const swense_grid_desc* desc,
                 float* nodes, float* eta, size_t* bytes);
int grid_with_scratch(const swense_modes* md, int32_t n_tl, const double* t, const swense_grid_desc* desc,
                      float* nodes, float* eta, void* ws, cudaStream_t stream);

// One gather of a batch (interp.cu): the grid and the points of one instance.
struct GatherItem {
  swense_grid grid;
  double t;
  const float* pts;
  const int32_t* perm;
  int64_t np;
  float *eta, *u, *v, *w, *p;
};
// Scratch (plan and queue counter) of interp_batch for these items, and the batch itself: every
// item's point chunks planned by one launch and gathered by one persistent launch whose CTAs
// take chunks from a device queue. `ws` holds interp_batch_bytes(items) bytes.
int interp_batch_bytes(const GatherItem* items, int n, size_t* bytes);
int interp_batch(const GatherItem* items, int n, int32_t p_mode, double rho, double grav, void* ws,
                 cudaStream_t stream);

size_t split_table_bytes(const swense_modes* md);
int direct_split_sorted(const swense_modes* md, double t, const float* srt, const int32_t* perm,
                        const uint8_t* tile_bad, int tile_pts, int64_t np, float* eta, float* u, float* v,
                        float* w, float* p, int32_t p_mode, double rho, double grav, cudaStream_t stream,
                        size_t ws_offset);

inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
inline int ilog2(int64_t v) { int r = 0; while ((int64_t(1) << r) < v) ++r; return r; }

// ---------------------------------------------------------------- device complex helpers
// Complex add and subtract as one packed FP32x2 instruction each (sm_100 and later): both
// halves are rounded to nearest like the scalar operations, so the results are unchanged.
__device__ __forceinline__ unsigned long long c_as_u64(float2 a) {
  return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ float2 u64_as_c(unsigned long long v) {
  return make_float2(__uint_as_float(unsigned(v)), __uint_as_float(unsigned(v >> 32)));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(c_as_u64(a)), "l"(c_as_u64(b)));
  return u64_as_c(d);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(c_as_u64(a)), "l"(c_as_u64(b)));
  return u64_as_c(d);
}
// Element-wise product (and fused product-sum) of pairs as one packed instruction (x with x,
// y with y), rounded like the scalar forms.
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(c_as_u64(a)), "l"(c_as_u64(b)));
  return u64_as_c(d);
}
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(c_as_u64(a)), "l"(c_as_u64(b)), "l"(c_as_u64(c)));
  return u64_as_c(d);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }   // i*a
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// x / L as an unsigned 32-bit fraction of a turn (FP64 once per point), so that a mode's phase
// m X (mod 2^32) is exact whatever |k x|.
__device__ __forceinline__ unsigned turn_fraction(float x, double inv_l) {
  const double f = double(x) * inv_l;
  const double fr = f - floor(f);                        // [0, 1)
  return unsigned((unsigned long long)(fr * 4294967296.0) & 0xffffffffull);
}

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) {
  return bits == 0 ? 0u : (__brev(v) >> (32 - bits));
}

}  // namespace swense
