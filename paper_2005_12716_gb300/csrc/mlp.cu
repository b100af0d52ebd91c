// Learned correction of the interpolated fields (not in the paper; an addition to its
// interpolation step): one multilayer perceptron shared by the four fields u, v, w, dphi/dt,
//   input  x = [stencil_f / s_f (64 time-blended 4x4x4 node values, x fastest, then y, then z),
//              dx, dy, dz (offsets of the point in the stencil's middle cell)],
//              s_f = max |stencil_f| + 1e-30,
//   layers 67 -> 64 -> 64 -> 4, GELU (tanh form) on the hidden layers, output y[f] used,
//   correction  f = lagrange_f + s_f y[f], pressure from the corrected fields (Bernoulli).
//
// Tensor cores: BF16 mma.sync (m16n8k16) with FP32 accumulation; one warp owns 16 rows, and a
// layer's accumulator fragments become the next layer's A fragments in registers. Inference
// splits inputs and activations into BF16 hi + lo (two MMAs per step) so the result tracks an
// FP64 evaluation of the same BF16 weights to ~1e-5; training uses plain BF16 operands.
// Weight gradients (sums over the batch) are reduced on the CUDA cores in FP32, then Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "mlp.cuh"

namespace swense {
namespace {

using namespace mlpnet;

// ------------------------------------------------------------------------------ pack
__global__ void k_mlp_pack(const float* __restrict__ P, Packed* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NH * KIN) {
    const int n = i / KIN, k = i % KIN;
    out->w1[n][k] = __float2bfloat16_rn(k < NIN ? P[OFF_W1 + n * NIN + k] : 0.f);
  }
  if (i < NH * NH) {
    const int n = i / NH, k = i % NH;
    out->w2[n][k] = __float2bfloat16_rn(P[OFF_W2 + n * NH + k]);
    out->w2t[n][k] = __float2bfloat16_rn(P[OFF_W2 + k * NH + n]);
  }
  if (i < NO * NH) {
    const int n = i / NH, k = i % NH;
    out->w3[n][k] = __float2bfloat16_rn(n < NOUT ? P[OFF_W3 + n * NH + k] : 0.f);
  }
  if (i < NH * 16) {
    const int n = i / 16, k = i % 16;
    out->w3t[n][k] = __float2bfloat16_rn(k < NOUT ? P[OFF_W3 + k * NH + n] : 0.f);
  }
  if (i < NH) {
    out->b1[i] = P[OFF_B1 + i];
    out->b2[i] = P[OFF_B2 + i];
  }
  if (i < NO) out->b3[i] = i < NOUT ? P[OFF_B3 + i] : 0.f;
}

// A fragments of 16 rows of x (FP32, leading dimension XLD, columns >= NIN read as 0).
template <bool SPLIT>
__device__ __forceinline__ void load_x(const float* __restrict__ x, int64_t row0, int64_t rows,
                                       const int32_t* __restrict__ idx, unsigned (&ahi)[5][4],
                                       unsigned (&alo)[5][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  int64_t r[2] = {row0 + g, row0 + g + 8};
  const float* xr[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const bool ok = r[h] < rows;
    const int64_t rr = ok ? (idx ? int64_t(idx[r[h]]) : r[h]) : 0;
    xr[h] = ok ? x + rr * XLD : nullptr;
  }
#pragma unroll
  for (int kk = 0; kk < 5; ++kk) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int h = q & 1;                         // a0, a2: row g; a1, a3: row g + 8
      const int col = 16 * kk + 2 * t + (q >= 2 ? 8 : 0);
      float v0 = 0.f, v1 = 0.f;
      if (xr[h]) {
        if (col < NIN) v0 = __ldg(&xr[h][col]);
        if (col + 1 < NIN) v1 = __ldg(&xr[h][col + 1]);
      }
      if (SPLIT) bf2_split(v0, v1, ahi[kk][q], alo[kk][q]);
      else ahi[kk][q] = bf2(v0, v1);
    }
  }
}

// Inference: y[row] = network(x[row])[row % 4] (rows ordered point-major, fields u, v, w, phit).
__global__ void __launch_bounds__(128) k_mlp_forward(const Packed* __restrict__ P, const float* __restrict__ x,
                                                     int64_t rows, float* __restrict__ y) {
  __shared__ Packed s;
  {
    const int4* src = reinterpret_cast<const int4*>(P);
    int4* dst = reinterpret_cast<int4*>(&s);
    for (int i = threadIdx.x; i < int(sizeof(Packed) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int64_t row0 = (int64_t(blockIdx.x) * 4 + warp) * 16; row0 < rows;
       row0 += int64_t(gridDim.x) * 64) {
    unsigned xh[5][4], xl[5][4];
    load_x<true>(x, row0, rows, nullptr, xh, xl, lane);
    float z1[8][4];
    layer<5, 8, true>(z1, xh, xl, &s.w1[0][0], KIN, s.b1, lane);
    unsigned h1h[4][4], h1l[4][4];
    to_a<8, true>(z1, h1h, h1l);
    float z2[8][4];
    layer<4, 8, true>(z2, h1h, h1l, &s.w2[0][0], NH, s.b2, lane);
    unsigned h2h[4][4], h2l[4][4];
    to_a<8, true>(z2, h2h, h2l);
    float o[1][4];
    layer<4, 1, true>(o, h2h, h2l, &s.w3[0][0], NH, s.b3, lane);
    // row r uses output column r % 4: c0/c1 hold columns 2t, 2t+1 of row g, c2/c3 of row g+8
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = row0 + g + 8 * h;
      const int f = (g + 8 * h) & 3;               // row0 is a multiple of 16
      const float yv = (f & 1) ? o[0][2 * h + 1] : o[0][2 * h];   // a select, not a local array
      if (r < rows && (f >> 1) == t) y[r] = yv * s.out_scale;
    }
  }
}

// ------------------------------------------------------------------------------ training
struct TrainArgs {
  const Packed* P;
  const float* x;          // [N][XLD] features
  const int32_t* field;    // [N]
  const float* target;     // [N]
  const int32_t* batch;    // [B] row indices into x
  int B;
  float* h1;               // [B][64] saved activations (FP32)
  float* h2;
  float* dz1;
  float* dz2;
  float* dy;               // [B][4]
  float* loss;             // scalar (sum of squared residuals / B)
};

__global__ void __launch_bounds__(128) k_mlp_train_fb(TrainArgs a) {
  __shared__ Packed s;
  {
    const int4* src = reinterpret_cast<const int4*>(a.P);
    int4* dst = reinterpret_cast<int4*>(&s);
    for (int i = threadIdx.x; i < int(sizeof(Packed) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const float invB = 1.f / float(a.B);
  float lsum = 0.f;
  for (int64_t row0 = (int64_t(blockIdx.x) * 4 + warp) * 16; row0 < a.B;
       row0 += int64_t(gridDim.x) * 64) {
    unsigned xh[5][4], xl[5][4];
    load_x<false>(a.x, row0, a.B, a.batch, xh, xl, lane);
    float z1[8][4];
    layer<5, 8, false>(z1, xh, xl, &s.w1[0][0], KIN, s.b1, lane);
    unsigned h1[4][4], unused1[4][4];
    to_a<8, false>(z1, h1, unused1);
    float z2[8][4];
    layer<4, 8, false>(z2, h1, unused1, &s.w2[0][0], NH, s.b2, lane);
    unsigned h2[4][4], unused2[4][4];
    to_a<8, false>(z2, h2, unused2);
    float o[1][4];
    layer<4, 1, false>(o, h2, unused2, &s.w3[0][0], NH, s.b3, lane);
    // dY: only the row's own output column carries 2 (y - target) / B
    float dyf[4];
    int64_t rr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      rr[h] = row0 + g + 8 * h;
      const bool ok = rr[h] < a.B;
      const int src = ok ? a.batch[rr[h]] : 0;
      const int f = ok ? a.field[src] : -1;
      const float tg = ok ? a.target[src] : 0.f;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = 2 * t + c;
        float d = 0.f;
        if (col == f) {
          const float res = o[0][2 * h + c] - tg;
          lsum = fmaf(res, res, lsum);
          d = 2.f * res * invB;
        }
        dyf[2 * h + c] = d;
      }
    }
    // dH2 = dY W3  (K = 8 padded to 16)
    unsigned ady[4] = {bf2(dyf[0], dyf[1]), bf2(dyf[2], dyf[3]), 0u, 0u};
    float dh2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      dh2[nt][0] = dh2[nt][1] = dh2[nt][2] = dh2[nt][3] = 0.f;
      const __nv_bfloat16* wr = &s.w3t[8 * nt + g][2 * t];
      mma16816(dh2[nt], ady, ld_u32(wr), ld_u32(wr + 8));
    }
    // dZ2 = dH2 * gelu'(Z2); dH1 = dZ2 W2
    float dz2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) dz2[nt][q] = dh2[nt][q] * gelu_grad(z2[nt][q]);
    unsigned adz2[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      adz2[kk][0] = bf2(dz2[2 * kk][0], dz2[2 * kk][1]);
      adz2[kk][1] = bf2(dz2[2 * kk][2], dz2[2 * kk][3]);
      adz2[kk][2] = bf2(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
      adz2[kk][3] = bf2(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
    }
    float dh1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      dh1[nt][0] = dh1[nt][1] = dh1[nt][2] = dh1[nt][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const __nv_bfloat16* wr = &s.w2t[8 * nt + g][16 * kk + 2 * t];
        mma16816(dh1[nt], adz2[kk], ld_u32(wr), ld_u32(wr + 8));
      }
    }
    // save per-row activations and gradients for the weight-gradient reduction
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (rr[h] >= a.B) continue;
      const int64_t r = rr[h];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int col = 8 * nt + 2 * t;
        const float e0 = z1[nt][2 * h], e1 = z1[nt][2 * h + 1];
        const float f0 = z2[nt][2 * h], f1 = z2[nt][2 * h + 1];
        *reinterpret_cast<float2*>(&a.h1[r * NH + col]) = make_float2(gelu(e0), gelu(e1));
        *reinterpret_cast<float2*>(&a.h2[r * NH + col]) = make_float2(gelu(f0), gelu(f1));
        *reinterpret_cast<float2*>(&a.dz2[r * NH + col]) = make_float2(dz2[nt][2 * h], dz2[nt][2 * h + 1]);
        *reinterpret_cast<float2*>(&a.dz1[r * NH + col]) =
            make_float2(dh1[nt][2 * h] * gelu_grad(e0), dh1[nt][2 * h + 1] * gelu_grad(e1));
      }
      if (t < 2) *reinterpret_cast<float2*>(&a.dy[r * 4 + 2 * t]) = make_float2(dyf[2 * h], dyf[2 * h + 1]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0 && a.loss) atomicAdd(a.loss, lsum * invB);
}

// Weight gradients: one thread per parameter, a slice of the batch per grid row, FP32 sums.
__global__ void k_mlp_wgrad(const float* __restrict__ x, const int32_t* __restrict__ batch, int B,
                            const float* __restrict__ h1, const float* __restrict__ h2,
                            const float* __restrict__ dz1, const float* __restrict__ dz2,
                            const float* __restrict__ dy, int slice, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const int r0 = blockIdx.y * slice, r1 = min(B, r0 + slice);
  float acc = 0.f;
  if (p < OFF_B1) {
    const int i = p / NIN, k = p % NIN;
    for (int r = r0; r < r1; ++r) acc = fmaf(dz1[r * NH + i], __ldg(&x[int64_t(batch[r]) * XLD + k]), acc);
  } else if (p < OFF_W2) {
    const int i = p - OFF_B1;
    for (int r = r0; r < r1; ++r) acc += dz1[r * NH + i];
  } else if (p < OFF_B2) {
    const int i = (p - OFF_W2) / NH, j = (p - OFF_W2) % NH;
    for (int r = r0; r < r1; ++r) acc = fmaf(dz2[r * NH + i], h1[r * NH + j], acc);
  } else if (p < OFF_W3) {
    const int i = p - OFF_B2;
    for (int r = r0; r < r1; ++r) acc += dz2[r * NH + i];
  } else if (p < OFF_B3) {
    const int o = (p - OFF_W3) / NH, j = (p - OFF_W3) % NH;
    for (int r = r0; r < r1; ++r) acc = fmaf(dy[r * 4 + o], h2[r * NH + j], acc);
  } else {
    const int o = p - OFF_B3;
    for (int r = r0; r < r1; ++r) acc += dy[r * 4 + o];
  }
  atomicAdd(&grad[p], acc);
}

__global__ void k_mlp_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, float lr, float b1, float b2, float eps,
                           float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const float gr = grad[p];
  const float mm = fmaf(b1, m[p], (1.f - b1) * gr);
  const float vv = fmaf(b2, v[p], (1.f - b2) * gr * gr);
  m[p] = mm;
  v[p] = vv;
  P[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_mlp_pack(const float* params, float out_scale, void* packed, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!params || !packed) return fail(SWENSE_ERR_ARG, "NULL params or packed buffer");
  if (reinterpret_cast<uintptr_t>(packed) & 15) return fail(SWENSE_ERR_ARG, "packed must be 16-byte aligned");
  if (!std::isfinite(out_scale) || !(out_scale > 0)) return fail(SWENSE_ERR_ARG, "out_scale must be finite and > 0");
  k_mlp_pack<<<(NH * KIN + 255) / 256, 256, 0, stream>>>(params, static_cast<Packed*>(packed));
  SWENSE_CUDA_TRY(cudaGetLastError());
  SWENSE_CUDA_TRY(cudaMemcpyAsync(&static_cast<Packed*>(packed)->out_scale, &out_scale, sizeof(float),
                                  cudaMemcpyHostToDevice, stream));
  SWENSE_CUDA_TRY(cudaStreamSynchronize(stream));
  count_launches(1);
  return SWENSE_OK;
}

extern "C" int swense_mlp_forward(const void* packed, const float* x, int64_t rows, float* y,
                                  void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (rows < 0) return fail(SWENSE_ERR_ARG, "rows must be >= 0");
  if (rows == 0) return SWENSE_OK;
  if (!packed || !x || !y) return fail(SWENSE_ERR_ARG, "NULL argument");
  if (reinterpret_cast<uintptr_t>(packed) & 15) return fail(SWENSE_ERR_ARG, "packed must be 16-byte aligned");
  const int64_t tiles = (rows + 63) / 64;
  const unsigned blocks = unsigned(std::min<int64_t>(tiles, 152 * 16));
  k_mlp_forward<<<blocks, 128, 0, stream>>>(static_cast<const Packed*>(packed), x, rows, y);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

extern "C" int swense_mlp_train_step(float* params, float* adam_m, float* adam_v, void* packed,
                                     int64_t step, const float* x, const int32_t* field,
                                     const float* target, const int32_t* batch, int32_t B, float lr,
                                     float beta1, float beta2, float eps, float* loss, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!params || !adam_m || !adam_v || !packed || !x || !field || !target || !batch)
    return fail(SWENSE_ERR_ARG, "NULL argument");
  if (B < 1 || B > (1 << 24)) return fail(SWENSE_ERR_ARG, "batch size must be in [1, 2^24]");
  if (step < 1) return fail(SWENSE_ERR_ARG, "step is 1-based");
  if (!(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return fail(SWENSE_ERR_ARG, "bad Adam hyper-parameters");
  const size_t act = size_t(B) * NH * sizeof(float);
  const size_t bytes = 4 * act + size_t(B) * 4 * sizeof(float) + NPARAM * sizeof(float) + 256;
  void* ws = nullptr;
  int st = workspace(bytes, stream, &ws);
  if (st) return st;
  char* w = static_cast<char*>(ws);
  float* grad = reinterpret_cast<float*>(w);
  float* h1 = reinterpret_cast<float*>(w + ((NPARAM * sizeof(float) + 255) & ~size_t(255)));
  float* h2 = h1 + size_t(B) * NH;
  float* dz1 = h2 + size_t(B) * NH;
  float* dz2 = dz1 + size_t(B) * NH;
  float* dy = dz2 + size_t(B) * NH;
  SWENSE_CUDA_TRY(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), stream));
  if (loss) SWENSE_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), stream));
  TrainArgs a{static_cast<const Packed*>(packed), x, field, target, batch, B, h1, h2, dz1, dz2, dy, loss};
  const unsigned blocks = unsigned(std::min<int64_t>((int64_t(B) + 63) / 64, 152 * 16));
  k_mlp_train_fb<<<blocks, 128, 0, stream>>>(a);
  SWENSE_CUDA_TRY(cudaGetLastError());
  const int slice = 256;
  k_mlp_wgrad<<<dim3((NPARAM + 255) / 256, (B + slice - 1) / slice), 256, 0, stream>>>(
      x, batch, B, h1, h2, dz1, dz2, dy, slice, grad);
  SWENSE_CUDA_TRY(cudaGetLastError());
  const double t = double(step);
  k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, stream>>>(params, adam_m, adam_v, grad, lr, beta1, beta2,
                                                        eps, float(1.0 - std::pow(double(beta1), t)),
                                                        float(1.0 - std::pow(double(beta2), t)));
  SWENSE_CUDA_TRY(cudaGetLastError());
  k_mlp_pack<<<(NH * KIN + 255) / 256, 256, 0, stream>>>(params, static_cast<Packed*>(packed));
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(4);
  return SWENSE_OK;
}

extern "C" int swense_mlp_grad(const void* packed, const float* x, const int32_t* field,
                               const float* target, const int32_t* batch, int32_t B, float* grad,
                               float* loss, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!packed || !x || !field || !target || !batch || !grad) return fail(SWENSE_ERR_ARG, "NULL argument");
  if (B < 1 || B > (1 << 24)) return fail(SWENSE_ERR_ARG, "batch size must be in [1, 2^24]");
  const size_t bytes = 4 * size_t(B) * NH * sizeof(float) + size_t(B) * 4 * sizeof(float);
  void* ws = nullptr;
  int st = workspace(bytes, stream, &ws);
  if (st) return st;
  float* h1 = static_cast<float*>(ws);
  float* h2 = h1 + size_t(B) * NH;
  float* dz1 = h2 + size_t(B) * NH;
  float* dz2 = dz1 + size_t(B) * NH;
  float* dy = dz2 + size_t(B) * NH;
  SWENSE_CUDA_TRY(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), stream));
  if (loss) SWENSE_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), stream));
  TrainArgs a{static_cast<const Packed*>(packed), x, field, target, batch, B, h1, h2, dz1, dz2, dy, loss};
  const unsigned blocks = unsigned(std::min<int64_t>((int64_t(B) + 63) / 64, 152 * 16));
  k_mlp_train_fb<<<blocks, 128, 0, stream>>>(a);
  SWENSE_CUDA_TRY(cudaGetLastError());
  const int slice = 256;
  k_mlp_wgrad<<<dim3((NPARAM + 255) / 256, (B + slice - 1) / slice), 256, 0, stream>>>(
      x, batch, B, h1, h2, dz1, dz2, dy, slice, grad);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(2);
  return SWENSE_OK;
}
