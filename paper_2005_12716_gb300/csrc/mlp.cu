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
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

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
  float* loss_part;        // [gridDim.x] per-block sums of squared residuals / B
  float tscale;            // targets are multiplied by this on reading
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
      const float tg = ok ? a.target[src] * a.tscale : 0.f;
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
  // per-block loss in a fixed order (no atomics: training is reproducible bit for bit)
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  __shared__ float wl[4];
  if (lane == 0) wl[warp] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) a.loss_part[blockIdx.x] = ((wl[0] + wl[1]) + (wl[2] + wl[3])) * invB;
}

// Weight gradients: one thread per parameter, a slice of the batch per grid row, FP32 sums;
// each slice's sum goes to its own row of `part` (summed in order by k_mlp_reduce).
__global__ void k_mlp_wgrad(const float* __restrict__ x, const int32_t* __restrict__ batch, int B,
                            const float* __restrict__ h1, const float* __restrict__ h2,
                            const float* __restrict__ dz1, const float* __restrict__ dz2,
                            const float* __restrict__ dy, int slice, float* __restrict__ part) {
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
  part[size_t(blockIdx.y) * NPARAM + p] = acc;
}

// grad = sum over the slices in order; loss = sum of the per-block losses in order.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nslices, float* __restrict__ grad,
                             const float* __restrict__ loss_part, int nblocks, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPARAM) {
    float acc = 0.f;
    for (int s = 0; s < nslices; ++s) acc += part[size_t(s) * NPARAM + p];
    grad[p] = acc;
  }
  if (p == 0 && loss) {
    float l = 0.f;
    for (int b = 0; b < nblocks; ++b) l += loss_part[b];
    *loss = l;
  }
}

// Mini-batch row indices of training step `step` (0-based): SplitMix64 (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", 2014) of the counter seed + step 2^32 + i,
// reduced modulo n; the same (seed, step) always draws the same batch.
__global__ void k_mlp_batch(uint64_t seed, int64_t step, int64_t n, int B, int32_t* __restrict__ idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  uint64_t z = seed + (uint64_t(step) << 32) + uint64_t(i) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  idx[i] = int32_t(z % uint64_t(n));
}

// Sum of squares of the n targets (FP64), for the RMS output scale.
__global__ void k_mlp_sumsq(const float* __restrict__ t, int64_t n, double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc += double(t[i]) * double(t[i]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Training targets of the learned correction: row 4 i + f (point i, field f = u, v, w, phi_t)
// gets (exact_f - lagrange_f) / s_f and field id f.
__global__ void k_mlp_targets(const float* __restrict__ eu, const float* __restrict__ ev,
                              const float* __restrict__ ew, const float* __restrict__ et,
                              const float* __restrict__ lag, const float* __restrict__ sc, int64_t np,
                              float* __restrict__ target, int32_t* __restrict__ field) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= 4 * np) return;
  const int64_t i = r >> 2;
  const int f = int(r & 3);
  const float ex = f == 0 ? eu[i] : f == 1 ? ev[i] : f == 2 ? ew[i] : et[i];
  target[r] = (ex - lag[r]) / sc[r];
  field[r] = f;
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

namespace {

constexpr int kWgradSlice = 256;

// Workspace layout of one training step for batch B (after `base` bytes the caller keeps).
struct StepWs {
  float *grad, *h1, *h2, *dz1, *dz2, *dy, *part, *loss_part;
  int32_t* idx;
  unsigned blocks;
  int nslices;
};
size_t step_ws_bytes(int B) {
  const unsigned blocks = unsigned(std::min<int64_t>((int64_t(B) + 63) / 64, 152 * 16));
  const int nslices = (B + kWgradSlice - 1) / kWgradSlice;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(NPARAM * sizeof(float)) + 4 * al(size_t(B) * NH * sizeof(float)) + al(size_t(B) * 4 * sizeof(float)) +
         al(size_t(nslices) * NPARAM * sizeof(float)) + al(blocks * sizeof(float)) + al(size_t(B) * sizeof(int32_t));
}
StepWs step_ws(void* ws, int B) {
  StepWs w{};
  w.blocks = unsigned(std::min<int64_t>((int64_t(B) + 63) / 64, 152 * 16));
  w.nslices = (B + kWgradSlice - 1) / kWgradSlice;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* c = static_cast<char*>(ws);
  w.grad = reinterpret_cast<float*>(c);
  c += al(NPARAM * sizeof(float));
  w.h1 = reinterpret_cast<float*>(c);
  c += al(size_t(B) * NH * sizeof(float));
  w.h2 = reinterpret_cast<float*>(c);
  c += al(size_t(B) * NH * sizeof(float));
  w.dz1 = reinterpret_cast<float*>(c);
  c += al(size_t(B) * NH * sizeof(float));
  w.dz2 = reinterpret_cast<float*>(c);
  c += al(size_t(B) * NH * sizeof(float));
  w.dy = reinterpret_cast<float*>(c);
  c += al(size_t(B) * 4 * sizeof(float));
  w.part = reinterpret_cast<float*>(c);
  c += al(size_t(w.nslices) * NPARAM * sizeof(float));
  w.loss_part = reinterpret_cast<float*>(c);
  c += al(w.blocks * sizeof(float));
  w.idx = reinterpret_cast<int32_t*>(c);
  return w;
}

// Forward + backward of batch rows `batch` into w.grad (and *loss if non-NULL), in a fixed order.
int grad_into(const StepWs& w, const void* packed, const float* x, const int32_t* field, const float* target,
              float tscale, const int32_t* batch, int B, float* loss, cudaStream_t stream) {
  TrainArgs a{static_cast<const Packed*>(packed), x, field, target, batch, B, w.h1, w.h2, w.dz1, w.dz2, w.dy,
              w.loss_part, tscale};
  k_mlp_train_fb<<<w.blocks, 128, 0, stream>>>(a);
  SWENSE_CUDA_TRY(cudaGetLastError());
  k_mlp_wgrad<<<dim3((NPARAM + 255) / 256, w.nslices), 256, 0, stream>>>(x, batch, B, w.h1, w.h2, w.dz1, w.dz2,
                                                                        w.dy, kWgradSlice, w.part);
  SWENSE_CUDA_TRY(cudaGetLastError());
  k_mlp_reduce<<<(NPARAM + 255) / 256, 256, 0, stream>>>(w.part, w.nslices, w.grad, w.loss_part, int(w.blocks),
                                                         loss);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(3);
  return SWENSE_OK;
}

// One Adam step (1-based `step`) on the gradient in w.grad, then the packed copy.
int adam_and_pack(const StepWs& w, float* params, float* adam_m, float* adam_v, void* packed, int64_t step,
                  float lr, float beta1, float beta2, float eps, cudaStream_t stream) {
  const double t = double(step);
  k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, stream>>>(params, adam_m, adam_v, w.grad, lr, beta1, beta2, eps,
                                                        float(1.0 - std::pow(double(beta1), t)),
                                                        float(1.0 - std::pow(double(beta2), t)));
  SWENSE_CUDA_TRY(cudaGetLastError());
  k_mlp_pack<<<(NH * KIN + 255) / 256, 256, 0, stream>>>(params, static_cast<Packed*>(packed));
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(2);
  return SWENSE_OK;
}

}  // namespace

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
  void* ws = nullptr;
  int st = workspace(step_ws_bytes(B), stream, &ws);
  if (st) return st;
  const StepWs w = step_ws(ws, B);
  st = grad_into(w, packed, x, field, target, 1.f, batch, B, loss, stream);
  if (!st) st = adam_and_pack(w, params, adam_m, adam_v, packed, step, lr, beta1, beta2, eps, stream);
  return st;
}

extern "C" int swense_mlp_grad(const void* packed, const float* x, const int32_t* field,
                               const float* target, const int32_t* batch, int32_t B, float* grad,
                               float* loss, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!packed || !x || !field || !target || !batch || !grad) return fail(SWENSE_ERR_ARG, "NULL argument");
  if (B < 1 || B > (1 << 24)) return fail(SWENSE_ERR_ARG, "batch size must be in [1, 2^24]");
  void* ws = nullptr;
  int st = workspace(step_ws_bytes(B), stream, &ws);
  if (st) return st;
  StepWs w = step_ws(ws, B);
  w.grad = grad;                                 // the caller's buffer receives the sums
  return grad_into(w, packed, x, field, target, 1.f, batch, B, loss, stream);
}

extern "C" int swense_mlp_targets(const float* exact_u, const float* exact_v, const float* exact_w,
                                  const float* exact_phit, const float* lagrange, const float* scale,
                                  int64_t np, float* target, int32_t* field, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (np < 0) return fail(SWENSE_ERR_ARG, "np must be >= 0");
  if (np == 0) return SWENSE_OK;
  if (!exact_u || !exact_v || !exact_w || !exact_phit || !lagrange || !scale || !target || !field)
    return fail(SWENSE_ERR_ARG, "NULL argument");
  k_mlp_targets<<<unsigned((4 * np + 255) / 256), 256, 0, stream>>>(exact_u, exact_v, exact_w, exact_phit,
                                                                   lagrange, scale, np, target, field);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

extern "C" int swense_mlp_train(swense_mlp* mlp, const float* x, const int32_t* field, const float* target,
                                int64_t n_rows, int32_t steps, int32_t B, float lr, int64_t schedule_steps,
                                float beta1, float beta2, float eps, float* losses, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!mlp || !mlp->params || !mlp->adam_m || !mlp->adam_v || !mlp->packed || !x || !field || !target)
    return fail(SWENSE_ERR_ARG, "NULL argument");
  if (n_rows < 1 || n_rows > (int64_t(1) << 31)) return fail(SWENSE_ERR_ARG, "n_rows must be in [1, 2^31]");
  if (steps < 0 || B < 1 || B > (1 << 24)) return fail(SWENSE_ERR_ARG, "steps >= 0, batch in [1, 2^24]");
  if (!(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0) || mlp->step < 0)
    return fail(SWENSE_ERR_ARG, "bad Adam hyper-parameters or step");
  if (reinterpret_cast<uintptr_t>(mlp->packed) & 15) return fail(SWENSE_ERR_ARG, "packed must be 16-byte aligned");
  void* ws = nullptr;
  int st = workspace(step_ws_bytes(B) + 256, stream, &ws);
  if (st) return st;
  const StepWs w = step_ws(ws, B);
  if (!(mlp->out_scale > 0)) {
    // the output scale: RMS of the raw targets (the network then trains on O(1) values)
    double* acc = reinterpret_cast<double*>(static_cast<char*>(ws) + step_ws_bytes(B));
    SWENSE_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double), stream));
    k_mlp_sumsq<<<unsigned(std::min<int64_t>((n_rows + 255) / 256, 152 * 8)), 256, 0, stream>>>(target, n_rows, acc);
    SWENSE_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    double ss = 0.0;
    SWENSE_CUDA_TRY(cudaMemcpyAsync(&ss, acc, sizeof(double), cudaMemcpyDeviceToHost, stream));
    SWENSE_CUDA_TRY(cudaStreamSynchronize(stream));
    const double rms = std::sqrt(ss / double(n_rows));
    mlp->out_scale = rms > 0 ? float(rms) : 1.f;
    st = swense_mlp_pack(mlp->params, mlp->out_scale, mlp->packed, stream_);
    if (st) return st;
  }
  const float tscale = 1.f / mlp->out_scale;
  for (int32_t i = 0; i < steps; ++i) {
    const int64_t s = mlp->step;                 // steps already taken
    k_mlp_batch<<<(B + 255) / 256, 256, 0, stream>>>(mlp->seed, s, n_rows, B, w.idx);
    SWENSE_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    double lr_s = lr;
    if (schedule_steps > 0)
      lr_s = lr * 0.5 * (1.0 + std::cos(3.14159265358979323846 * double(std::min(s, schedule_steps)) /
                                        double(schedule_steps)));
    st = grad_into(w, mlp->packed, x, field, target, tscale, w.idx, B, losses ? losses + i : nullptr, stream);
    if (!st) st = adam_and_pack(w, mlp->params, mlp->adam_m, mlp->adam_v, mlp->packed, s + 1,
                                float(std::max(lr_s, 1e-30)), beta1, beta2, eps, stream);
    if (st) return st;
    mlp->step = s + 1;
  }
  return SWENSE_OK;
}

// Checkpoint, little-endian: "SWMLP002", int64 step, uint64 seed, int64 nparam, float64
// out_scale, then params, Adam m, Adam v as float32.
extern "C" int swense_mlp_save(const swense_mlp* mlp, const char* path, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!mlp || !path || !mlp->params || !mlp->adam_m || !mlp->adam_v) return fail(SWENSE_ERR_ARG, "NULL argument");
  std::vector<float> buf(3 * size_t(NPARAM));
  const float* src[3] = {mlp->params, mlp->adam_m, mlp->adam_v};
  for (int q = 0; q < 3; ++q)
    SWENSE_CUDA_TRY(cudaMemcpyAsync(buf.data() + size_t(q) * NPARAM, src[q], NPARAM * sizeof(float),
                                    cudaMemcpyDeviceToHost, stream));
  SWENSE_CUDA_TRY(cudaStreamSynchronize(stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(SWENSE_ERR_ARG, std::string("cannot open ") + path + " for writing");
  const int64_t step = mlp->step, np = NPARAM;
  const uint64_t seed = mlp->seed;
  const double os = mlp->out_scale;
  bool ok = std::fwrite("SWMLP002", 1, 8, f) == 8 && std::fwrite(&step, 8, 1, f) == 1 &&
            std::fwrite(&seed, 8, 1, f) == 1 && std::fwrite(&np, 8, 1, f) == 1 && std::fwrite(&os, 8, 1, f) == 1 &&
            std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(SWENSE_ERR_ARG, std::string("writing ") + path + " failed");
  return SWENSE_OK;
}

extern "C" int swense_mlp_load(swense_mlp* mlp, const char* path, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!mlp || !path || !mlp->params || !mlp->adam_m || !mlp->adam_v || !mlp->packed)
    return fail(SWENSE_ERR_ARG, "NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(SWENSE_ERR_ARG, std::string("cannot open ") + path);
  char magic[8];
  int64_t step = 0, np = 0;
  uint64_t seed = 0;
  double os = 0.0;
  std::vector<float> buf(3 * size_t(NPARAM));
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "SWMLP002", 8) == 0 &&
            std::fread(&step, 8, 1, f) == 1 && std::fread(&seed, 8, 1, f) == 1 && std::fread(&np, 8, 1, f) == 1 &&
            np == NPARAM && std::fread(&os, 8, 1, f) == 1 &&
            std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok || step < 0 || !(os > 0) || !std::isfinite(os))
    return fail(SWENSE_ERR_ARG, std::string(path) + " is not a swense MLP checkpoint (SWMLP002)");
  float* dst[3] = {mlp->params, mlp->adam_m, mlp->adam_v};
  for (int q = 0; q < 3; ++q)
    SWENSE_CUDA_TRY(cudaMemcpyAsync(dst[q], buf.data() + size_t(q) * NPARAM, NPARAM * sizeof(float),
                                    cudaMemcpyHostToDevice, stream));
  mlp->step = step;
  mlp->seed = seed;
  mlp->out_scale = float(os);
  return swense_mlp_pack(mlp->params, mlp->out_scale, mlp->packed, stream_);   // synchronises
}
