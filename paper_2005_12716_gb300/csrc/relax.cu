// Incident VOF fraction and relaxation-zone blending on CFD cells.
//
// Paper: subsection on the prevention of wave reflections with the relaxation zone technique.
// A cell's relaxation weight is w = -2x^3 + 3x^2 (Eq. weightFunction) of its non-dimensional
// distance x into a zone; the complementary velocity is blended to zero (Eq. swUcRelax) and the
// VOF fraction to the incident one (Eq. swVOFRelax), both instances of Eq. relaxationZone. The
// incident fraction alpha_I comes from the incident elevation eta_I (reconstruction section,
// interpolation step): the surface is taken as horizontal across the cell at eta_I of its centre,
// and alpha_I is the part of the cell's vertical extent below it.
//
// Cells over threads, grid-stride, several per thread; the zones are a kernel parameter. Cells
// outside every zone (w = 0) keep alpha and u_C as they are and are not rewritten, so the kernel
// writes little beyond alpha_I in the body of the domain.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace swense {
namespace {

struct Zones {
  int n;
  int kind[SWENSE_MAX_ZONES];
  float inner[SWENSE_MAX_ZONES], inv_len[SWENSE_MAX_ZONES], cx[SWENSE_MAX_ZONES], cy[SWENSE_MAX_ZONES];
};

// clamp to [0, 1] that keeps NaN
__device__ __forceinline__ float unit_clamp(float x) { return x < 0.f ? 0.f : (x > 1.f ? 1.f : x); }

__device__ __forceinline__ float zone_weight(const Zones& Z, float x, float y) {
  float w = 0.f;
  for (int k = 0; k < Z.n; ++k) {
    float s;
    if (Z.kind[k] == SWENSE_ZONE_X) s = x;
    else if (Z.kind[k] == SWENSE_ZONE_Y) s = y;
    else s = sqrtf((x - Z.cx[k]) * (x - Z.cx[k]) + (y - Z.cy[k]) * (y - Z.cy[k]));
    const float xn = unit_clamp((s - Z.inner[k]) * Z.inv_len[k]);
    w = fmaxf(w, xn * xn * (3.f - 2.f * xn));
  }
  return w;
}

// Each thread takes CPT cells a grid stride apart and issues all their loads before using any,
// so a thread keeps several DRAM requests in flight.
constexpr int CPT = 4;

__global__ void __launch_bounds__(256) k_relax_cells(const float* __restrict__ xyz,
                                                     const float2* __restrict__ zext,
                                                     const float* __restrict__ eta, int64_t nc,
                                                     Zones Z, float* __restrict__ alpha_i,
                                                     float* __restrict__ alpha,
                                                     float* __restrict__ uc,
                                                     float* __restrict__ weight) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t c0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c0 < nc; c0 += CPT * stride) {
    float x[CPT], y[CPT], e[CPT];
    float2 ze[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int64_t c = c0 + k * stride;
      if (c < nc) {
        x[k] = __ldg(&xyz[3 * c]);
        y[k] = __ldg(&xyz[3 * c + 1]);
        ze[k] = __ldg(&zext[c]);
        e[k] = __ldg(&eta[c]);
      }
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int64_t c = c0 + k * stride;
      if (c >= nc) break;
      const float w = zone_weight(Z, x[k], y[k]);
      const float ai = unit_clamp((e[k] - ze[k].x) / (ze[k].y - ze[k].x));
      if (alpha_i) alpha_i[c] = ai;
      if (weight) weight[c] = w;
      if (w > 0.f) {
        const float keep = 1.f - w;
        if (alpha) alpha[c] = fmaf(w, ai, keep * alpha[c]);
        if (uc) {
          uc[3 * c] *= keep;
          uc[3 * c + 1] *= keep;
          uc[3 * c + 2] *= keep;
        }
      }
    }
  }
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_relax_cells(const float* cell_xyz, const float* cell_zext, const float* eta_c,
                                  int64_t nc, const swense_relax_zone* zones, int32_t n_zones,
                                  float* alpha_i, float* alpha, float* u_c, float* weight,
                                  void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (nc < 0) return fail(SWENSE_ERR_ARG, "negative cell count");
  if (n_zones < 0 || n_zones > SWENSE_MAX_ZONES)
    return fail(SWENSE_ERR_ARG, "n_zones must lie in 0..SWENSE_MAX_ZONES");
  if (n_zones > 0 && !zones) return fail(SWENSE_ERR_ARG, "NULL zones");
  Zones Z{};
  Z.n = n_zones;
  for (int k = 0; k < n_zones; ++k) {
    const swense_relax_zone& z = zones[k];
    if (z.kind != SWENSE_ZONE_X && z.kind != SWENSE_ZONE_Y && z.kind != SWENSE_ZONE_RADIAL)
      return fail(SWENSE_ERR_ARG, "unknown zone kind");
    if (!(std::isfinite(z.inner) && std::isfinite(z.outer)) || z.inner == z.outer)
      return fail(SWENSE_ERR_ARG, "zone boundaries must be finite and distinct");
    Z.kind[k] = z.kind;
    Z.inner[k] = z.inner;
    Z.inv_len[k] = float(1.0 / (double(z.outer) - double(z.inner)));
    Z.cx[k] = z.cx;
    Z.cy[k] = z.cy;
  }
  if (nc == 0) return SWENSE_OK;
  if (!cell_xyz || !cell_zext || !eta_c) return fail(SWENSE_ERR_ARG, "NULL input");
  if (reinterpret_cast<uintptr_t>(cell_zext) & 7) return fail(SWENSE_ERR_ARG, "cell_zext must be 8-byte aligned");
  // one resident wave (SMs x resident blocks per SM), or fewer blocks for small meshes: every
  // thread then loops, keeping the memory system busy without a tail of partial waves
  const int threads = 256;
  int dev = 0, sms = 0, per_sm = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  SWENSE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SWENSE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax_cells, threads, 0));
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((nc + threads * CPT - 1) / (threads * CPT),
                                                                int64_t(sms) * std::max(per_sm, 1)));
  k_relax_cells<<<unsigned(blocks), threads, 0, stream>>>(
      cell_xyz, reinterpret_cast<const float2*>(cell_zext), eta_c, nc, Z, alpha_i, alpha, u_c, weight);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}
