// Finite-volume divergence of the reconstructed face-centre velocity (paper: subsection
// "Reconstruction error: velocity divergence": div u_I = sum_f u_I,f . A_f / dV, with the face
// average replaced by the face-centre value).
//
// One thread per cell; the cell's six signed face references make the sum deterministic (no
// atomics), so repeated calls give bit-identical results.
#include <algorithm>

#include "internal.cuh"

namespace swense {
namespace {

__global__ void __launch_bounds__(256) k_fv_divergence(const float* __restrict__ u,
                                                       const float* __restrict__ v,
                                                       const float* __restrict__ w,
                                                       const float* __restrict__ area,
                                                       const int* __restrict__ cell_faces,
                                                       const float* __restrict__ vol,
                                                       int64_t nc, float* __restrict__ div) {
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < nc;
       c += int64_t(gridDim.x) * blockDim.x) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int r = __ldg(&cell_faces[6 * c + j]);
      const int64_t f = int64_t(r > 0 ? r : -r) - 1;
      const float flux = fmaf(__ldg(&u[f]), __ldg(&area[3 * f]),
                              fmaf(__ldg(&v[f]), __ldg(&area[3 * f + 1]),
                                   __ldg(&w[f]) * __ldg(&area[3 * f + 2])));
      acc += r > 0 ? flux : -flux;
    }
    div[c] = acc / __ldg(&vol[c]);
  }
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_fv_divergence(const float* u_face, const float* v_face, const float* w_face,
                                    int64_t n_faces, const float* area, const int32_t* cell_faces,
                                    const float* cell_volume, int64_t n_cells, float* div,
                                    void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (n_cells < 0 || n_faces < 0) return fail(SWENSE_ERR_ARG, "negative sizes");
  if (n_cells == 0) return SWENSE_OK;
  if (!u_face || !v_face || !w_face || !area || !cell_faces || !cell_volume || !div)
    return fail(SWENSE_ERR_ARG, "NULL input or output");
  if (n_faces == 0) return fail(SWENSE_ERR_ARG, "cells need faces");
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((n_cells + threads - 1) / threads, int64_t(1) << 30);
  k_fv_divergence<<<unsigned(blocks), threads, 0, stream>>>(u_face, v_face, w_face, area, cell_faces,
                                                            cell_volume, n_cells, div);
  SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
  return SWENSE_OK;
}
