// Wave-tank (wall-bounded) modes onto the periodic transform pipeline.
//
// Paper: the HOS-NWT solver reproduces a rectangular tank with perfectly reflective side walls,
// so its horizontal basis is cos(m pi x / Lx) cos(n pi y / Ly) instead of e^{i k.x}. A cosine
// series on [0, Lx] x [0, Ly] is the Fourier series of its even extension over the doubled
// domain [0, 2 Lx) x [0, 2 Ly): wavenumbers m pi / Lx = 2 pi m / (2 Lx), and
//   A cos(kx x) cos(ky y) = Re[(A/2) e^{i(kx x + ky y)} + (A/2) e^{i(kx x - ky y)}],
// so each real tank amplitude becomes two (or one, on an axis) coefficients of the one-sided
// half-spectrum. The tank nodes x_i = i Lx / (nx_t - 1) are the first nx_t nodes of that
// periodic grid, and near a wall the gather's stencil reads the mirrored nodes, which hold the
// even (eta, phi, w, dphi/dt) or odd (the wall-normal velocity) extension the walls impose. The
// transforms are the periodic ones on nx = 2 (nx_t - 1) points: a type-1 cosine transform done as
// a real transform of the even extension. The highest tank mode of each axis is that grid's
// Nyquist mode, which the pipeline leaves out.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace swense {
namespace {

// One thread per output slot [snap][r][m], m in 0..nx/2, r in FFT row order.
__global__ void __launch_bounds__(256) k_tank_modes(const float* __restrict__ ae, const float* __restrict__ ap,
                                                    const float* __restrict__ at, int nx_t, int ny_t,
                                                    int nx, int ny, int64_t total, float2* __restrict__ oe,
                                                    float2* __restrict__ op, float2* __restrict__ ot) {
  const int nh1 = nx / 2 + 1;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int m = int(i % nh1);
    const int64_t rest = i / nh1;
    const int r = int(rest % ny);
    const int64_t snap = rest / ny;
    const int n = ny == 1 ? 0 : (r < ny / 2 ? r : r - ny);   // signed row wavenumber index
    const int nt = n < 0 ? -n : n;                       // tank index along y
    // coefficient of one signed slot: A for (0, 0), A/2 on an axis, A/4 off both axes
    const float f = (m == 0 ? 1.f : 0.5f) * (ny > 1 && nt != 0 ? 0.5f : 1.f);
    const int64_t src = (snap * ny_t + nt) * nx_t + m;
    oe[i] = make_float2(f * __ldg(&ae[src]), 0.f);
    op[i] = make_float2(f * __ldg(&ap[src]), 0.f);
    ot[i] = make_float2(f * __ldg(&at[src]), 0.f);
  }
}

bool pow2_in(int64_t v, int64_t lo, int64_t hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_tank_modes(const float* A_eta, const float* A_phi, const float* A_phit, int32_t nx_t,
                                 int32_t ny_t, int32_t n_snap, double Lx, double Ly, double depth,
                                 float* out_eta, float* out_phi, float* out_phit, swense_modes* out,
                                 void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!out) return fail(SWENSE_ERR_ARG, "NULL output modes");
  if (nx_t < 3 || !pow2_in(2 * int64_t(nx_t - 1), 4, SWENSE_MAX_FFT))
    return fail(SWENSE_ERR_SIZE, "2 (nx_t - 1) must be a power of two in [4, SWENSE_MAX_FFT]");
  if (ny_t != 1 && (ny_t < 3 || !pow2_in(2 * int64_t(ny_t - 1), 4, SWENSE_MAX_FFT)))
    return fail(SWENSE_ERR_SIZE, "ny_t must be 1 or have 2 (ny_t - 1) a power of two in [4, SWENSE_MAX_FFT]");
  if (n_snap < 1 || n_snap > SWENSE_MAX_TL) return fail(SWENSE_ERR_ARG, "n_snap must lie in 1..SWENSE_MAX_TL");
  if (!(Lx > 0.0) || !std::isfinite(Lx) || (ny_t > 1 && (!(Ly > 0.0) || !std::isfinite(Ly))))
    return fail(SWENSE_ERR_ARG, "tank lengths must be positive and finite");
  if (!std::isfinite(depth)) return fail(SWENSE_ERR_ARG, "depth must be finite (<= 0 for deep water)");
  if (!A_eta || !A_phi || !A_phit || !out_eta || !out_phi || !out_phit)
    return fail(SWENSE_ERR_ARG, "NULL amplitude array");
  if ((reinterpret_cast<uintptr_t>(out_eta) | reinterpret_cast<uintptr_t>(out_phi) |
       reinterpret_cast<uintptr_t>(out_phit)) & 7)
    return fail(SWENSE_ERR_ARG, "complex outputs must be 8-byte aligned");
  const int nx = 2 * (nx_t - 1), ny = ny_t > 1 ? 2 * (ny_t - 1) : 1;
  const int64_t total = int64_t(n_snap) * ny * (nx / 2 + 1);
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, int64_t(1) << 30);
  k_tank_modes<<<unsigned(blocks), threads, 0, stream>>>(
      A_eta, A_phi, A_phit, nx_t, ny_t, nx, ny, total, reinterpret_cast<float2*>(out_eta),
      reinterpret_cast<float2*>(out_phi), reinterpret_cast<float2*>(out_phit));
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  swense_modes& m = *out;
  m.nx = nx;
  m.ny = ny;
  m.Lx = 2.0 * Lx;
  m.Ly = ny_t > 1 ? 2.0 * Ly : 1.0;
  m.depth = depth;
  m.n_snap = n_snap;
  m.A_eta = out_eta;
  m.A_phi = out_phi;
  m.A_phit = out_phit;
  m.omega = nullptr;
  m.t_ref = 0.0;
  return SWENSE_OK;
}
