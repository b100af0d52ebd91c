// Direct ("analytical") evaluation of the modal sums at arbitrary points.
//
// Paper: reconstruction section, subsection on the analytical evaluation of u_I and w_I
// (substituting the point coordinates into the modal sums; cost proportional to the number of
// Fourier components per point), with the spectral decomposition of Eqs. whatIsSpectralMethod1
// and whatIsSpectralMethod and Bernoulli for the pressure. Used for small mode counts and for
// near-body points that must not carry interpolation error.
//
// FP32 path: one thread per point, modes streamed through shared memory in tiles (every lane
// reads the same mode: broadcast). The phase k.x is carried as an exact 32-bit fraction of a
// turn: per point X = frac(x / Lx) * 2^32 and Y = frac(y / Ly) * 2^32 (formed in FP64 once per
// point), per mode the integer product m X + n Y (mod 2^32), so the argument error does not grow
// with |k x|. Depth factors use a compensated |k| z product. Sums are accumulated per tile and
// then added to the running totals to limit FP32 round-off growth over many modes.
#include <algorithm>
#include <cmath>

#include "fft.cuh"
#include "internal.cuh"

namespace swense {
namespace {

// Coefficients of one mode, 64 bytes:
//   c0 = (m, n as int bits, |k|, 1 / (1 + e^{-2|k|h}) or 1 in deep water)
//   c1 = (W_eta, W_u), c2 = (W_v, W_w), c3 = (W_t, 0, 0)
// with W_eta = c A^eta, W_u = c i kx A^phi, W_v = c i ky A^phi, W_w = c |k| A^phi,
// W_t = c A^phit and c = 1 for m = 0, 2 otherwise (one-sided spectrum weights).
struct ModeCoef {
  float4 c0, c1, c2, c3;
};

__global__ void k_direct_prep(const float2* __restrict__ Ae, const float2* __restrict__ Ap,
                              const float2* __restrict__ At, const double* __restrict__ omega,
                              double dt, int nx, int ny, float kxs, float kys, float depth,
                              ModeCoef* __restrict__ out) {
  const int nxh1 = nx / 2 + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ny * nxh1) return;
  const int r = i / nxh1, m = i - r * nxh1;
  ModeCoef mc;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  mc.c0 = make_float4(__int_as_float(0), __int_as_float(0), 0.f, 1.f);
  mc.c1 = mc.c2 = mc.c3 = zero;
  if (m >= nx / 2 || (ny > 1 && r == ny / 2)) {           // Nyquist slots are ignored
    out[i] = mc;
    return;
  }
  float2 e = Ae[i], p = Ap[i], t = At[i];
  if (omega) {
    const double turns = omega[i] * dt * 0.15915494309189533577;
    const double frac = turns - rint(turns);
    float s, c;
    sincospif(2.f * float(frac), &s, &c);
    e = make_float2(fmaf(e.x, c, e.y * s), fmaf(e.y, c, -e.x * s));
    p = make_float2(fmaf(p.x, c, p.y * s), fmaf(p.y, c, -p.x * s));
    t = make_float2(fmaf(t.x, c, t.y * s), fmaf(t.y, c, -t.x * s));
  }
  const int n = ny > 1 ? (r < ny / 2 ? r : r - ny) : 0;
  const float kx = float(m) * kxs, ky = float(n) * kys;
  const float k = sqrtf(kx * kx + ky * ky);
  const float wgt = m == 0 ? 1.f : 2.f;
  const float invd = depth > 0.f ? 1.f / (1.f + expf(-2.f * k * depth)) : 1.f;
  mc.c0 = make_float4(__int_as_float(m), __int_as_float(n), k, invd);
  mc.c1 = make_float4(wgt * e.x, wgt * e.y, -wgt * kx * p.y, wgt * kx * p.x);
  mc.c2 = make_float4(-wgt * ky * p.y, wgt * ky * p.x, wgt * k * p.x, wgt * k * p.y);
  mc.c3 = make_float4(wgt * t.x, wgt * t.y, 0.f, 0.f);
  out[i] = mc;
}

constexpr int kDirThreads = 256;
constexpr int kDirTile = 256;   // modes per shared-memory tile

struct DirectArgs {
  const ModeCoef* modes;
  unsigned n_modes;
  const float* pts;
  float *o_eta, *o_u, *o_v, *o_w, *o_p;
  int64_t np;
  double inv_lx, inv_ly;
  float depth;
  int p_mode;
  float rho, g;
};

// x / L as an unsigned 32-bit fraction of a turn.
__device__ __forceinline__ unsigned turn_fraction(float x, double inv_l) {
  const double f = double(x) * inv_l;
  const double fr = f - floor(f);                        // [0, 1)
  return unsigned((unsigned long long)(fr * 4294967296.0) & 0xffffffffull);
}

__global__ void __launch_bounds__(kDirThreads) k_direct_fp32(DirectArgs a) {
  __shared__ ModeCoef tile[kDirTile];
  const unsigned nm = a.n_modes;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool live = i < a.np;
  float x = 0.f, y = 0.f, z = 0.f;
  if (live) {
    x = a.pts[3 * i];
    y = a.pts[3 * i + 1];
    z = a.pts[3 * i + 2];
  }
  const unsigned X = turn_fraction(x, a.inv_lx), Y = turn_fraction(y, a.inv_ly);
  const float h = a.depth;
  // e^{i 2 pi x / Lx}: the phase step from mode m to m + 1 along a row (same n)
  float sstep, cstep;
  sincospif(2.f * (float(int(X)) * 2.3283064365386963e-10f), &sstep, &cstep);
  int prev_m = -2, prev_n = 0, run = 0;
  float sn = 0.f, cs = 1.f;
  float s_eta = 0.f, s_u = 0.f, s_v = 0.f, s_w = 0.f, s_t = 0.f;
  for (unsigned base = 0; base < nm; base += kDirTile) {
    const unsigned cnt = min(unsigned(kDirTile), nm - base);
    __syncthreads();
    for (unsigned j = threadIdx.x; j < cnt; j += blockDim.x) tile[j] = a.modes[base + j];
    __syncthreads();
    float t_eta = 0.f, t_u = 0.f, t_v = 0.f, t_w = 0.f, t_t = 0.f;
    for (unsigned j = 0; j < cnt; ++j) {
      const float4 c0 = tile[j].c0, c1 = tile[j].c1, c2 = tile[j].c2, c3 = tile[j].c3;
      const int m = __float_as_int(c0.x), n = __float_as_int(c0.y);
      if (m == prev_m + 1 && n == prev_n && run < 15) {
        // consecutive mode of the same row: advance the phase by the per-point step
        const float c2 = fmaf(cs, cstep, -sn * sstep);
        sn = fmaf(sn, cstep, cs * sstep);
        cs = c2;
        ++run;
      } else {
        // exact phase m X + n Y (mod 2^32) every 16 modes and at row starts
        const unsigned ph = unsigned(m) * X + unsigned(n) * Y;
        const float turns = float(int(ph)) * 2.3283064365386963e-10f;   // 2^-32, in [-0.5, 0.5)
        sincospif(2.f * turns, &sn, &cs);
        run = 0;
      }
      prev_m = m;
      prev_n = n;
      const float k = c0.z;
      float F, S;
      depth_factors(k, z, h, F, S);
      t_eta = fmaf(c1.x, cs, fmaf(-c1.y, sn, t_eta));
      t_u = fmaf(F, fmaf(c1.z, cs, -c1.w * sn), t_u);
      t_v = fmaf(F, fmaf(c2.x, cs, -c2.y * sn), t_v);
      t_w = fmaf(S, fmaf(c2.z, cs, -c2.w * sn), t_w);
      t_t = fmaf(F, fmaf(c3.x, cs, -c3.y * sn), t_t);
    }
    s_eta += t_eta;
    s_u += t_u;
    s_v += t_v;
    s_w += t_w;
    s_t += t_t;
  }
  if (!live) return;
  if (a.o_eta) a.o_eta[i] = s_eta;
  if (a.o_u) a.o_u[i] = s_u;
  if (a.o_v) a.o_v[i] = s_v;
  if (a.o_w) a.o_w[i] = s_w;
  if (a.o_p) {
    float p;
    if (a.p_mode == SWENSE_P_PHIT) {
      p = s_t;
    } else {
      p = -a.rho * (s_t + 0.5f * (s_u * s_u + s_v * s_v + s_w * s_w));
      if (a.p_mode == SWENSE_P_TOTAL) p -= a.rho * a.g * z;
    }
    a.o_p[i] = p;
  }
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_direct(const swense_modes* md, double t, const float* pts, int64_t np,
                             float* eta, float* u, float* v, float* w, float* p, int32_t p_mode,
                             double rho, double grav, int32_t precision, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!md || !md->A_eta || !md->A_phi || !md->A_phit) return fail(SWENSE_ERR_ARG, "NULL modes");
  if (np < 0) return fail(SWENSE_ERR_ARG, "np must be >= 0");
  if (np > 0 && !pts) return fail(SWENSE_ERR_ARG, "NULL pts");
  const int nx = md->nx, ny = md->ny;
  if (!is_pow2(nx) || nx < 4 || !is_pow2(ny) || (ny != 1 && ny < 4) || nx > (1 << 16) || ny > (1 << 16))
    return fail(SWENSE_ERR_SIZE, "nx must be a power of two in [4, 65536], ny 1 or a power of two in [4, 65536]");
  if (md->n_snap != 1) return fail(SWENSE_ERR_ARG, "swense_direct takes one snapshot (n_snap = 1)");
  if (!(md->Lx > 0) || !std::isfinite(md->Lx) || (ny > 1 && (!(md->Ly > 0) || !std::isfinite(md->Ly))))
    return fail(SWENSE_ERR_ARG, "domain lengths must be finite and positive");
  if (!std::isfinite(t) || !std::isfinite(md->depth) || !std::isfinite(rho) || !std::isfinite(grav))
    return fail(SWENSE_ERR_ARG, "non-finite t, depth, rho or g");
  if (p_mode != SWENSE_P_DYN && p_mode != SWENSE_P_PHIT && p_mode != SWENSE_P_TOTAL)
    return fail(SWENSE_ERR_ARG, "unknown p_mode");
  if (precision != SWENSE_DIRECT_FP32)
    return fail(SWENSE_ERR_UNSUPPORTED, "precision: only SWENSE_DIRECT_FP32 is implemented");
  if (np == 0) return SWENSE_OK;
  const size_t nslot = size_t(ny) * (nx / 2 + 1);
  const size_t bytes = nslot * sizeof(ModeCoef);
  void* ws = nullptr;
  int st = workspace(bytes, stream, &ws);
  if (st) return st;
  ModeCoef* modes = static_cast<ModeCoef*>(ws);
  const float depth = md->depth > 0 ? float(md->depth) : 0.f;
  k_direct_prep<<<unsigned((nslot + 255) / 256), 256, 0, stream>>>(
      reinterpret_cast<const float2*>(md->A_eta), reinterpret_cast<const float2*>(md->A_phi),
      reinterpret_cast<const float2*>(md->A_phit), md->omega, t - md->t_ref, nx, ny,
      float(6.283185307179586476925 / md->Lx), ny > 1 ? float(6.283185307179586476925 / md->Ly) : 0.f,
      depth, modes);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  DirectArgs a{};
  a.modes = modes;
  a.n_modes = unsigned(nslot);
  a.pts = pts;
  a.o_eta = eta;
  a.o_u = u;
  a.o_v = v;
  a.o_w = w;
  a.o_p = p;
  a.np = np;
  a.inv_lx = 1.0 / md->Lx;
  a.inv_ly = ny > 1 ? 1.0 / md->Ly : 0.0;
  a.depth = depth;
  a.p_mode = p_mode;
  a.rho = float(rho);
  a.g = float(grav);
  const int64_t blocks = (np + kDirThreads - 1) / kDirThreads;
  if (blocks >= (int64_t(1) << 31)) return fail(SWENSE_ERR_SIZE, "too many points for one call");
  k_direct_fp32<<<unsigned(blocks), kDirThreads, 0, stream>>>(a);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}
