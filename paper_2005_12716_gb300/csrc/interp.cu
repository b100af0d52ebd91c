// Stage 2 of the reconstruction: grid fields -> arbitrary points (cell and face centres).
//
// Paper: reconstruction section, step "Interpolation" (HOS grid -> CFD mesh). Scheme: tensor
// product 4-point Lagrange in x, y (uniform, periodic) and z (arbitrary levels, stencil shifted
// inside the level range at the ends), Lagrange over the stored time levels, then Bernoulli.
//
// One thread per point. The point's horizontal cell is located with a compensated FP32 product
// (x * nx_r / Lx as hi + lo) so the in-cell offset keeps ~1e-7 absolute accuracy even for points
// hundreds of cells from the origin. The 4x4x4 (x TL) float4 stencil loads go through L1/L2:
// points arrive in mesh order, so neighbouring threads share most of their stencil lines.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace swense {
namespace {

struct Levels {
  float z[SWENSE_MAX_LEVELS];
};

struct InterpArgs {
  const float4* nodes;   // [TL][nz][Nyr][Nxr]
  const float* eta;      // [TL][Nyr][Nxr]
  const float* pts;      // [np][3]
  float* o_eta;
  float* o_u;
  float* o_v;
  float* o_w;
  float* o_p;
  unsigned long long* n_oor;
  int64_t np;
  int Nxr, Nyr, nz, n_tl;
  float sx_hi, sx_lo, sy_hi, sy_lo;   // nx_r / Lx and ny_r / Ly as hi + lo
  float wt[SWENSE_MAX_TL];            // time weights
  int p_mode;
  float rho, g;
};

// Cell index (mod n) and in-cell offset f in [0, 1] of coordinate x for the node spacing
// 1 / (s_hi + s_lo); the product is carried as an unevaluated sum (fma residual).
__device__ __forceinline__ void locate(float x, float s_hi, float s_lo, int n, int& i0, float& f) {
  const float p = x * s_hi;
  const float e = fmaf(x, s_hi, -p);
  const float lo = fmaf(x, s_lo, e);
  const float fl = floorf(p);
  f = (p - fl) + lo;
  int i = int(fl);
  if (f < 0.f) {
    f += 1.f;
    i -= 1;
  } else if (f >= 1.f) {
    f -= 1.f;
    i += 1;
  }
  i0 = i & (n - 1);
}

// Lagrange basis of the nodes -1, 0, 1, 2 at f.
__device__ __forceinline__ void lagrange4_uniform(float f, float w[4]) {
  const float fm1 = f - 1.f, fm2 = f - 2.f, fp1 = f + 1.f;
  w[0] = -f * fm1 * fm2 * (1.f / 6.f);
  w[1] = 0.5f * fp1 * fm1 * fm2;
  w[2] = -0.5f * fp1 * f * fm2;
  w[3] = fp1 * f * fm1 * (1.f / 6.f);
}

// Lagrange basis of the 4 arbitrary nodes zn at z.
__device__ __forceinline__ void lagrange4(const float zn[4], float z, float w[4]) {
  const float d0 = z - zn[0], d1 = z - zn[1], d2 = z - zn[2], d3 = z - zn[3];
  w[0] = (d1 * d2 * d3) / ((zn[0] - zn[1]) * (zn[0] - zn[2]) * (zn[0] - zn[3]));
  w[1] = (d0 * d2 * d3) / ((zn[1] - zn[0]) * (zn[1] - zn[2]) * (zn[1] - zn[3]));
  w[2] = (d0 * d1 * d3) / ((zn[2] - zn[0]) * (zn[2] - zn[1]) * (zn[2] - zn[3]));
  w[3] = (d0 * d1 * d2) / ((zn[3] - zn[0]) * (zn[3] - zn[1]) * (zn[3] - zn[2]));
}

__global__ void __launch_bounds__(256, 3) k_interp(InterpArgs a, Levels L) {
  __shared__ float zs[SWENSE_MAX_LEVELS];
  for (int i = threadIdx.x; i < a.nz; i += blockDim.x) zs[i] = L.z[i];
  __syncthreads();
  const int nz = a.nz;
  const size_t plane = size_t(a.Nyr) * a.Nxr;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.np;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float x = a.pts[3 * i], y = a.pts[3 * i + 1], z = a.pts[3 * i + 2];
    int ix;
    float fx, wx[4];
    locate(x, a.sx_hi, a.sx_lo, a.Nxr, ix, fx);
    lagrange4_uniform(fx, wx);
    int xi[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) xi[c] = (ix - 1 + c) & (a.Nxr - 1);
    int yi[4] = {0, 0, 0, 0};
    float wy[4] = {1.f, 0.f, 0.f, 0.f};
    const int nys = a.Nyr > 1 ? 4 : 1;
    if (a.Nyr > 1) {
      int iy;
      float fy;
      locate(y, a.sy_hi, a.sy_lo, a.Nyr, iy, fy);
      lagrange4_uniform(fy, wy);
#pragma unroll
      for (int b = 0; b < 4; ++b) yi[b] = (iy - 1 + b) & (a.Nyr - 1);
    }
    // bracket: largest j with zs[j] <= z, clamped to [0, nz-2]; stencil j0 = clamp(j-1, 0, nz-4)
    const bool inside = (z >= zs[0]) && (z <= zs[nz - 1]);
    int lo = 0, hi = nz;  // first index with zs[idx] > z
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (zs[mid] <= z) lo = mid + 1; else hi = mid;
    }
    int j = lo - 1;
    j = min(max(j, 0), nz - 2);
    const int j0 = min(max(j - 1, 0), nz - 4);
    float zn[4], wz[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) zn[q] = zs[j0 + q];
    lagrange4(zn, z, wz);

    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    float acc_eta = 0.f;
    for (int tl = 0; tl < a.n_tl; ++tl) {
      const float wtl = a.wt[tl];
      const float4* base_t = a.nodes + size_t(tl) * nz * plane;
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        const float4* lev = base_t + size_t(j0 + q) * plane;
        const float wzq = wtl * wz[q];
        for (int b = 0; b < nys; ++b) {
          const float4* row = lev + size_t(yi[b]) * a.Nxr;
          const float wzy = wzq * wy[b];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 gv = __ldg(&row[xi[c]]);
            const float ww = wzy * wx[c];
            acc.x = fmaf(ww, gv.x, acc.x);
            acc.y = fmaf(ww, gv.y, acc.y);
            acc.z = fmaf(ww, gv.z, acc.z);
            acc.w = fmaf(ww, gv.w, acc.w);
          }
        }
      }
      const float* et = a.eta + size_t(tl) * plane;
      for (int b = 0; b < nys; ++b) {
        const float* row = et + size_t(yi[b]) * a.Nxr;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc_eta = fmaf(wtl * wy[b] * wx[c], __ldg(&row[xi[c]]), acc_eta);
      }
    }
    if (!inside) {
      const float qnan = __int_as_float(0x7fc00000);
      acc = make_float4(qnan, qnan, qnan, qnan);
      if (a.n_oor) atomicAdd(a.n_oor, 1ULL);
    }
    if (a.o_eta) a.o_eta[i] = acc_eta;
    if (a.o_u) a.o_u[i] = acc.x;
    if (a.o_v) a.o_v[i] = acc.y;
    if (a.o_w) a.o_w[i] = acc.z;
    if (a.o_p) {
      float p;
      if (a.p_mode == SWENSE_P_PHIT) {
        p = acc.w;
      } else {
        const float q2 = acc.x * acc.x + acc.y * acc.y + acc.z * acc.z;
        p = -a.rho * (acc.w + 0.5f * q2);
        if (a.p_mode == SWENSE_P_TOTAL) p -= a.rho * a.g * z;
      }
      a.o_p[i] = p;
    }
  }
}

void split(double v, float& hi, float& lo) {
  hi = float(v);
  lo = float(v - double(hi));
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_interp(const swense_grid* g, double t, const float* pts, int64_t np,
                             float* eta, float* u, float* v, float* w, float* p, int32_t p_mode,
                             double rho, double grav, int64_t* n_out_of_range, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!g || !g->nodes || !g->eta || !g->z_levels || !g->t_levels)
    return fail(SWENSE_ERR_ARG, "NULL grid, grid arrays or level lists");
  if (np < 0) return fail(SWENSE_ERR_ARG, "np must be >= 0");
  if (np > 0 && !pts) return fail(SWENSE_ERR_ARG, "NULL pts");
  if (!is_pow2(g->nx_r) || g->nx_r < 4 || g->nx_r > SWENSE_MAX_FFT || !is_pow2(g->ny_r) ||
      (g->ny_r != 1 && g->ny_r < 4) || g->ny_r > SWENSE_MAX_FFT)
    return fail(SWENSE_ERR_SIZE, "nx_r must be a power of two in [4, MAX], ny_r 1 or a power of two in [4, MAX]");
  if (g->nz < 4 || g->nz > SWENSE_MAX_LEVELS) return fail(SWENSE_ERR_LEVELS, "need 4 <= nz <= SWENSE_MAX_LEVELS");
  if (g->n_tl < 1 || g->n_tl > SWENSE_MAX_TL) return fail(SWENSE_ERR_ARG, "n_tl must be in [1, SWENSE_MAX_TL]");
  if (p_mode != SWENSE_P_DYN && p_mode != SWENSE_P_PHIT && p_mode != SWENSE_P_TOTAL)
    return fail(SWENSE_ERR_ARG, "unknown p_mode");
  if (!(g->Lx > 0) || !std::isfinite(g->Lx) || (g->ny_r > 1 && (!(g->Ly > 0) || !std::isfinite(g->Ly))))
    return fail(SWENSE_ERR_ARG, "domain lengths must be finite and positive");
  if (!std::isfinite(t) || !std::isfinite(rho) || !std::isfinite(grav))
    return fail(SWENSE_ERR_ARG, "non-finite t, rho or g");
  if (reinterpret_cast<uintptr_t>(g->nodes) & 15) return fail(SWENSE_ERR_ARG, "nodes must be 16-byte aligned");
  Levels lev;
  for (int l = 0; l < g->nz; ++l) {
    lev.z[l] = g->z_levels[l];
    if (!std::isfinite(lev.z[l]) || (l > 0 && !(lev.z[l] > lev.z[l - 1])))
      return fail(SWENSE_ERR_LEVELS, "z_levels must be finite and strictly increasing");
  }
  InterpArgs a{};
  for (int l = 0; l < g->n_tl; ++l) {
    if (!std::isfinite(g->t_levels[l]) || (l > 0 && !(g->t_levels[l] > g->t_levels[l - 1])))
      return fail(SWENSE_ERR_ARG, "t_levels must be finite and strictly increasing");
  }
  // Lagrange weights over the time levels, in FP64 on the host
  for (int l = 0; l < g->n_tl; ++l) {
    double wl = 1.0;
    for (int m = 0; m < g->n_tl; ++m)
      if (m != l) wl *= (t - g->t_levels[m]) / (g->t_levels[l] - g->t_levels[m]);
    a.wt[l] = float(wl);
  }
  unsigned long long* d_count = nullptr;
  if (n_out_of_range) {
    void* ws = nullptr;
    int st = workspace(256, stream, &ws);
    if (st) return st;
    d_count = static_cast<unsigned long long*>(ws);
    SWENSE_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream));
  }
  if (np > 0) {
    a.nodes = reinterpret_cast<const float4*>(g->nodes);
    a.eta = g->eta;
    a.pts = pts;
    a.o_eta = eta;
    a.o_u = u;
    a.o_v = v;
    a.o_w = w;
    a.o_p = p;
    a.n_oor = d_count;
    a.np = np;
    a.Nxr = g->nx_r;
    a.Nyr = g->ny_r;
    a.nz = g->nz;
    a.n_tl = g->n_tl;
    split(double(g->nx_r) / g->Lx, a.sx_hi, a.sx_lo);
    if (g->ny_r > 1) split(double(g->ny_r) / g->Ly, a.sy_hi, a.sy_lo);
    a.p_mode = p_mode;
    a.rho = float(rho);
    a.g = float(grav);
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((np + threads - 1) / threads, int64_t(1) << 30);
    k_interp<<<unsigned(blocks), threads, 0, stream>>>(a, lev);
    SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
  }
  if (n_out_of_range) {
    unsigned long long h = 0;
    SWENSE_CUDA_TRY(cudaMemcpyAsync(&h, d_count, sizeof(h), cudaMemcpyDeviceToHost, stream));
    SWENSE_CUDA_TRY(cudaStreamSynchronize(stream));
    *n_out_of_range = int64_t(h);
  }
  return SWENSE_OK;
}
