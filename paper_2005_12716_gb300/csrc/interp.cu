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

// Stencil of one point: cell indices, Lagrange weights and the in-range flag.
struct PointCell {
  int ix, iy, j0;       // first stencil node in x, y (before the -1 shift) and first level
  float wx[4], wy[4], wz[4];
  bool inside;
};

__device__ __forceinline__ PointCell point_cell(const InterpArgs& a, const float* zs, float x,
                                                float y, float z) {
  PointCell c;
  float fx;
  locate(x, a.sx_hi, a.sx_lo, a.Nxr, c.ix, fx);
  lagrange4_uniform(fx, c.wx);
  c.iy = 0;
  c.wy[0] = 1.f;
  c.wy[1] = c.wy[2] = c.wy[3] = 0.f;
  if (a.Nyr > 1) {
    float fy;
    locate(y, a.sy_hi, a.sy_lo, a.Nyr, c.iy, fy);
    lagrange4_uniform(fy, c.wy);
  }
  // bracket: largest j with zs[j] <= z, clamped to [0, nz-2]; stencil j0 = clamp(j-1, 0, nz-4)
  const int nz = a.nz;
  c.inside = (z >= zs[0]) && (z <= zs[nz - 1]);
  int lo = 0, hi = nz;  // first index with zs[idx] > z
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (zs[mid] <= z) lo = mid + 1; else hi = mid;
  }
  const int j = min(max(lo - 1, 0), nz - 2);
  c.j0 = min(max(j - 1, 0), nz - 4);
  float zn[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) zn[q] = zs[c.j0 + q];
  lagrange4(zn, z, c.wz);
  return c;
}

// Stencil sums straight from global memory (L1/L2), all time levels.
__device__ __forceinline__ void gather_global(const InterpArgs& a, const PointCell& c, float4& acc,
                                              float& acc_eta) {
  const size_t plane = size_t(a.Nyr) * a.Nxr;
  const int nys = a.Nyr > 1 ? 4 : 1;
  int xi[4], yi[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    xi[q] = (c.ix - 1 + q) & (a.Nxr - 1);
    yi[q] = a.Nyr > 1 ? ((c.iy - 1 + q) & (a.Nyr - 1)) : 0;
  }
  acc = make_float4(0.f, 0.f, 0.f, 0.f);
  acc_eta = 0.f;
  for (int tl = 0; tl < a.n_tl; ++tl) {
    const float wtl = a.wt[tl];
    const float4* base_t = a.nodes + size_t(tl) * a.nz * plane;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      const float4* lev = base_t + size_t(c.j0 + q) * plane;
      const float wzq = wtl * c.wz[q];
      for (int b = 0; b < nys; ++b) {
        const float4* row = lev + size_t(yi[b]) * a.Nxr;
        const float wzy = wzq * c.wy[b];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 gv = __ldg(&row[xi[k]]);
          const float ww = wzy * c.wx[k];
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
      for (int k = 0; k < 4; ++k) acc_eta = fmaf(wtl * c.wy[b] * c.wx[k], __ldg(&row[xi[k]]), acc_eta);
    }
  }
}

__device__ __forceinline__ void store_point(const InterpArgs& a, int64_t i, float4 acc,
                                            float acc_eta, float z, bool inside) {
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

// One thread per point, stencils read from global memory. Used for scattered point sets.
__global__ void __launch_bounds__(256, 3) k_interp(InterpArgs a, Levels L) {
  __shared__ float zs[SWENSE_MAX_LEVELS];
  for (int i = threadIdx.x; i < a.nz; i += blockDim.x) zs[i] = L.z[i];
  __syncthreads();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.np;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float x = a.pts[3 * i], y = a.pts[3 * i + 1], z = a.pts[3 * i + 2];
    const PointCell c = point_cell(a, zs, x, y, z);
    float4 acc;
    float acc_eta;
    gather_global(a, c, acc, acc_eta);
    store_point(a, i, acc, acc_eta, z, c.inside);
  }
}

// Box-staged gather for spatially coherent point sets (mesh order). Each CTA takes BOX_PTS
// consecutive points, finds the bounding box of their stencils, loads that box of the grid into
// shared memory already blended in time (sum_t w_t G_t, exact reordering of the linear sums),
// then evaluates every point from shared memory, where threads of a warp mostly share cells
// (broadcast reads). A CTA whose box exceeds BOX_NODES falls back to global gathers.
constexpr int BOX_THREADS = 256;
constexpr int BOX_PPT = 2;                         // points per thread
constexpr int BOX_PTS = BOX_THREADS * BOX_PPT;
constexpr int BOX_NODES = 4096;                    // float4 nodes (64 KB)
constexpr int BOX_COLS = 2048;                     // eta columns (8 KB)
constexpr size_t BOX_SMEM = size_t(BOX_NODES) * sizeof(float4) + size_t(BOX_COLS) * sizeof(float);

__device__ __forceinline__ int wrap_rel(int i, int ref, int n) {
  // i - ref folded into [-n/2, n/2)
  return ((i - ref + (n >> 1)) & (n - 1)) - (n >> 1);
}

__global__ void __launch_bounds__(BOX_THREADS, 3) k_interp_box(InterpArgs a, Levels L) {
  extern __shared__ float4 sbox[];
  float* seta = reinterpret_cast<float*>(sbox + BOX_NODES);
  __shared__ float zs[SWENSE_MAX_LEVELS];
  __shared__ int s_red[6][BOX_THREADS / 32];
  __shared__ int s_ref[2];
  for (int i = threadIdx.x; i < a.nz; i += blockDim.x) zs[i] = L.z[i];
  const int64_t p0 = int64_t(blockIdx.x) * BOX_PTS;
  __syncthreads();
  if (threadIdx.x == 0) {
    const PointCell c = point_cell(a, zs, a.pts[3 * p0], a.pts[3 * p0 + 1], a.pts[3 * p0 + 2]);
    s_ref[0] = c.ix;
    s_ref[1] = c.iy;
  }
  PointCell cell[BOX_PPT];
  float zq[BOX_PPT];
  int rx[BOX_PPT], ry[BOX_PPT];
  __syncthreads();
  const int refx = s_ref[0], refy = s_ref[1];
  int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
#pragma unroll
  for (int k = 0; k < BOX_PPT; ++k) {
    const int64_t i = p0 + k * BOX_THREADS + threadIdx.x;
    if (i < a.np) {
      zq[k] = a.pts[3 * i + 2];
      cell[k] = point_cell(a, zs, a.pts[3 * i], a.pts[3 * i + 1], zq[k]);
      rx[k] = wrap_rel(cell[k].ix, refx, a.Nxr);
      ry[k] = a.Nyr > 1 ? wrap_rel(cell[k].iy, refy, a.Nyr) : 0;
      mn[0] = min(mn[0], rx[k]);
      mx[0] = max(mx[0], rx[k]);
      mn[1] = min(mn[1], ry[k]);
      mx[1] = max(mx[1], ry[k]);
      mn[2] = min(mn[2], cell[k].j0);
      mx[2] = max(mx[2], cell[k].j0);
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[d] = min(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
      mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      s_red[d][warp] = mn[d];
      s_red[3 + d][warp] = mx[d];
    }
  }
  __syncthreads();
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    mn[d] = s_red[d][0];
    mx[d] = s_red[3 + d][0];
    for (int w = 1; w < BOX_THREADS / 32; ++w) {
      mn[d] = min(mn[d], s_red[d][w]);
      mx[d] = max(mx[d], s_red[3 + d][w]);
    }
  }
  // box: x nodes rel (mn0-1) .. (mx0+2), y likewise (one row in 2-D), levels mn2 .. mx2+3
  const int bx = mx[0] - mn[0] + 4;
  const int by = a.Nyr > 1 ? mx[1] - mn[1] + 4 : 1;
  const int bz = mx[2] - mn[2] + 4;
  const bool fits = int64_t(bx) * by * bz <= BOX_NODES && int64_t(bx) * by <= BOX_COLS &&
                    bx <= a.Nxr && by <= a.Nyr;
  if (fits) {
    const size_t plane = size_t(a.Nyr) * a.Nxr;
    const int x0 = refx + mn[0] - 1, y0 = a.Nyr > 1 ? refy + mn[1] - 1 : 0, l0 = mn[2];
    const int nbox = bx * by * bz;
    for (int idx = threadIdx.x; idx < nbox; idx += BOX_THREADS) {
      const int lx = idx % bx;
      const int rest = idx / bx;
      const int ly = rest % by, lz = rest / by;
      const size_t g = size_t(l0 + lz) * plane + size_t((y0 + ly) & (a.Nyr - 1)) * a.Nxr +
                       ((x0 + lx) & (a.Nxr - 1));
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int tl = 0; tl < a.n_tl; ++tl) {
        const float4 gv = __ldg(&a.nodes[size_t(tl) * a.nz * plane + g]);
        const float w = a.wt[tl];
        v.x = fmaf(w, gv.x, v.x);
        v.y = fmaf(w, gv.y, v.y);
        v.z = fmaf(w, gv.z, v.z);
        v.w = fmaf(w, gv.w, v.w);
      }
      sbox[idx] = v;
    }
    for (int idx = threadIdx.x; idx < bx * by; idx += BOX_THREADS) {
      const int lx = idx % bx, ly = idx / bx;
      const size_t g = size_t((y0 + ly) & (a.Nyr - 1)) * a.Nxr + ((x0 + lx) & (a.Nxr - 1));
      float v = 0.f;
      for (int tl = 0; tl < a.n_tl; ++tl) v = fmaf(a.wt[tl], __ldg(&a.eta[size_t(tl) * plane + g]), v);
      seta[idx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BOX_PPT; ++k) {
      const int64_t i = p0 + k * BOX_THREADS + threadIdx.x;
      if (i >= a.np) continue;
      const PointCell& c = cell[k];
      const int ox = rx[k] - mn[0], oy = ry[k] - mn[1], oz = c.j0 - mn[2];
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      float acc_eta = 0.f;
      const int nys = a.Nyr > 1 ? 4 : 1;
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        for (int b = 0; b < nys; ++b) {
          const float4* row = sbox + ((oz + q) * by + (oy + b)) * bx + ox;
          const float wzy = c.wz[q] * c.wy[b];
#pragma unroll
          for (int kx = 0; kx < 4; ++kx) {
            const float4 gv = row[kx];
            const float ww = wzy * c.wx[kx];
            acc.x = fmaf(ww, gv.x, acc.x);
            acc.y = fmaf(ww, gv.y, acc.y);
            acc.z = fmaf(ww, gv.z, acc.z);
            acc.w = fmaf(ww, gv.w, acc.w);
          }
        }
      }
      for (int b = 0; b < nys; ++b) {
        const float* row = seta + (oy + b) * bx + ox;
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) acc_eta = fmaf(c.wy[b] * c.wx[kx], row[kx], acc_eta);
      }
      store_point(a, i, acc, acc_eta, zq[k], c.inside);
    }
  } else {
#pragma unroll
    for (int k = 0; k < BOX_PPT; ++k) {
      const int64_t i = p0 + k * BOX_THREADS + threadIdx.x;
      if (i >= a.np) continue;
      float4 acc;
      float acc_eta;
      gather_global(a, cell[k], acc, acc_eta);
      store_point(a, i, acc, acc_eta, zq[k], cell[k].inside);
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
    const int64_t blocks = (np + BOX_PTS - 1) / BOX_PTS;
    if (blocks >= (int64_t(1) << 31)) return fail(SWENSE_ERR_SIZE, "too many points for one call");
    SWENSE_CUDA_TRY(cudaFuncSetAttribute((const void*)k_interp_box,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(BOX_SMEM)));
    k_interp_box<<<unsigned(blocks), BOX_THREADS, BOX_SMEM, stream>>>(a, lev);
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
