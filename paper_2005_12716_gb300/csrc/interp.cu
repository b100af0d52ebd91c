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
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "mlp.cuh"

namespace swense {
namespace {

// z lookup: ZLUT equal buckets over [z_0, z_{nz-1}]; lut[b] = largest level index j with
// z_j <= z_0 + b h. A point starts its search one bucket below its own (so rounding of the
// bucket index cannot place it past its level) and steps up: one or two steps for any level
// spacing that is not much finer than h.
constexpr int ZLUT = 256;

// Level tables, built on the host once per call and passed as a kernel parameter: levels,
// inverse Lagrange denominators of each 4-level window (inv[j] for nodes j..j+3) and the lookup.
struct Levels {
  float z[SWENSE_MAX_LEVELS];
  float4 inv[SWENSE_MAX_LEVELS];
  unsigned lut4[ZLUT / 4];          // lut bytes, four per word
  float z0, inv_h;
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
  const int32_t* perm;   // output index of each point (NULL: identity); points are pre-sorted
  int64_t np;
  int Nxr, Nyr, nz, n_tl;
  float sx_hi, sx_lo, sy_hi, sy_lo;   // nx_r / Lx and ny_r / Ly as hi + lo
  float wt[SWENSE_MAX_TL];            // time weights
  int p_mode;
  float rho, g;
  int spline;            // cubic B-spline weights in x and y (grid holds spline coefficients)
  int p2;                // both node counts are powers of two (mask wrap; the kernels' <true>)
};

// Periodic node index i mod n. Grids whose horizontal node counts are powers of two (every
// grid zero-padded by a power of two) wrap with a mask; the others (padding factors 3, 5, 6, 7)
// take the remainder. The kernels are instantiated for both, so the mask path is unchanged.
template <bool P2>
__device__ __forceinline__ int wrapi(int i, int n) {
  if constexpr (P2) {
    return i & (n - 1);
  } else {
    const int r = i % n;
    return r < 0 ? r + n : r;
  }
}

// Cell index (mod n) and in-cell offset f in [0, 1] of coordinate x for the node spacing
// 1 / (s_hi + s_lo); the product is carried as an unevaluated sum (fma residual).
template <bool P2 = true>
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
  i0 = wrapi<P2>(i, n);
}

// Uniform cubic B-spline basis of the coefficients -1, 0, 1, 2 at f.
__device__ __forceinline__ void bspline4(float f, float w[4]) {
  const float g = 1.f - f, f2 = f * f, f3 = f2 * f;
  w[0] = g * g * g * (1.f / 6.f);
  w[1] = fmaf(0.5f * f3, 1.f, fmaf(-f2, 1.f, 2.f / 3.f));      // (3f^3 - 6f^2 + 4) / 6
  w[2] = fmaf(-0.5f, f3, fmaf(0.5f, f2, fmaf(0.5f, f, 1.f / 6.f)));   // (-3f^3 + 3f^2 + 3f + 1) / 6
  w[3] = f3 * (1.f / 6.f);
}

// Lagrange basis of the nodes -1, 0, 1, 2 at f.
__device__ __forceinline__ void lagrange4_uniform(float f, float w[4]) {
  const float fm1 = f - 1.f, fm2 = f - 2.f, fp1 = f + 1.f;
  w[0] = -f * fm1 * fm2 * (1.f / 6.f);
  w[1] = 0.5f * fp1 * fm1 * fm2;
  w[2] = -0.5f * fp1 * f * fm2;
  w[3] = fp1 * f * fm1 * (1.f / 6.f);
}

// Lagrange basis of the 4 arbitrary nodes zn at z; inv holds 1 / prod_{b != a} (zn[a] - zn[b]).
__device__ __forceinline__ void lagrange4(const float zn[4], float4 inv, float z, float w[4]) {
  const float d0 = z - zn[0], d1 = z - zn[1], d2 = z - zn[2], d3 = z - zn[3];
  w[0] = (d1 * d2 * d3) * inv.x;
  w[1] = (d0 * d2 * d3) * inv.y;
  w[2] = (d0 * d1 * d3) * inv.z;
  w[3] = (d0 * d1 * d2) * inv.w;
}

// Shared-memory copy of the levels and, per stencil start j0, the inverse Lagrange
// denominators of the levels j0 .. j0+3 (computed once per CTA: no divisions per point).
struct LevelTables {
  float z[SWENSE_MAX_LEVELS];
  float4 inv[SWENSE_MAX_LEVELS];
  alignas(4) unsigned char lut[ZLUT];
  float z0, inv_h;
};

// Copy of the level tables in shared memory (per-thread indices would serialise on the
// parameter bank).
__device__ __forceinline__ void fill_level_tables(LevelTables& T, const Levels& L, int nz) {
  if (threadIdx.x == 0) {
    T.z0 = L.z0;
    T.inv_h = L.inv_h;
  }
  for (int i = threadIdx.x; i < ZLUT / 4; i += blockDim.x) reinterpret_cast<unsigned*>(T.lut)[i] = L.lut4[i];
  for (int i = threadIdx.x; i < nz; i += blockDim.x) T.z[i] = L.z[i];
  for (int j = threadIdx.x; j <= nz - 4; j += blockDim.x) T.inv[j] = L.inv[j];
}

struct PointCell {
  int ix, iy, j0;       // first stencil node in x, y (before the -1 shift) and first level
  float wx[4], wy[4], wz[4];
  bool inside;
};

// Horizontal part of a point's cell: first stencil nodes and weights in x and y.
template <bool P2 = true>
__device__ __forceinline__ void point_xy(const InterpArgs& a, float x, float y, PointCell& c) {
  float fx;
  locate<P2>(x, a.sx_hi, a.sx_lo, a.Nxr, c.ix, fx);
  if (a.spline) bspline4(fx, c.wx); else lagrange4_uniform(fx, c.wx);
  c.iy = 0;
  c.wy[0] = 1.f;
  c.wy[1] = c.wy[2] = c.wy[3] = 0.f;
  if (a.Nyr > 1) {
    float fy;
    locate<P2>(y, a.sy_hi, a.sy_lo, a.Nyr, c.iy, fy);
    if (a.spline) bspline4(fy, c.wy); else lagrange4_uniform(fy, c.wy);
  }
}

// Vertical part: first stencil level j0, level weights and whether z lies inside the levels.
__device__ __forceinline__ void point_level(const InterpArgs& a, const LevelTables& T, float z,
                                            PointCell& c) {
  const float* zs = T.z;
  // bracket: largest j with zs[j] <= z, clamped to [0, nz-2]; stencil j0 = clamp(j-1, 0, nz-4)
  const int nz = a.nz;
  c.inside = (z >= zs[0]) && (z <= zs[nz - 1]);
  const float bf = fminf(fmaxf((z - T.z0) * T.inv_h, 0.f), float(ZLUT - 1));   // NaN -> 0
  int jj = T.lut[max(int(bf) - 1, 0)];
  while (jj + 1 < nz && zs[jj + 1] <= z) ++jj;
  const int j = min(jj, nz - 2);
  c.j0 = min(max(j - 1, 0), nz - 4);
  float zn[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) zn[q] = zs[c.j0 + q];
  lagrange4(zn, T.inv[c.j0], z, c.wz);
}

template <bool P2 = true>
__device__ __forceinline__ PointCell point_cell(const InterpArgs& a, const LevelTables& T, float x,
                                                float y, float z) {
  PointCell c;
  point_xy<P2>(a, x, y, c);
  point_level(a, T, z, c);
  return c;
}

// Stencil sums straight from global memory (L1/L2), all time levels.
template <bool P2 = true>
__device__ __forceinline__ void gather_global(const InterpArgs& a, const PointCell& c, float4& acc,
                                              float& acc_eta) {
  const size_t plane = size_t(a.Nyr) * a.Nxr;
  const int nys = a.Nyr > 1 ? 4 : 1;
  int xi[4], yi[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    xi[q] = wrapi<P2>(c.ix - 1 + q, a.Nxr);
    yi[q] = a.Nyr > 1 ? wrapi<P2>(c.iy - 1 + q, a.Nyr) : 0;
  }
  acc = make_float4(0.f, 0.f, 0.f, 0.f);
  acc_eta = 0.f;
  for (int tl = 0; tl < a.n_tl; ++tl) {
    const float wtl = a.wt[tl];
    const float4* base_t = a.nodes + size_t(tl) * a.nz * plane;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      const float4* lev = base_t + size_t(c.j0 + q) * plane;
      // select instead of a dynamic index so the weights stay in registers
      const float wzq = wtl * (q == 0 ? c.wz[0] : q == 1 ? c.wz[1] : q == 2 ? c.wz[2] : c.wz[3]);
#pragma unroll 1
      for (int b = 0; b < nys; ++b) {
        const int yb = b == 0 ? yi[0] : b == 1 ? yi[1] : b == 2 ? yi[2] : yi[3];
        const float wyb = b == 0 ? c.wy[0] : b == 1 ? c.wy[1] : b == 2 ? c.wy[2] : c.wy[3];
        const float4* row = lev + size_t(yb) * a.Nxr;
        const float wzy = wzq * wyb;
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
#pragma unroll 1
    for (int b = 0; b < nys; ++b) {
      const int yb = b == 0 ? yi[0] : b == 1 ? yi[1] : b == 2 ? yi[2] : yi[3];
      const float wyb = b == 0 ? c.wy[0] : b == 1 ? c.wy[1] : b == 2 ? c.wy[2] : c.wy[3];
      const float* row = et + size_t(yb) * a.Nxr;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc_eta = fmaf(wtl * wyb * c.wx[k], __ldg(&row[xi[k]]), acc_eta);
    }
  }
}

__device__ __forceinline__ void store_point(const InterpArgs& a, int64_t i, float4 acc,
                                            float acc_eta, float z, bool inside) {
  if (a.perm) i = a.perm[i];
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

// Box-staged gather for spatially coherent point sets (mesh order). Each CTA takes BOX_PTS
// consecutive points, finds the bounding box of their stencils, loads that box of the grid into
// shared memory already blended in time (sum_t w_t G_t, exact reordering of the linear sums),
// then evaluates every point from shared memory, where threads of a warp mostly share cells
// (broadcast reads). A CTA whose box exceeds BOX_NODES falls back to global gathers.
constexpr int BOX_THREADS = 256;
constexpr int BOX_PPT = 4;                         // points per thread
constexpr int BOX_PTS = BOX_THREADS * BOX_PPT;
constexpr int BOX_NODES = 4096;                    // float4 nodes (64 KB; 99 % of the 1024-point mesh chunks fit)
constexpr int BOX_COLS = BOX_NODES / 4;             // eta columns (a box has at least 4 levels)
constexpr size_t BOX_SMEM = size_t(BOX_NODES) * sizeof(float4) + size_t(BOX_COLS) * sizeof(float);
// Level-flat chunks (every point at the same z, as the cell and face centres of one layer of an
// extruded mesh) stage one z-collapsed plane instead of the box: float4 columns and eta.
constexpr int FLAT_COLS = 3456;
static_assert(size_t(FLAT_COLS) * (sizeof(float4) + sizeof(float)) <= BOX_SMEM, "flat plane fits the tile");
// Chunks whose points lie at two z values (a chunk that straddles two layers) stage two
// collapsed planes and one eta plane.
constexpr int FLAT2_COLS = 1920;
static_assert(size_t(FLAT2_COLS) * (2 * sizeof(float4) + sizeof(float)) <= BOX_SMEM, "two planes fit the tile");

// One chunk's plan, 16 bytes: x0, y0 (first staged node, wrapped), l0 | FLAT_BIT, extents.
//   3-D box:  w = bx | by << 11 | bz << 22 (bz >= 4), z = l0
//   flat:     w = bx | by << 12 (4 levels from l0), z = l0 | FLAT_BIT
//   two z:    w = bx | by << 12, z = FLAT_BIT | FLAT2_BIT (the z values are those of the chunk's
//             first and last points; their level windows are looked up by the gather)
//   neither fits the tile: w = -1 (global gathers)
constexpr int FLAT_BIT = 1 << 30;
constexpr int FLAT2_BIT = 1 << 29;
struct BoxPlan {
  int x0, y0, l0, bx, by, bz;
  bool flat;     // z-collapsed plane
  bool two;      // two z-collapsed planes (flat is set too)
  bool box3d;    // the 3-D box fits BOX_NODES / BOX_COLS
};
__device__ __forceinline__ BoxPlan decode_plan(int4 pl) {
  BoxPlan b;
  b.x0 = pl.x;
  b.y0 = pl.y;
  b.flat = pl.w >= 0 && (pl.z & FLAT_BIT);
  b.two = b.flat && (pl.z & FLAT2_BIT);
  b.l0 = pl.z & 0xffff;
  if (b.flat) {
    b.bx = pl.w & 4095;
    b.by = (pl.w >> 12) & 4095;
    b.bz = 4;
  } else {
    b.bx = pl.w & 2047;
    b.by = (pl.w >> 11) & 2047;
    b.bz = (pl.w >> 22) & 511;
  }
  const int sbx = b.bx + ((4 - b.bx) & 7);
  b.box3d = pl.w >= 0 && !b.two && (!b.flat || (sbx * b.by * 4 <= BOX_NODES && sbx * b.by <= BOX_COLS));
  return b;
}

// Level-plane stride of the box (unpadded: padding it to separate z-neighbours' bank groups
// removed only 6 % of the wavefronts and made more chunks miss the tile).
__host__ __device__ __forceinline__ int box_zstride(int sbx, int by) { return by * sbx; }

template <bool P2 = true>
__device__ __forceinline__ int wrap_rel(int i, int ref, int n) {
  // i - ref folded into [-n/2, n/2)
  return wrapi<P2>(i - ref + (n >> 1), n) - (n >> 1);
}

// Two FP32 lanes packed in 64 bits for the Blackwell paired FMA (fma.rn.f32x2).
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  return (unsigned long long)__float_as_uint(a) | ((unsigned long long)__float_as_uint(b) << 32);
}
__device__ __forceinline__ void fma2(unsigned long long& acc, unsigned long long w, unsigned long long v) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(w), "l"(v));
}
__device__ __forceinline__ float lo2(unsigned long long v) { return __uint_as_float(unsigned(v)); }
__device__ __forceinline__ float hi2(unsigned long long v) { return __uint_as_float(unsigned(v >> 32)); }

// One stencil row of four staged nodes summed along x: (u, v) and (w, phi_t) pairs with the
// x weights given as (w, w) pairs, and (second form) the row's eta values with the same weights.
__device__ __forceinline__ void row_sum(const float4* row, const unsigned long long (&wx2)[4],
                                        unsigned long long& ruv, unsigned long long& rwt) {
  ruv = pack2(0.f, 0.f);
  rwt = pack2(0.f, 0.f);
#pragma unroll
  for (int kx = 0; kx < 4; ++kx) {
    const float4 gv = row[kx];
    fma2(ruv, wx2[kx], pack2(gv.x, gv.y));
    fma2(rwt, wx2[kx], pack2(gv.z, gv.w));
  }
}
__device__ __forceinline__ void row_sum(const float4* row, const float* erow,
                                        const unsigned long long (&wx2)[4], const float (&wx)[4],
                                        unsigned long long& ruv, unsigned long long& rwt, float& re) {
  row_sum(row, wx2, ruv, rwt);
  re = 0.f;
#pragma unroll
  for (int kx = 0; kx < 4; ++kx) re = fmaf(wx[kx], erow[kx], re);
}

// Time-blended box of grid nodes x0..x0+bx-1, y0..y0+by-1 (wrapped), levels l0..l0+bz-1 into
// shared memory (row stride sbx, level-plane stride zst float4), and the eta rows (stride sbx).
// Rows (ly, lz) over warps, two rows per warp at a time (more loads in flight), x over lanes;
// the time blend happens here, once per node.
template <bool P2 = true>
__device__ __forceinline__ void stage_box(const InterpArgs& a, int x0, int y0, int l0, int bx, int by,
                                          int bz, int sbx, int zst, float4* sbox, float* seta) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const size_t plane = size_t(a.Nyr) * a.Nxr;
  const size_t tl_stride = size_t(a.nz) * plane;
  const int nrows = by * bz;
  for (int r0 = warp; r0 < nrows; r0 += 2 * nw) {
    const int r1 = min(r0 + nw, nrows - 1);       // a duplicate of r0's last row when past the end
    const int lz0 = r0 / by, ly0 = r0 - lz0 * by, lz1 = r1 / by, ly1 = r1 - lz1 * by;
    const float4* src0 = a.nodes + size_t(l0 + lz0) * plane + size_t(wrapi<P2>(y0 + ly0, a.Nyr)) * a.Nxr;
    const float4* src1 = a.nodes + size_t(l0 + lz1) * plane + size_t(wrapi<P2>(y0 + ly1, a.Nyr)) * a.Nxr;
    for (int lx = lane; lx < bx; lx += 32) {
      const int gx = wrapi<P2>(x0 + lx, a.Nxr);
      float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
      for (int tl = 0; tl < a.n_tl; ++tl) {
        const float4 g0 = __ldg(&src0[size_t(tl) * tl_stride + gx]);
        const float4 g1 = __ldg(&src1[size_t(tl) * tl_stride + gx]);
        const float w = a.wt[tl];
        v0.x = fmaf(w, g0.x, v0.x);
        v0.y = fmaf(w, g0.y, v0.y);
        v0.z = fmaf(w, g0.z, v0.z);
        v0.w = fmaf(w, g0.w, v0.w);
        v1.x = fmaf(w, g1.x, v1.x);
        v1.y = fmaf(w, g1.y, v1.y);
        v1.z = fmaf(w, g1.z, v1.z);
        v1.w = fmaf(w, g1.w, v1.w);
      }
      sbox[lz0 * zst + ly0 * sbx + lx] = v0;
      sbox[lz1 * zst + ly1 * sbx + lx] = v1;       // same value when r1 repeats a row
    }
  }
  for (int ly = warp; ly < by; ly += nw) {
    const float* src = a.eta + size_t(wrapi<P2>(y0 + ly, a.Nyr)) * a.Nxr;
    for (int lx = lane; lx < bx; lx += 32) {
      const int gx = wrapi<P2>(x0 + lx, a.Nxr);
      float v = 0.f;
      for (int tl = 0; tl < a.n_tl; ++tl) v = fmaf(a.wt[tl], __ldg(&src[size_t(tl) * plane + gx]), v);
      seta[ly * sbx + lx] = v;
    }
  }
}

// Level-flat chunk: the z-collapsed, time-blended plane P = sum_t w_t sum_q wz_q G_t[l0 + q] of
// columns x0..x0+bx-1, y0..y0+by-1 (wrapped) into shared memory (row stride sbx), and the eta
// rows. Columns over all threads (index -> (ly, lx)), so every thread has 4 x n_tl node loads
// and n_tl eta loads of one column in flight.
template <bool P2 = true>
__device__ __forceinline__ void stage_plane(const InterpArgs& a, int x0, int y0, int l0, int bx,
                                            int by, int sbx, const float wz[4], float4* splane,
                                            float* seta, bool with_eta = true) {
  const size_t plane = size_t(a.Nyr) * a.Nxr;
  const size_t tl_stride = size_t(a.nz) * plane;
  const int ncol = bx * by;
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const int ly = c / bx, lx = c - ly * bx;
    const size_t col = size_t(wrapi<P2>(y0 + ly, a.Nyr)) * a.Nxr + wrapi<P2>(x0 + lx, a.Nxr);
    const float4* src = a.nodes + size_t(l0) * plane + col;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    float e = 0.f;
#pragma unroll
    for (int tl = 0; tl < SWENSE_MAX_TL; ++tl) {
      if (tl >= a.n_tl) break;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 g = __ldg(&src[size_t(tl) * tl_stride + size_t(q) * plane]);
        const float w = a.wt[tl] * wz[q];
        v.x = fmaf(w, g.x, v.x);
        v.y = fmaf(w, g.y, v.y);
        v.z = fmaf(w, g.z, v.z);
        v.w = fmaf(w, g.w, v.w);
      }
      if (with_eta) e = fmaf(a.wt[tl], __ldg(&a.eta[size_t(tl) * plane + col]), e);
    }
    splane[ly * sbx + lx] = v;
    if (with_eta) seta[ly * sbx + lx] = e;
  }
}

// Box plan of one 1024-point chunk: box origin (grid node indices, wrapped) and extents, or
// dims = -1 when the box does not fit the shared-memory tile (the chunk then gathers from
// global memory). Computed by its own kernel so the gather kernel can start its box load at
// once, without first waiting for its points. One warp per chunk (32 points per lane, loads
// coalesced across the lanes): the chunk's reductions stay in the warp, with no block barrier
// and no single-thread tail, and eight chunks of a block share one copy of the level tables.
constexpr int PLAN_WARPS = BOX_THREADS / 32;
__host__ __device__ __forceinline__ int64_t plan_blocks(int64_t np) {
  return ((np + BOX_PTS - 1) / BOX_PTS + PLAN_WARPS - 1) / PLAN_WARPS;
}

// Plan of chunk `chunk` of the points of `a`, by one warp (no block barrier).
template <bool P2>
__device__ __forceinline__ void plan_chunk(const InterpArgs& a, const LevelTables& zs, int64_t chunk,
                                           int4* __restrict__ plan, int lane) {
  const int64_t p0 = chunk * BOX_PTS;
  if (p0 >= a.np) return;
  // every lane derives the chunk's reference cell (its first point's) itself: broadcast loads
  int refx, refy, refj0;
  const float refz = __ldg(&a.pts[3 * p0 + 2]);
  {
    const PointCell c = point_cell<P2>(a, zs, __ldg(&a.pts[3 * p0]), __ldg(&a.pts[3 * p0 + 1]), refz);
    refx = c.ix;
    refy = c.iy;
    refj0 = c.j0;
  }
  int same_z = 1;                                   // every point of the chunk at z == refz (bitwise)
  int two_z = 1;                                    // every point at refz or at the last point's z
  const float lastz = __ldg(&a.pts[3 * ((p0 + BOX_PTS < a.np ? p0 + BOX_PTS : a.np) - 1) + 2]);
  int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  // four points per lane per round, their twelve loads issued before any of them is used
  constexpr int PU = 4;
  static_assert((BOX_PTS / 32) % PU == 0, "whole rounds");
#pragma unroll 1
  for (int k0 = 0; k0 < BOX_PTS / 32; k0 += PU) {
    float qx[PU], qy[PU], qz[PU];
#pragma unroll
    for (int u = 0; u < PU; ++u) {
      const int64_t i = p0 + (k0 + u) * 32 + lane;
      const int64_t ic = i < a.np ? i : a.np - 1;     // in-bounds duplicate past the end, unused
      qx[u] = __ldg(&a.pts[3 * ic]);
      qy[u] = __ldg(&a.pts[3 * ic + 1]);
      qz[u] = __ldg(&a.pts[3 * ic + 2]);
    }
#pragma unroll
    for (int u = 0; u < PU; ++u) {
      const int64_t i = p0 + (k0 + u) * 32 + lane;
      if (i < a.np) {
        const float pz = qz[u];
        PointCell c;
        point_xy<P2>(a, qx[u], qy[u], c);
        // the level window only where z differs from the chunk's first point (a layer of an
        // extruded mesh shares one z)
        const bool zeq = __float_as_int(pz) == __float_as_int(refz);
        same_z &= zeq;
        two_z &= zeq || __float_as_int(pz) == __float_as_int(lastz);
        if (zeq) c.j0 = refj0;
        else point_level(a, zs, pz, c);
        const int rx = wrap_rel<P2>(c.ix, refx, a.Nxr);
        const int ry = a.Nyr > 1 ? wrap_rel<P2>(c.iy, refy, a.Nyr) : 0;
        mn[0] = min(mn[0], rx);
        mx[0] = max(mx[0], rx);
        mn[1] = min(mn[1], ry);
        mx[1] = max(mx[1], ry);
        mn[2] = min(mn[2], c.j0);
        mx[2] = max(mx[2], c.j0);
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[d] = min(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
      mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
    }
  }
  const bool flat = __all_sync(0xffffffffu, same_z);
  const bool flat2 = !flat && __all_sync(0xffffffffu, two_z);
  if (lane != 0) return;
  // box: x nodes rel (mn0-1) .. (mx0+2), y likewise (one row in 2-D), levels mn2 .. mx2+3
  const int bx = mx[0] - mn[0] + 4;
  const int sbx = bx + ((4 - bx) & 7);
  const int by = a.Nyr > 1 ? mx[1] - mn[1] + 4 : 1;
  const int bz = mx[2] - mn[2] + 4;
  const int zst = box_zstride(sbx, by);
  const bool inside_grid = bx <= a.Nxr && by <= a.Nyr;
  const bool fits = int64_t(zst) * bz <= BOX_NODES && int64_t(sbx) * by <= BOX_COLS && inside_grid;
  const bool fits_flat = flat && int64_t(sbx) * by <= FLAT_COLS && inside_grid;
  const bool fits_two = flat2 && int64_t(sbx) * by <= FLAT2_COLS && inside_grid;
  const int x0 = wrapi<P2>(refx + mn[0] - 1, a.Nxr);
  const int y0 = a.Nyr > 1 ? wrapi<P2>(refy + mn[1] - 1, a.Nyr) : 0;
  plan[chunk] = fits_flat  ? make_int4(x0, y0, mn[2] | FLAT_BIT, bx | (by << 12))
              : fits_two   ? make_int4(x0, y0, FLAT_BIT | FLAT2_BIT, bx | (by << 12))
                           : make_int4(x0, y0, mn[2], fits ? (bx | (by << 11) | (bz << 22)) : -1);
}

template <bool P2>
__global__ void __launch_bounds__(BOX_THREADS) k_interp_plan(InterpArgs a, Levels L, int4* __restrict__ plan) {
  __shared__ LevelTables zs;
  fill_level_tables(zs, L, a.nz);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  plan_chunk<P2>(a, zs, int64_t(blockIdx.x) * PLAN_WARPS + warp, plan, lane);
}

// True when a chunk's plan stages no tile (or is a plan made for another level list): its points
// gather their stencils from global memory.
__device__ __forceinline__ bool plan_is_global(const int4 pl, int nz) {
  if (pl.w < 0) return true;
  const BoxPlan bp = decode_plan(pl);
  return bp.l0 + bp.bz > nz;
}

// Points p0 + k * BOX_THREADS + threadIdx.x (k < BOX_PPT) gathered from global memory.
template <bool P2>
__device__ __forceinline__ void global_points(const InterpArgs& a, const LevelTables& zs, int64_t p0) {
#pragma unroll 1
  for (int k = 0; k < BOX_PPT; ++k) {
    const int64_t i = p0 + k * BOX_THREADS + threadIdx.x;
    if (i >= a.np) break;                           // later points of this thread are past np too
    const float pz = __ldg(&a.pts[3 * i + 2]);
    const PointCell c = point_cell<P2>(a, zs, __ldg(&a.pts[3 * i]), __ldg(&a.pts[3 * i + 1]), pz);
    float4 acc;
    float acc_eta;
    gather_global<P2>(a, c, acc, acc_eta);
    store_point(a, i, acc, acc_eta, pz, c.inside);
  }
}

// Gather of chunk `chunk` of the points of `a` with its plan `pl`, by the whole CTA; the level
// tables zs are complete after the first barrier inside. kGlobal: also the chunks without a
// staged tile (else those are left to k_interp_global).
template <bool P2, bool kGlobal = true>
__device__ __forceinline__ void box_chunk(const InterpArgs& a, const LevelTables& zs, int64_t chunk,
                                          const int4 pl, float4* sbox, float* seta) {
  const int64_t p0 = chunk * BOX_PTS;
  // the first point's coordinates are in flight during the box load; each later point's while
  // the previous one is processed
  float nx_ = 0.f, ny_ = 0.f, nz_ = 0.f;
  {
    const int64_t i = p0 + threadIdx.x;
    if (i < a.np) {
      nx_ = __ldg(&a.pts[3 * i]);
      ny_ = __ldg(&a.pts[3 * i + 1]);
      nz_ = __ldg(&a.pts[3 * i + 2]);
    }
  }
  const BoxPlan bp = decode_plan(pl);
  if (plan_is_global(pl, a.nz)) {                  // no tile, or a plan of another level list
    __syncthreads();
    if (kGlobal) global_points<P2>(a, zs, p0);
    return;
  }
  const int bx = bp.bx, by = bp.by, bz = bp.bz;
  // shared-memory row stride = 4 (mod 8) float4: reads of neighbouring cells (dx, dy in {0, 1})
  // by one quarter-warp fall into different bank groups
  const int sbx = bx + ((4 - bx) & 7);
  const int x0 = bp.x0, y0 = bp.y0, l0 = bp.l0;
  const int nys = a.Nyr > 1 ? 4 : 1;
  if (bp.flat) {
    // one z (or two: a chunk across two layers) for the whole chunk: level weights once per z
    // (from the level tables, so after the barrier that completes them), the z-collapsed
    // plane(s) and the eta plane, then a 2-D gather of 16 float4 per point
    const bool two = bp.two;
    const float zc = __ldg(&a.pts[3 * p0 + 2]);
    const float zc2 = two ? __ldg(&a.pts[3 * ((p0 + BOX_PTS < a.np ? p0 + BOX_PTS : a.np) - 1) + 2]) : zc;
    __syncthreads();
    PointCell cz, cz2;
    point_level(a, zs, zc, cz);
    if (two) point_level(a, zs, zc2, cz2);
    else cz2 = cz;
    float4* planeB = two ? sbox + FLAT2_COLS : sbox;
    float* fe = reinterpret_cast<float*>(sbox + (two ? 2 * FLAT2_COLS : FLAT_COLS));
    stage_plane<P2>(a, x0, y0, cz.j0, bx, by, sbx, cz.wz, sbox, fe);
    if (two) stage_plane<P2>(a, x0, y0, cz2.j0, bx, by, sbx, cz2.wz, planeB, fe, false);
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < BOX_PPT; ++k) {
      const int64_t i = p0 + k * BOX_THREADS + threadIdx.x;
      if (i >= a.np) break;
      const float px = nx_, py = ny_, pz = nz_;
      if (k + 1 < BOX_PPT && i + BOX_THREADS < a.np) {
        nx_ = __ldg(&a.pts[3 * (i + BOX_THREADS)]);
        ny_ = __ldg(&a.pts[3 * (i + BOX_THREADS) + 1]);
        if (two) nz_ = __ldg(&a.pts[3 * (i + BOX_THREADS) + 2]);
      }
      const bool onA = !two || __float_as_int(pz) == __float_as_int(zc);
      PointCell c;
      point_xy<P2>(a, px, py, c);
      const int lx = min(max(wrapi<P2>(c.ix - 1 - x0, a.Nxr), 0), bx - 4);
      const int ly = a.Nyr > 1 ? min(max(wrapi<P2>(c.iy - 1 - y0, a.Nyr), 0), by - 4) : 0;
      const float4* base = (onA ? sbox : planeB) + ly * sbx + lx;
      const float* ebase = fe + ly * sbx + lx;
      // separable tensor product: each stencil row summed along x with the paired x weights,
      // then the rows combined with the y weights
      unsigned long long wx2[4];
#pragma unroll
      for (int kx = 0; kx < 4; ++kx) wx2[kx] = pack2(c.wx[kx], c.wx[kx]);
      unsigned long long uv = pack2(0.f, 0.f), wt = pack2(0.f, 0.f);
      float acc_eta = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (b >= nys) break;
        unsigned long long ruv, rwt;
        float re;
        row_sum(base + b * sbx, ebase + b * sbx, wx2, c.wx, ruv, rwt, re);
        const unsigned long long wy2 = pack2(c.wy[b], c.wy[b]);
        fma2(uv, wy2, ruv);
        fma2(wt, wy2, rwt);
        acc_eta = fmaf(c.wy[b], re, acc_eta);
      }
      store_point(a, i, make_float4(lo2(uv), hi2(uv), lo2(wt), hi2(wt)), acc_eta, pz,
                  onA ? cz.inside : cz2.inside);
    }
    return;
  }
  const int zst = box_zstride(sbx, by);
  stage_box<P2>(a, x0, y0, l0, bx, by, bz, sbx, zst, sbox, seta);
  __syncthreads();
  const int zstride = zst;
#pragma unroll 1
  for (int k = 0; k < BOX_PPT; ++k) {
    const int64_t i = p0 + k * BOX_THREADS + threadIdx.x;
    if (i >= a.np) break;                          // later points of this thread are past np too
    const float px = nx_, py = ny_, pz = nz_;
    if (k + 1 < BOX_PPT && i + BOX_THREADS < a.np) {
      nx_ = __ldg(&a.pts[3 * (i + BOX_THREADS)]);
      ny_ = __ldg(&a.pts[3 * (i + BOX_THREADS) + 1]);
      nz_ = __ldg(&a.pts[3 * (i + BOX_THREADS) + 2]);
    }
    const PointCell c = point_cell<P2>(a, zs, px, py, pz);
    // node offsets inside the box; the plan kernel bounded them with the same point_cell, and
    // the clamps keep every shared-memory read inside the box regardless
    const int lx = min(max(wrapi<P2>(c.ix - 1 - x0, a.Nxr), 0), bx - 4);
    const int ly = a.Nyr > 1 ? min(max(wrapi<P2>(c.iy - 1 - y0, a.Nyr), 0), by - 4) : 0;
    const int lz = min(max(c.j0 - l0, 0), bz - 4);
    const float4* base = sbox + lz * zst + ly * sbx + lx;
    // separable tensor product: rows along x, then y within each level, then the levels in z
    unsigned long long wx2[4];
#pragma unroll
    for (int kx = 0; kx < 4; ++kx) wx2[kx] = pack2(c.wx[kx], c.wx[kx]);
    unsigned long long uv = pack2(0.f, 0.f), wt = pack2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned long long quv = pack2(0.f, 0.f), qwt = pack2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (b >= nys) break;
        unsigned long long ruv, rwt;
        row_sum(base + q * zstride + b * sbx, wx2, ruv, rwt);
        const unsigned long long wy2 = pack2(c.wy[b], c.wy[b]);
        fma2(quv, wy2, ruv);
        fma2(qwt, wy2, rwt);
      }
      const unsigned long long wz2 = pack2(c.wz[q], c.wz[q]);
      fma2(uv, wz2, quv);
      fma2(wt, wz2, qwt);
    }
    float acc_eta = 0.f;
    const float* ebase = seta + ly * sbx + lx;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (b >= nys) break;
      float re = 0.f;
#pragma unroll
      for (int kx = 0; kx < 4; ++kx) re = fmaf(c.wx[kx], ebase[b * sbx + kx], re);
      acc_eta = fmaf(c.wy[b], re, acc_eta);
    }
    store_point(a, i, make_float4(lo2(uv), hi2(uv), lo2(wt), hi2(wt)), acc_eta, pz, c.inside);
  }
}

// The chunks with a staged tile (box, plane or two planes); kSplit: k_interp_global takes the
// others, else this kernel gathers them too (from global memory, with L1 reduced by the tile).
template <bool P2, bool kSplit>
__global__ void __launch_bounds__(BOX_THREADS, 3) k_interp_box(InterpArgs a, Levels L,
                                                                const int4* __restrict__ plan) {
  extern __shared__ float4 sbox[];
  float* seta = reinterpret_cast<float*>(sbox + BOX_NODES);
  __shared__ LevelTables zs;
  const int4 pl = plan[blockIdx.x];
  if (kSplit && plan_is_global(pl, a.nz)) return;   // uniform over the CTA
  fill_level_tables(zs, L, a.nz);
  box_chunk<P2, !kSplit>(a, zs, blockIdx.x, pl, sbox, seta);
}

// The chunks without a staged tile (scattered points: the stencils of a 1024-point chunk span
// more nodes than shared memory holds). No dynamic shared memory, so that L1 keeps the rows
// neighbouring points share: launched apart from k_interp_box, whose 68 KB tile per CTA would
// leave L1 a fifth of its size.
// One quarter of a chunk (256 points, one a thread) per CTA, in point order: the CTAs in flight
// then cover consecutive points, whose stencils share rows in L2, over a quarter of the span that
// whole chunks per CTA would (3 % faster on the large sea); the quarters of chunks with a staged
// tile exit at once.
template <bool P2>
__global__ void __launch_bounds__(BOX_THREADS, 4) k_interp_global(InterpArgs a, Levels L,
                                                                   const int4* __restrict__ plan) {
  __shared__ LevelTables zs;
  const int64_t sub = blockIdx.x, chunk = sub / BOX_PPT;
  const int4 pl = plan[chunk];
  if (!plan_is_global(pl, a.nz)) return;            // uniform over the CTA
  fill_level_tables(zs, L, a.nz);
  __syncthreads();
  const int64_t i = chunk * BOX_PTS + (sub % BOX_PPT) * BOX_THREADS + threadIdx.x;
  if (i >= a.np) return;
  const float pz = __ldg(&a.pts[3 * i + 2]);
  const PointCell c = point_cell<P2>(a, zs, __ldg(&a.pts[3 * i]), __ldg(&a.pts[3 * i + 1]), pz);
  float4 acc;
  float acc_eta;
  gather_global<P2>(a, c, acc, acc_eta);
  store_point(a, i, acc, acc_eta, pz, c.inside);
}

// ---------------------------------------------------------------------------------------------
// Batched gather (many instances, swense_batch_run): the point chunks of every instance form
// one list. One launch plans them all (a warp per chunk, the warp's own copy of its instance's
// arguments and level tables), then one persistent launch gathers them: each CTA takes the next
// chunk from a device counter and reloads the instance's arguments and level tables only when
// the instance changes (chunks are listed instance by instance, so rarely).
struct BatchInst {
  InterpArgs a;
  Levels L;
};

__device__ __forceinline__ int batch_instance(const int64_t* chunk0, int n, int64_t c) {
  int lo = 0, hi = n - 1;                           // last instance whose first chunk <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chunk0[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void copy_words(void* dst, const void* src, int bytes, int t, int nt) {
  const int* s = static_cast<const int*>(src);
  int* d = static_cast<int*>(dst);
  for (int i = t; i < bytes / 4; i += nt) d[i] = __ldg(&s[i]);
}

__global__ void __launch_bounds__(BOX_THREADS) k_interp_plan_batch(const BatchInst* __restrict__ inst,
                                                                   const int64_t* __restrict__ chunk0, int n,
                                                                   int4* __restrict__ plan) {
  extern __shared__ unsigned char smb[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  InterpArgs* sa = reinterpret_cast<InterpArgs*>(smb) + warp;
  LevelTables* zs = reinterpret_cast<LevelTables*>(smb + PLAN_WARPS * sizeof(InterpArgs)) + warp;
  const int64_t c = int64_t(blockIdx.x) * PLAN_WARPS + warp;
  if (c >= chunk0[n]) return;                       // no block barrier in this kernel
  const int i = batch_instance(chunk0, n, c);
  copy_words(sa, &inst[i].a, int(sizeof(InterpArgs)), lane, 32);
  const Levels& L = inst[i].L;
  const int nz = inst[i].a.nz;
  if (lane == 0) {
    zs->z0 = L.z0;
    zs->inv_h = L.inv_h;
  }
  for (int k = lane; k < ZLUT / 4; k += 32) reinterpret_cast<unsigned*>(zs->lut)[k] = L.lut4[k];
  for (int k = lane; k < nz; k += 32) zs->z[k] = L.z[k];
  for (int j = lane; j <= nz - 4; j += 32) zs->inv[j] = L.inv[j];
  __syncwarp();
  plan_chunk<true>(*sa, *zs, c - chunk0[i], plan + chunk0[i], lane);
}

__global__ void __launch_bounds__(BOX_THREADS, 3) k_interp_box_batch(const BatchInst* __restrict__ inst,
                                                                      const int64_t* __restrict__ chunk0, int n,
                                                                      const int4* __restrict__ plan,
                                                                      unsigned* __restrict__ counter) {
  extern __shared__ float4 sbox[];
  float* seta = reinterpret_cast<float*>(sbox + BOX_NODES);
  __shared__ LevelTables zs;
  __shared__ InterpArgs sa;
  __shared__ int64_t s_item;
  const int64_t total = chunk0[n];
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = int64_t(atomicAdd(counter, 1u));
    __syncthreads();
    const int64_t c = s_item;
    if (c >= total) break;                          // uniform over the CTA
    const int i = batch_instance(chunk0, n, c);
    if (i != cur) {
      copy_words(&sa, &inst[i].a, int(sizeof(InterpArgs)), threadIdx.x, blockDim.x);
      fill_level_tables(zs, inst[i].L, inst[i].a.nz);
      cur = i;
    }
    __syncthreads();                                // arguments and tables in place
    box_chunk<true>(sa, zs, c - chunk0[i], plan[c], sbox, seta);
    __syncthreads();                                // shared memory free for the next chunk
  }
}

// ---------------------------------------------------------------------------------------------
// Fused learned gather: the plain Lagrange gather, the network's inputs and its three layers in
// one kernel, per 1024-point chunk. The chunk's stencils come from the staged box (as in
// k_interp_box) when it fits, else from per-point stencil arrays gathered from global memory
// (64 points at a time) in the same shared memory. Per sub-batch of points:
//   A (one thread per point): cell, Lagrange weights, offsets, eta, stencil base -> LPoint;
//   B (warps, m16n8k16): rows (point, field), 16 rows = 4 points x 4 fields per tile; each lane
//     reads its fragment's stencil values, the quad reduces the row's Lagrange value and
//     max |value|, the normalised values (hi + lo BF16) feed layers 1-3, and the lane holding
//     column f of row (point, f) writes lagrange + s_f * out_scale * y[f];
//   C (one thread per point): Bernoulli, NaN outside the levels, stores.
struct LPoint {
  int base;                 // staged node index of stencil node (x 0, y 0, level 0)
  float w[12];              // wx[4], wy[4], wz[4]; the corrected fields overwrite w[0..3]
  float off[3];             // dx, dy in the cell; dz in the stencil's middle level interval
  float eta, z;
  int inside, pad_;
};
static_assert(sizeof(LPoint) == 80, "LPoint layout");

using mlpnet::PackedFwd;

// Shared-memory copy of the forward weights with padded rows: the B-fragment loads of a warp
// (row 8 nt + g, word 8 kk + q) then fall into 32 different banks (an unpadded 64-wide row
// maps all eight g to one bank).
constexpr int W1LD = mlpnet::KIN + 8, W2LD = mlpnet::NH + 8;
struct WeightsSmem {
  __nv_bfloat16 w1[mlpnet::NH][W1LD];
  __nv_bfloat16 w2[mlpnet::NH][W2LD];
  __nv_bfloat16 w3[mlpnet::NO][W2LD];
  float b1[mlpnet::NH], b2[mlpnet::NH], b3[mlpnet::NO];
  float out_scale, pad_[3];
};

constexpr int LRN_SB = 128;                            // points per sub-batch (box mode)
constexpr int LRN_SB_PP = 64;                          // points per sub-batch (per-point stencils)
static_assert(LRN_SB_PP * 64 <= BOX_NODES, "per-point stencils fit the box area");
constexpr size_t LRN_SMEM = size_t(BOX_NODES) * sizeof(float4) + size_t(BOX_COLS) * sizeof(float) +
                            size_t(LRN_SB) * sizeof(LPoint) + sizeof(WeightsSmem);

// Phase B for `ntile` 16-row tiles of this warp. Node (x k, y b, level q) of point j is
// nodes[rec[j].base + q * SZ + b * SY + k].
__device__ __forceinline__ void learned_tiles(const float4* nodes, int SY, int SZ, LPoint* rec,
                                              const WeightsSmem& W, int tile0, int ntile, int npts) {
  using namespace mlpnet;
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int f = g & 3;                                 // field of rows g and g + 8
  const float* nf = reinterpret_cast<const float*>(nodes) + f;
  for (int t = tile0; t < tile0 + ntile; ++t) {
    const int j0 = 4 * t + (g >> 2), j1 = j0 + 2;      // points of rows g and g + 8
    if (4 * t >= npts) break;                          // uniform over the warp
    float lag[2], sc[2];
    unsigned xh[5][4], xl[5][4];
    float v[2][4][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const LPoint& P = rec[min(h ? j1 : j0, npts - 1)];
      const int base = P.base;
      float lg = 0.f, mx = 0.f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int b = (q >> 1) + 2 * (e >> 1), k = 2 * (q & 1) + (e & 1);
          const float val = nf[4 * (base + kk * SZ + b * SY + k)];
          v[h][kk][e] = val;
          lg = fmaf(P.w[8 + kk] * P.w[4 + b] * P.w[k], val, lg);
          mx = fmaxf(mx, fabsf(val));
        }
      }
      lg += __shfl_xor_sync(0xffffffffu, lg, 1);
      lg += __shfl_xor_sync(0xffffffffu, lg, 2);
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      lag[h] = lg;
      sc[h] = mx + 1e-30f;
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float inv = 1.f / sc[h];
        bf2_split(v[h][kk][0] * inv, v[h][kk][1] * inv, xh[kk][h], xl[kk][h]);
        bf2_split(v[h][kk][2] * inv, v[h][kk][3] * inv, xh[kk][2 + h], xl[kk][2 + h]);
      }
    }
    // inputs 64..79: dx, dy, dz, then zeros (columns 2q, 2q+1 of the fifth k-tile)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const LPoint& P = rec[min(h ? j1 : j0, npts - 1)];
      const float o0 = q == 0 ? P.off[0] : (q == 1 ? P.off[2] : 0.f);
      const float o1 = q == 0 ? P.off[1] : 0.f;
      bf2_split(o0, o1, xh[4][h], xl[4][h]);
      xh[4][2 + h] = xl[4][2 + h] = 0u;
    }
    float z1[8][4];
    layer<5, 8, true>(z1, xh, xl, &W.w1[0][0], W1LD, W.b1, lane);
    unsigned h1h[4][4], h1l[4][4];
    to_a<8, true>(z1, h1h, h1l);
    float z2[8][4];
    layer<4, 8, true>(z2, h1h, h1l, &W.w2[0][0], W2LD, W.b2, lane);
    unsigned h2h[4][4], h2l[4][4];
    to_a<8, true>(z2, h2h, h2l);
    float o[1][4];
    layer<4, 1, true>(o, h2h, h2l, &W.w3[0][0], W2LD, W.b3, lane);
    __syncwarp();                                      // every lane has read its records
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int jh = h ? j1 : j0;
      const float yv = (f & 1) ? o[0][2 * h + 1] : o[0][2 * h];   // a select, not a local array
      if ((f >> 1) == q && jh < npts) rec[jh].w[f] = fmaf(sc[h] * W.out_scale, yv, lag[h]);
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(BOX_THREADS, 2) k_interp_learned(InterpArgs a, Levels L,
                                                                    const int4* __restrict__ plan,
                                                                    const PackedFwd* __restrict__ Wg) {
  extern __shared__ float4 sbox[];
  float* seta = reinterpret_cast<float*>(sbox + BOX_NODES);
  LPoint* rec = reinterpret_cast<LPoint*>(seta + BOX_COLS);
  WeightsSmem& W = *reinterpret_cast<WeightsSmem*>(rec + LRN_SB);
  __shared__ LevelTables zs;
  fill_level_tables(zs, L, a.nz);
  {
    // rows re-strided into the padded layout, 16 bytes (8 bf16) at a time
    using namespace mlpnet;
    const uint4* g1 = reinterpret_cast<const uint4*>(&Wg->w1[0][0]);
    const uint4* g2 = reinterpret_cast<const uint4*>(&Wg->w2[0][0]);
    const uint4* g3 = reinterpret_cast<const uint4*>(&Wg->w3[0][0]);
    for (int i = threadIdx.x; i < NH * KIN / 8; i += blockDim.x)
      *reinterpret_cast<uint4*>(&W.w1[i / (KIN / 8)][8 * (i % (KIN / 8))]) = __ldg(&g1[i]);
    for (int i = threadIdx.x; i < NH * NH / 8; i += blockDim.x)
      *reinterpret_cast<uint4*>(&W.w2[i / (NH / 8)][8 * (i % (NH / 8))]) = __ldg(&g2[i]);
    for (int i = threadIdx.x; i < NO * NH / 8; i += blockDim.x)
      *reinterpret_cast<uint4*>(&W.w3[i / (NH / 8)][8 * (i % (NH / 8))]) = __ldg(&g3[i]);
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
      W.b1[i] = __ldg(&Wg->b1[i]);
      W.b2[i] = __ldg(&Wg->b2[i]);
    }
    if (threadIdx.x < NO) W.b3[threadIdx.x] = __ldg(&Wg->b3[threadIdx.x]);
    if (threadIdx.x == 0) W.out_scale = __ldg(&Wg->out_scale);
  }
  const int64_t p0 = int64_t(blockIdx.x) * BOX_PTS;
  const int4 pl = plan[blockIdx.x];
  const BoxPlan bp = decode_plan(pl);
  const int bx = bp.bx, by = bp.by;
  const int sbx = bx + ((4 - bx) & 7);
  const int zst = box_zstride(sbx, by);
  int l0 = bp.l0, bz = bp.bz;
  bool box3d = bp.box3d;
  if (bp.two) {
    // a chunk across two layers: the box spans the level windows of its first and last
    // point's z (the level tables are complete after this barrier)
    __syncthreads();
    PointCell ca, cb;
    point_level(a, zs, __ldg(&a.pts[3 * p0 + 2]), ca);
    point_level(a, zs, __ldg(&a.pts[3 * ((p0 + BOX_PTS < a.np ? p0 + BOX_PTS : a.np) - 1) + 2]), cb);
    l0 = min(ca.j0, cb.j0);
    bz = abs(ca.j0 - cb.j0) + 4;
    box3d = int64_t(zst) * bz <= BOX_NODES && int64_t(sbx) * by <= BOX_COLS;
  }
  const bool boxed = box3d && l0 + bz <= a.nz;
  const int x0 = bp.x0, y0 = bp.y0;
  const size_t plane = size_t(a.Nyr) * a.Nxr;
  if (boxed) stage_box(a, x0, y0, l0, bx, by, bz, sbx, zst, sbox, seta);
  __syncthreads();
  const int SB = boxed ? LRN_SB : LRN_SB_PP;
  const int warp = threadIdx.x >> 5;
  for (int s0 = 0; s0 < BOX_PTS; s0 += SB) {
    const int npts = int(a.np - (p0 + s0) < int64_t(SB) ? a.np - (p0 + s0) : int64_t(SB));
    if (npts <= 0) break;                              // uniform over the block
    // ---- A
    if (boxed) {
      const int t = threadIdx.x;
      if (t < npts) {
        const int64_t i = p0 + s0 + t;
        const float px = __ldg(&a.pts[3 * i]), py = __ldg(&a.pts[3 * i + 1]), pz = __ldg(&a.pts[3 * i + 2]);
        const PointCell c = point_cell(a, zs, px, py, pz);
        const int lx = min(max((c.ix - 1 - x0) & (a.Nxr - 1), 0), bx - 4);
        const int ly = min(max((c.iy - 1 - y0) & (a.Nyr - 1), 0), by - 4);
        const int lz = min(max(c.j0 - l0, 0), bz - 4);
        LPoint& P = rec[t];
        P.base = lz * zst + ly * sbx + lx;
        float e = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int k = 0; k < 4; ++k) e = fmaf(c.wy[b] * c.wx[k], seta[(ly + b) * sbx + lx + k], e);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          P.w[k] = c.wx[k];
          P.w[4 + k] = c.wy[k];
          P.w[8 + k] = c.wz[k];
        }
        float fx, fy;
        int ixx, iyy;
        locate(px, a.sx_hi, a.sx_lo, a.Nxr, ixx, fx);
        locate(py, a.sy_hi, a.sy_lo, a.Nyr, iyy, fy);
        const float z1 = zs.z[c.j0 + 1], z2 = zs.z[c.j0 + 2];
        P.off[0] = fx;
        P.off[1] = fy;
        P.off[2] = (pz - z1) / (z2 - z1);
        P.eta = e;
        P.z = pz;
        P.inside = c.inside;
      }
    } else {
      // per-point stencils: four threads per point, each blends 16 of its 64 nodes
      const int j = threadIdx.x >> 2, qq = threadIdx.x & 3;
      if (j < npts) {
        const int64_t i = p0 + s0 + j;
        const float px = __ldg(&a.pts[3 * i]), py = __ldg(&a.pts[3 * i + 1]), pz = __ldg(&a.pts[3 * i + 2]);
        const PointCell c = point_cell(a, zs, px, py, pz);
        const size_t tl_stride = size_t(a.nz) * plane;
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
          const int node = 16 * qq + kk, zq = node >> 4, b = (node >> 2) & 3, k = node & 3;
          const size_t gi = size_t(c.j0 + zq) * plane + size_t((c.iy - 1 + b) & (a.Nyr - 1)) * a.Nxr +
                            size_t((c.ix - 1 + k) & (a.Nxr - 1));
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int tl = 0; tl < a.n_tl; ++tl) {
            const float4 gv = __ldg(&a.nodes[size_t(tl) * tl_stride + gi]);
            const float w = a.wt[tl];
            v.x = fmaf(w, gv.x, v.x);
            v.y = fmaf(w, gv.y, v.y);
            v.z = fmaf(w, gv.z, v.z);
            v.w = fmaf(w, gv.w, v.w);
          }
          sbox[64 * j + node] = v;
        }
        if (qq == 0) {
          LPoint& P = rec[j];
          P.base = 64 * j;
          float e = 0.f;
          for (int tl = 0; tl < a.n_tl; ++tl)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
              for (int k = 0; k < 4; ++k)
                e = fmaf(a.wt[tl] * c.wy[b] * c.wx[k],
                         __ldg(&a.eta[size_t(tl) * plane + size_t((c.iy - 1 + b) & (a.Nyr - 1)) * a.Nxr +
                                      ((c.ix - 1 + k) & (a.Nxr - 1))]), e);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            P.w[k] = c.wx[k];
            P.w[4 + k] = c.wy[k];
            P.w[8 + k] = c.wz[k];
          }
          float fx, fy;
          int ixx, iyy;
          locate(px, a.sx_hi, a.sx_lo, a.Nxr, ixx, fx);
          locate(py, a.sy_hi, a.sy_lo, a.Nyr, iyy, fy);
          const float z1 = zs.z[c.j0 + 1], z2 = zs.z[c.j0 + 2];
          P.off[0] = fx;
          P.off[1] = fy;
          P.off[2] = (pz - z1) / (z2 - z1);
          P.eta = e;
          P.z = pz;
          P.inside = c.inside;
        }
      }
    }
    __syncthreads();
    // ---- B: SB points = SB / 4 tiles, spread over the warps
    const int ntiles = (npts + 3) / 4, per = (SB / 4 + (blockDim.x >> 5) - 1) / (blockDim.x >> 5);
    if (boxed) learned_tiles(sbox, sbx, zst, rec, W, warp * per, min(per, max(ntiles - warp * per, 0)), npts);
    else learned_tiles(sbox, 4, 16, rec, W, warp * per, min(per, max(ntiles - warp * per, 0)), npts);
    __syncthreads();
    // ---- C
    if (threadIdx.x < npts) {
      const LPoint& P = rec[threadIdx.x];
      store_point(a, p0 + s0 + threadIdx.x, make_float4(P.w[0], P.w[1], P.w[2], P.w[3]), P.eta, P.z,
                  P.inside != 0);
    }
    __syncthreads();
  }
}

void split(double v, float& hi, float& lo) {
  hi = float(v);
  lo = float(v - double(hi));
}

}  // namespace
}  // namespace swense

// ---------------------------------------------------------------------------------------------
// Inputs of the learned correction: per point and field f in (u, v, w, dphi/dt) one row
//   x = [stencil_f / s_f (64 time-blended node values, x fastest, then y, then z), dx, dy, dz, 0]
// with s_f = max |stencil_f| + 1e-30 and dz the offset in the stencil's middle level interval,
// plus s_f, the plain Lagrange value of f, and the plain eta.
namespace swense {
namespace {

constexpr int MLP_XLD = 68;

struct FeatArgs {
  InterpArgs a;          // grid, points, time weights (o_* unused)
  float* x;              // [4 np][68]
  float* scale;          // [4 np]
  float* lag;            // [4 np]
  float* eta_out;        // [np] or NULL
};

__global__ void __launch_bounds__(128) k_mlp_features(FeatArgs f, Levels L) {
  __shared__ LevelTables zs;
  const InterpArgs& a = f.a;
  fill_level_tables(zs, L, a.nz);
  __syncthreads();
  const size_t plane = size_t(a.Nyr) * a.Nxr;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.np;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float px = a.pts[3 * i], py = a.pts[3 * i + 1], pz = a.pts[3 * i + 2];
    const PointCell c = point_cell(a, zs, px, py, pz);
    float fx, fy;
    int ixx, iyy;
    locate(px, a.sx_hi, a.sx_lo, a.Nxr, ixx, fx);
    locate(py, a.sy_hi, a.sy_lo, a.Nyr, iyy, fy);
    const float z1 = zs.z[c.j0 + 1], z2 = zs.z[c.j0 + 2];
    const float fz = (pz - z1) / (z2 - z1);
    int xi[4], yi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      xi[q] = (c.ix - 1 + q) & (a.Nxr - 1);
      yi[q] = (c.iy - 1 + q) & (a.Nyr - 1);
    }
    if (f.eta_out) {
      float e = 0.f;
      for (int tl = 0; tl < a.n_tl; ++tl)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            e = fmaf(a.wt[tl] * c.wy[b] * c.wx[k], __ldg(&a.eta[tl * plane + size_t(yi[b]) * a.Nxr + xi[k]]), e);
      f.eta_out[i] = e;
    }
#pragma unroll 1
    for (int fld = 0; fld < 4; ++fld) {
      float* xr = f.x + (4 * i + fld) * MLP_XLD;
      float smax = 0.f, lagv = 0.f;
      // pass 1: time-blended stencil values -> row (unscaled), max, Lagrange value
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        const float wzq = q == 0 ? c.wz[0] : q == 1 ? c.wz[1] : q == 2 ? c.wz[2] : c.wz[3];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const size_t node = size_t(c.j0 + q) * plane + size_t(yi[b]) * a.Nxr + xi[k];
            float v = 0.f;
            for (int tl = 0; tl < a.n_tl; ++tl)
              v = fmaf(a.wt[tl], __ldg(reinterpret_cast<const float*>(&a.nodes[tl * a.nz * plane + node]) + fld), v);
            xr[(q * 4 + b) * 4 + k] = v;
            smax = fmaxf(smax, fabsf(v));
            lagv = fmaf(wzq * c.wy[b] * c.wx[k], v, lagv);
          }
        }
      }
      const float s = smax + 1e-30f;
      const float inv = 1.f / s;
      for (int k = 0; k < 64; ++k) xr[k] *= inv;
      xr[64] = fx;
      xr[65] = fy;
      xr[66] = fz;
      xr[67] = 0.f;
      f.scale[4 * i + fld] = s;
      f.lag[4 * i + fld] = lagv;
    }
  }
}

// Validate a grid request and fill the launch arguments shared by the interpolation entry points.
int prepare_interp(const swense_grid* g, double t, const float* pts, int64_t np, int32_t p_mode,
                   double rho, double grav, InterpArgs* a, Levels* lev) {
  if (!g || !g->nodes || !g->eta || !g->z_levels || !g->t_levels)
    return fail(SWENSE_ERR_ARG, "NULL grid, grid arrays or level lists");
  if (np < 0) return fail(SWENSE_ERR_ARG, "np must be >= 0");
  if (np > 0 && !pts) return fail(SWENSE_ERR_ARG, "NULL pts");
  // node counts: even in [4, MAX] (powers of two, or a non-power-of-two padding factor times
  // one); ny_r = 1 for a 2-D grid
  if ((g->nx_r & 1) || g->nx_r < 4 || g->nx_r > SWENSE_MAX_FFT ||
      (g->ny_r != 1 && ((g->ny_r & 1) || g->ny_r < 4)) || g->ny_r > SWENSE_MAX_FFT)
    return fail(SWENSE_ERR_SIZE, "nx_r must be even in [4, MAX], ny_r 1 or even in [4, MAX]");
  if (g->nz < 4 || g->nz > SWENSE_MAX_LEVELS) return fail(SWENSE_ERR_LEVELS, "need 4 <= nz <= SWENSE_MAX_LEVELS");
  if (g->n_tl < 1 || g->n_tl > SWENSE_MAX_TL) return fail(SWENSE_ERR_ARG, "n_tl must be in [1, SWENSE_MAX_TL]");
  if (p_mode != SWENSE_P_DYN && p_mode != SWENSE_P_PHIT && p_mode != SWENSE_P_TOTAL)
    return fail(SWENSE_ERR_ARG, "unknown p_mode");
  if (!(g->Lx > 0) || !std::isfinite(g->Lx) || (g->ny_r > 1 && (!(g->Ly > 0) || !std::isfinite(g->Ly))))
    return fail(SWENSE_ERR_ARG, "domain lengths must be finite and positive");
  if (!std::isfinite(t) || !std::isfinite(rho) || !std::isfinite(grav))
    return fail(SWENSE_ERR_ARG, "non-finite t, rho or g");
  if (reinterpret_cast<uintptr_t>(g->nodes) & 15) return fail(SWENSE_ERR_ARG, "nodes must be 16-byte aligned");
  for (int l = 0; l < g->nz; ++l) {
    lev->z[l] = g->z_levels[l];
    if (!std::isfinite(lev->z[l]) || (l > 0 && !(lev->z[l] > lev->z[l - 1])))
      return fail(SWENSE_ERR_LEVELS, "z_levels must be finite and strictly increasing");
  }
  {
    const int nz = g->nz;
    for (int j = 0; j + 3 < nz; ++j) {
      double zn[4], d[4];
      for (int q = 0; q < 4; ++q) zn[q] = lev->z[j + q];
      for (int q = 0; q < 4; ++q) {
        d[q] = 1.0;
        for (int r = 0; r < 4; ++r)
          if (r != q) d[q] *= zn[q] - zn[r];
      }
      lev->inv[j] = make_float4(float(1.0 / d[0]), float(1.0 / d[1]), float(1.0 / d[2]), float(1.0 / d[3]));
    }
    const double z0 = lev->z[0], h = (double(lev->z[nz - 1]) - z0) / ZLUT;
    lev->z0 = lev->z[0];
    lev->inv_h = float(1.0 / h);
    unsigned char lut[ZLUT];
    int j = 0;
    for (int b = 0; b < ZLUT; ++b) {
      const double zb = z0 + b * h;
      while (j + 1 < nz && double(lev->z[j + 1]) <= zb) ++j;
      lut[b] = (unsigned char)j;
    }
    std::memcpy(lev->lut4, lut, sizeof(lut));
  }
  for (int l = 0; l < g->n_tl; ++l) {
    if (!std::isfinite(g->t_levels[l]) || (l > 0 && !(g->t_levels[l] > g->t_levels[l - 1])))
      return fail(SWENSE_ERR_ARG, "t_levels must be finite and strictly increasing");
  }
  *a = InterpArgs{};
  for (int l = 0; l < g->n_tl; ++l) {
    double wl = 1.0;
    for (int m = 0; m < g->n_tl; ++m)
      if (m != l) wl *= (t - g->t_levels[m]) / (g->t_levels[l] - g->t_levels[m]);
    a->wt[l] = float(wl);
  }
  a->nodes = reinterpret_cast<const float4*>(g->nodes);
  a->eta = g->eta;
  a->pts = pts;
  a->np = np;
  a->Nxr = g->nx_r;
  a->Nyr = g->ny_r;
  a->nz = g->nz;
  a->n_tl = g->n_tl;
  split(double(g->nx_r) / g->Lx, a->sx_hi, a->sx_lo);
  if (g->ny_r > 1) split(double(g->ny_r) / g->Ly, a->sy_hi, a->sy_lo);
  a->p_mode = p_mode;
  a->rho = float(rho);
  a->g = float(grav);
  if (g->scheme != SWENSE_LAGRANGE3 && g->scheme != SWENSE_SPLINE3)
    return fail(SWENSE_ERR_ARG, "unknown interpolation scheme");
  a->spline = g->scheme == SWENSE_SPLINE3;
  a->p2 = is_pow2(g->nx_r) && is_pow2(g->ny_r);
  return SWENSE_OK;
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_mlp_features(const swense_grid* g, double t, const float* pts, int64_t np,
                                   float* x, float* scale, float* lagrange, float* eta,
                                   void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  InterpArgs a;
  Levels lev;
  int st = prepare_interp(g, t, pts, np, SWENSE_P_DYN, 1.0, 1.0, &a, &lev);
  if (st) return st;
  if (g->ny_r < 4) return fail(SWENSE_ERR_UNSUPPORTED, "the learned correction needs a 3-D grid");
  if (a.spline) return fail(SWENSE_ERR_UNSUPPORTED, "the learned correction is defined on LAGRANGE3 grids");
  if (!a.p2) return fail(SWENSE_ERR_UNSUPPORTED, "the learned correction needs power-of-two node counts");
  if (np == 0) return SWENSE_OK;
  if (!x || !scale || !lagrange) return fail(SWENSE_ERR_ARG, "NULL feature outputs");
  FeatArgs f{a, x, scale, lagrange, eta};
  const unsigned blocks = unsigned(std::min<int64_t>((np + 127) / 128, 152 * 64));
  k_mlp_features<<<blocks, 128, 0, stream>>>(f, lev);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

extern "C" int swense_interp_learned(const swense_grid* g, double t, const float* pts, int64_t np,
                                     float* eta, float* u, float* v, float* w, float* p,
                                     int32_t p_mode, double rho, double grav, const void* packed,
                                     int64_t* n_out_of_range, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  InterpArgs a;
  Levels lev;
  int st = prepare_interp(g, t, pts, np, p_mode, rho, grav, &a, &lev);
  if (st) return st;
  if (g->ny_r < 4) return fail(SWENSE_ERR_UNSUPPORTED, "the learned correction needs a 3-D grid");
  if (a.spline) return fail(SWENSE_ERR_UNSUPPORTED, "the learned correction is defined on LAGRANGE3 grids");
  if (!a.p2) return fail(SWENSE_ERR_UNSUPPORTED, "the learned correction needs power-of-two node counts");
  if (!packed) return fail(SWENSE_ERR_ARG, "NULL packed weights");
  if (reinterpret_cast<uintptr_t>(packed) & 15) return fail(SWENSE_ERR_ARG, "packed weights must be 16-byte aligned");
  // workspace: [0, 256) out-of-range counter, then one int4 box plan per 1024-point chunk
  const int64_t blocks = (np + BOX_PTS - 1) / BOX_PTS;
  if (blocks >= (int64_t(1) << 31)) return fail(SWENSE_ERR_SIZE, "too many points for one call");
  void* ws = nullptr;
  st = workspace(256 + size_t(blocks) * sizeof(int4), stream, &ws);
  if (st) return st;
  unsigned long long* d_count = static_cast<unsigned long long*>(ws);
  if (n_out_of_range) SWENSE_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream));
  if (np > 0) {
    a.o_eta = eta;
    a.o_u = u;
    a.o_v = v;
    a.o_w = w;
    a.o_p = p;
    a.n_oor = n_out_of_range ? d_count : nullptr;
    int4* plan = reinterpret_cast<int4*>(static_cast<char*>(ws) + 256);
    k_interp_plan<true><<<unsigned(plan_blocks(np)), BOX_THREADS, 0, stream>>>(a, lev, plan);
    SWENSE_CUDA_TRY(cudaGetLastError());
    SWENSE_CUDA_TRY(cudaFuncSetAttribute((const void*)k_interp_learned,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(LRN_SMEM)));
    k_interp_learned<<<unsigned(blocks), BOX_THREADS, LRN_SMEM, stream>>>(
        a, lev, plan, static_cast<const PackedFwd*>(packed));
    SWENSE_CUDA_TRY(cudaGetLastError());
    count_launches(2);
  }
  if (n_out_of_range) {
    unsigned long long h = 0;
    SWENSE_CUDA_TRY(cudaMemcpyAsync(&h, d_count, sizeof(h), cudaMemcpyDeviceToHost, stream));
    SWENSE_CUDA_TRY(cudaStreamSynchronize(stream));
    *n_out_of_range = int64_t(h);
  }
  return SWENSE_OK;
}

namespace swense {
namespace {

// plan_in: a plan made earlier by swense_interp_plan for these points and this grid geometry
// (NULL: make one in the workspace first).
int interp_impl(const swense_grid* g, double t, const float* pts, const int32_t* perm, int64_t np,
                float* eta, float* u, float* v, float* w, float* p, int32_t p_mode, double rho,
                double grav, int64_t* n_out_of_range, cudaStream_t stream,
                const int4* plan_in = nullptr) {
  InterpArgs a;
  Levels lev;
  int st = prepare_interp(g, t, pts, np, p_mode, rho, grav, &a, &lev);
  if (st) return st;
  // workspace: [0, 256) out-of-range counter, then one int4 box plan per 1024-point chunk
  void* ws = nullptr;
  st = workspace(256 + (plan_in ? 0 : size_t((np + BOX_PTS - 1) / BOX_PTS) * sizeof(int4)), stream, &ws);
  if (st) return st;
  unsigned long long* d_count = nullptr;
  if (n_out_of_range) {
    d_count = static_cast<unsigned long long*>(ws);
    SWENSE_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream));
  }
  if (np > 0) {
    a.o_eta = eta;
    a.o_u = u;
    a.o_v = v;
    a.o_w = w;
    a.o_p = p;
    a.n_oor = d_count;
    a.perm = perm;
    const int64_t blocks = (np + BOX_PTS - 1) / BOX_PTS;
    if (blocks >= (int64_t(1) << 31)) return fail(SWENSE_ERR_SIZE, "too many points for one call");
    const int4* plan = plan_in;
    if (!plan) {
      int4* pw = reinterpret_cast<int4*>(static_cast<char*>(ws) + 256);
      if (a.p2) k_interp_plan<true><<<unsigned(plan_blocks(np)), BOX_THREADS, 0, stream>>>(a, lev, pw);
      else k_interp_plan<false><<<unsigned(plan_blocks(np)), BOX_THREADS, 0, stream>>>(a, lev, pw);
      SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
      plan = pw;
    }
    // Sparse point sets (fewer points than a quarter of a time level's nodes: a chunk's
    // stencils then rarely fit a tile) send the chunks without a tile to k_interp_global, where
    // L1 is not reduced by the tile; dense ones (meshes at their grid's resolution) gather the
    // rare such chunks inside k_interp_box and skip the second launch.
    const bool split = double(np) < 0.25 * double(a.Nxr) * double(a.Nyr) * double(a.nz);
    const void* kbox = a.p2 ? (split ? (const void*)k_interp_box<true, true> : (const void*)k_interp_box<true, false>)
                            : (split ? (const void*)k_interp_box<false, true> : (const void*)k_interp_box<false, false>);
    SWENSE_CUDA_TRY(cudaFuncSetAttribute(kbox, cudaFuncAttributeMaxDynamicSharedMemorySize, int(BOX_SMEM)));
    if (split) {
      if (a.p2) k_interp_box<true, true><<<unsigned(blocks), BOX_THREADS, BOX_SMEM, stream>>>(a, lev, plan);
      else k_interp_box<false, true><<<unsigned(blocks), BOX_THREADS, BOX_SMEM, stream>>>(a, lev, plan);
      if (a.p2) k_interp_global<true><<<unsigned(blocks * BOX_PPT), BOX_THREADS, 0, stream>>>(a, lev, plan);
      else k_interp_global<false><<<unsigned(blocks * BOX_PPT), BOX_THREADS, 0, stream>>>(a, lev, plan);
      count_launches(2);
    } else {
      if (a.p2) k_interp_box<true, false><<<unsigned(blocks), BOX_THREADS, BOX_SMEM, stream>>>(a, lev, plan);
      else k_interp_box<false, false><<<unsigned(blocks), BOX_THREADS, BOX_SMEM, stream>>>(a, lev, plan);
      count_launches(1);
    }
    SWENSE_CUDA_TRY(cudaGetLastError());
  }
  if (n_out_of_range) {
    unsigned long long h = 0;
    SWENSE_CUDA_TRY(cudaMemcpyAsync(&h, d_count, sizeof(h), cudaMemcpyDeviceToHost, stream));
    SWENSE_CUDA_TRY(cudaStreamSynchronize(stream));
    *n_out_of_range = int64_t(h);
  }
  return SWENSE_OK;
}

}  // namespace
}  // namespace swense

extern "C" int64_t swense_interp_plan_bytes(int64_t np) {
  return np <= 0 ? 0 : ((np + BOX_PTS - 1) / BOX_PTS) * int64_t(sizeof(int4));
}

extern "C" int swense_interp_plan(const swense_grid* g, const float* pts, int64_t np, void* plan,
                                  void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  InterpArgs a;
  Levels lev;
  const double t0 = g && g->t_levels ? g->t_levels[0] : 0.0;
  int st = prepare_interp(g, t0, pts, np, SWENSE_P_DYN, 1.0, 1.0, &a, &lev);
  if (st) return st;
  if (np == 0) return SWENSE_OK;
  if (!plan || (reinterpret_cast<uintptr_t>(plan) & 15)) return fail(SWENSE_ERR_ARG, "plan must be non-NULL and 16-byte aligned");
  const int64_t blocks = (np + BOX_PTS - 1) / BOX_PTS;
  if (blocks >= (int64_t(1) << 31)) return fail(SWENSE_ERR_SIZE, "too many points for one call");
  if (a.p2) k_interp_plan<true><<<unsigned(plan_blocks(np)), BOX_THREADS, 0, stream>>>(a, lev, static_cast<int4*>(plan));
  else k_interp_plan<false><<<unsigned(plan_blocks(np)), BOX_THREADS, 0, stream>>>(a, lev, static_cast<int4*>(plan));
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

extern "C" int swense_interp_with_plan(const swense_grid* g, double t, const float* pts, int64_t np,
                                       const void* plan, float* eta, float* u, float* v, float* w,
                                       float* p, int32_t p_mode, double rho, double grav,
                                       int64_t* n_out_of_range, void* stream) {
  if (np > 0 && (!plan || (reinterpret_cast<uintptr_t>(plan) & 15)))
    return fail(SWENSE_ERR_ARG, "plan must be non-NULL and 16-byte aligned");
  return interp_impl(g, t, pts, nullptr, np, eta, u, v, w, p, p_mode, rho, grav, n_out_of_range,
                     static_cast<cudaStream_t>(stream), static_cast<const int4*>(plan));
}

extern "C" int swense_interp(const swense_grid* g, double t, const float* pts, int64_t np,
                             float* eta, float* u, float* v, float* w, float* p, int32_t p_mode,
                             double rho, double grav, int64_t* n_out_of_range, void* stream) {
  return interp_impl(g, t, pts, nullptr, np, eta, u, v, w, p, p_mode, rho, grav, n_out_of_range,
                     static_cast<cudaStream_t>(stream));
}

extern "C" int swense_interp_permuted(const swense_grid* g, double t, const float* pts_sorted,
                                      const int32_t* perm, int64_t np, float* eta, float* u,
                                      float* v, float* w, float* p, int32_t p_mode, double rho,
                                      double grav, int64_t* n_out_of_range, void* stream) {
  if (np > 0 && !perm) return fail(SWENSE_ERR_ARG, "NULL perm");
  return interp_impl(g, t, pts_sorted, perm, np, eta, u, v, w, p, p_mode, rho, grav,
                     n_out_of_range, static_cast<cudaStream_t>(stream));
}

namespace swense {
namespace {

// Per device: the batch tables in device memory (instances' arguments and level tables, chunk
// offsets) and their host copy. Rewritten (synchronously, so never during a stream capture)
// only when a batch's tables differ from the last ones; a captured batch therefore replays the
// tables of the uncaptured call that preceded it.
struct BatchTables {
  void* dev = nullptr;
  size_t cap = 0;
  std::vector<double> key;          // the inputs the tables were built from
  int64_t nchunks = 0;
};

// Everything the batch tables depend on, field by field (no struct padding).
std::vector<double> batch_key(const GatherItem* items, int n, int32_t p_mode, double rho, double grav) {
  std::vector<double> k{double(n), double(p_mode), rho, grav};
  auto ptr = [&](const void* q) { k.push_back(double(reinterpret_cast<uintptr_t>(q))); };
  for (int i = 0; i < n; ++i) {
    const GatherItem& it = items[i];
    const swense_grid& g = it.grid;
    ptr(g.nodes); ptr(g.eta); ptr(it.pts); ptr(it.perm);
    ptr(it.eta); ptr(it.u); ptr(it.v); ptr(it.w); ptr(it.p);
    k.insert(k.end(), {double(it.np), it.t, double(g.nx_r), double(g.ny_r), double(g.nz), double(g.n_tl),
                       g.Lx, g.Ly, double(g.scheme)});
    for (int l = 0; l < g.nz && g.z_levels; ++l) k.push_back(double(g.z_levels[l]));
    for (int l = 0; l < g.n_tl && g.t_levels; ++l) k.push_back(g.t_levels[l]);
  }
  return k;
}
std::mutex g_batch_mutex;
BatchTables g_batch[64];

int batch_tables(const GatherItem* items, int n, int32_t p_mode, double rho, double grav, cudaStream_t stream,
                 const BatchInst** d_inst, const int64_t** d_chunk0, int64_t* nchunks) {
  int dev = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SWENSE_ERR_UNSUPPORTED, "device index too large");
  std::vector<double> key = batch_key(items, n, p_mode, rho, grav);
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  BatchTables& T = g_batch[dev];
  if (T.dev && T.key == key) {                      // the same batch as last time: tables in place
    *d_inst = static_cast<const BatchInst*>(T.dev);
    *d_chunk0 = reinterpret_cast<const int64_t*>(static_cast<const char*>(T.dev) + size_t(n) * sizeof(BatchInst));
    *nchunks = T.nchunks;
    return SWENSE_OK;
  }
  std::vector<unsigned char> h(size_t(n) * sizeof(BatchInst) + size_t(n + 1) * sizeof(int64_t));
  BatchInst* bi = reinterpret_cast<BatchInst*>(h.data());
  int64_t* c0 = reinterpret_cast<int64_t*>(h.data() + size_t(n) * sizeof(BatchInst));
  c0[0] = 0;
  for (int k = 0; k < n; ++k) {
    const GatherItem& it = items[k];
    InterpArgs a;
    Levels lev;
    int st = prepare_interp(&it.grid, it.t, it.pts, it.np, p_mode, rho, grav, &a, &lev);
    if (st) return st;
    if (!a.p2) return fail(SWENSE_ERR_UNSUPPORTED, "batched gathers take power-of-two node counts");
    a.o_eta = it.eta;
    a.o_u = it.u;
    a.o_v = it.v;
    a.o_w = it.w;
    a.o_p = it.p;
    a.perm = it.perm;
    a.n_oor = nullptr;
    std::memcpy(&bi[k].a, &a, sizeof(InterpArgs));
    std::memcpy(&bi[k].L, &lev, sizeof(Levels));
    c0[k + 1] = c0[k] + (it.np + BOX_PTS - 1) / BOX_PTS;
  }
  {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SWENSE_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
    if (cap != cudaStreamCaptureStatusNone)
      return fail(SWENSE_ERR_ARG, "a captured swense_batch_run must follow an uncaptured call with the "
                                  "same instances (its tables are uploaded outside the capture)");
    SWENSE_CUDA_TRY(cudaStreamSynchronize(stream));
    if (h.size() > T.cap) {
      if (T.dev) SWENSE_CUDA_TRY(cudaFree(T.dev));
      T.dev = nullptr;
      T.cap = 0;
      cudaError_t e = cudaMalloc(&T.dev, h.size());
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SWENSE_ERR_OOM, "cudaMalloc of the batch tables failed");
      }
      T.cap = h.size();
    }
    SWENSE_CUDA_TRY(cudaMemcpy(T.dev, h.data(), h.size(), cudaMemcpyHostToDevice));
    T.key.swap(key);
    T.nchunks = c0[n];
  }
  *d_inst = static_cast<const BatchInst*>(T.dev);
  *d_chunk0 = reinterpret_cast<const int64_t*>(static_cast<const char*>(T.dev) + size_t(n) * sizeof(BatchInst));
  *nchunks = T.nchunks;
  return SWENSE_OK;
}

}  // namespace

int interp_batch_bytes(const GatherItem* items, int n, size_t* bytes) {
  int64_t chunks = 0;
  for (int k = 0; k < n; ++k) chunks += (items[k].np + BOX_PTS - 1) / BOX_PTS;
  *bytes = 256 + size_t(chunks) * sizeof(int4);
  return SWENSE_OK;
}

int interp_batch(const GatherItem* items, int n, int32_t p_mode, double rho, double grav, void* ws,
                 cudaStream_t stream) {
  if (n <= 0) return SWENSE_OK;
  const BatchInst* d_inst = nullptr;
  const int64_t* d_chunk0 = nullptr;
  int64_t nchunks = 0;
  int st = batch_tables(items, n, p_mode, rho, grav, stream, &d_inst, &d_chunk0, &nchunks);
  if (st) return st;
  if (nchunks == 0) return SWENSE_OK;
  if (nchunks >= (int64_t(1) << 31)) return fail(SWENSE_ERR_SIZE, "too many point chunks in one batch");
  unsigned* counter = static_cast<unsigned*>(ws);
  int4* plan = reinterpret_cast<int4*>(static_cast<char*>(ws) + 256);
  const size_t plan_smem = size_t(PLAN_WARPS) * (sizeof(InterpArgs) + sizeof(LevelTables));
  SWENSE_CUDA_TRY(cudaFuncSetAttribute((const void*)k_interp_plan_batch,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(plan_smem)));
  k_interp_plan_batch<<<unsigned((nchunks + PLAN_WARPS - 1) / PLAN_WARPS), BOX_THREADS, plan_smem, stream>>>(
      d_inst, d_chunk0, n, plan);
  SWENSE_CUDA_TRY(cudaGetLastError());
  SWENSE_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), stream));
  SWENSE_CUDA_TRY(cudaFuncSetAttribute((const void*)k_interp_box_batch,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(BOX_SMEM)));
  int dev = 0, sms = 0, per_sm = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  SWENSE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SWENSE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interp_box_batch, BOX_THREADS,
                                                                BOX_SMEM));
  const int64_t ctas = std::min<int64_t>(nchunks, int64_t(std::max(1, sms * std::max(1, per_sm))));
  k_interp_box_batch<<<unsigned(ctas), BOX_THREADS, BOX_SMEM, stream>>>(d_inst, d_chunk0, n, plan, counter);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(2);
  return SWENSE_OK;
}

}  // namespace swense
