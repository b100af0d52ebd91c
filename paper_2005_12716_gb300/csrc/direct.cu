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
#include "mma.cuh"

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

// Weighted coefficients of slot i = r (nx/2 + 1) + m of the one-sided spectrum at time offset dt
// (linear propagation e^{-i omega dt} when omega is given). Nyquist slots return live = false.
struct SlotCoef {
  bool live;
  int m, n;
  float k, invd;
  float2 we, wu, wv, ww, wt;
};

__device__ __forceinline__ SlotCoef slot_coef(int i, const float2* __restrict__ Ae,
                                              const float2* __restrict__ Ap, const float2* __restrict__ At,
                                              const double* __restrict__ omega, double dt, int nx, int ny,
                                              float kxs, float kys, float depth) {
  const int nxh1 = nx / 2 + 1;
  const int r = i / nxh1, m = i - r * nxh1;
  SlotCoef sc{};
  sc.live = !(m >= nx / 2 || (ny > 1 && r == ny / 2));    // Nyquist slots are ignored
  sc.invd = 1.f;
  if (!sc.live) return sc;
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
  sc.m = m;
  sc.n = n;
  sc.k = k;
  sc.invd = depth > 0.f ? 1.f / (1.f + expf(-2.f * k * depth)) : 1.f;
  sc.we = make_float2(wgt * e.x, wgt * e.y);
  sc.wu = make_float2(-wgt * kx * p.y, wgt * kx * p.x);     // c i kx A^phi
  sc.wv = make_float2(-wgt * ky * p.y, wgt * ky * p.x);     // c i ky A^phi
  sc.ww = make_float2(wgt * k * p.x, wgt * k * p.y);        // c |k| A^phi
  sc.wt = make_float2(wgt * t.x, wgt * t.y);                // c A^phit
  return sc;
}

__global__ void k_direct_prep(const float2* __restrict__ Ae, const float2* __restrict__ Ap,
                              const float2* __restrict__ At, const double* __restrict__ omega,
                              double dt, int nx, int ny, float kxs, float kys, float depth,
                              ModeCoef* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ny * (nx / 2 + 1)) return;
  const SlotCoef sc = slot_coef(i, Ae, Ap, At, omega, dt, nx, ny, kxs, kys, depth);
  ModeCoef mc;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!sc.live) {
    mc.c0 = make_float4(__int_as_float(0), __int_as_float(0), 0.f, 1.f);
    mc.c1 = mc.c2 = mc.c3 = zero;
    out[i] = mc;
    return;
  }
  mc.c0 = make_float4(__int_as_float(sc.m), __int_as_float(sc.n), sc.k, sc.invd);
  mc.c1 = make_float4(sc.we.x, sc.we.y, sc.wu.x, sc.wu.y);
  mc.c2 = make_float4(sc.wv.x, sc.wv.y, sc.ww.x, sc.ww.y);
  mc.c3 = make_float4(sc.wt.x, sc.wt.y, 0.f, 0.f);
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

// ------------------------------------------------------------------------------------------------
// Split-BF16 tensor-core path. The sums over modes are a contraction of the points-by-(mode,
// re/im) matrix A[p][2j] = cos(theta_pj) f_j(z_p), A[p][2j+1] = sin(theta_pj) f_j(z_p) with the
// (mode, re/im)-by-field matrix B[2j][c] = Re W_c[j], B[2j+1][c] = -Im W_c[j], c = u, v, w, phi_t
// (columns 4..7 zero). A is generated in registers directly in the m16n8k16 fragment layout (no
// shared-memory round trip) and both operands are split into BF16 hi + lo; three MMAs
// (hi.hi + hi.lo + lo.hi) accumulate in FP32, which leaves a relative error of about 2^-16 per
// product. eta has no depth factor and one column, so it is summed in FP32 on the side from the
// same phases. Finite depth writes the factors as a + b and a - b with a = e^{kz} / (1 + e^{-2kh})
// and b = a e^{-2k(z+h)} (so f = a + b for u, v, phi_t and g = a - b for w): A carries (cos, sin)
// times a and times b, and B's w column takes the sign flip on the b half.
//
// Table: modes in rows of constant n (Nyquist row skipped), m = 0 .. nx/2 - 1 padded with zero
// modes to a multiple of 8, cut into k-steps of KM = 8 modes (deep) or 4 modes (finite depth).
// Lane (g, q) of a k-step holds modes q and q + 4 (deep) or mode q in its a and b halves.
struct SplitStep {
  uint4 b[32];      // per lane: (b0 hi, b1 hi, b0 lo, b1 lo)
  float4 info[8];   // per mode of the step: (|k| log2 e, 1 / (1 + e^{-2kh}), W_eta)
};
static_assert(sizeof(SplitStep) == 640, "split step record");

constexpr int kSplitThreads = 256;
constexpr int kSplitTiles = 2;     // 16-point MMA tiles per warp
constexpr int kSplitStage = 32;    // k-steps per shared-memory stage (double-buffered)
constexpr int kSplitAnchor = 16;   // exact phase every this many k-steps

// 2^x (PTX ex2.approx: relative error about 2^-22, far below the split products' 2^-16)
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float2 pick_w(const SlotCoef& sc, int c) {
  return c == 0 ? sc.wu : c == 1 ? sc.wv : c == 2 ? sc.ww : c == 3 ? sc.wt : make_float2(0.f, 0.f);
}

__global__ void k_direct_prep_split(const float2* __restrict__ Ae, const float2* __restrict__ Ap,
                                    const float2* __restrict__ At, const double* __restrict__ omega,
                                    double dt, int nx, int ny, float kxs, float kys, float depth,
                                    int km, int spr, int nsteps, SplitStep* __restrict__ out) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  if (gt >= nsteps * 32) return;
  const int s = gt >> 5, L = gt & 31;
  const int ri = s / spr, m0 = (s - ri * spr) * km;
  const int r = (ny > 1 && ri >= ny / 2) ? ri + 1 : ri;
  const int nxh1 = nx / 2 + 1;
  auto coef = [&](int j) {
    const int m = m0 + j;
    SlotCoef sc{};
    if (m < nx / 2) sc = slot_coef(r * nxh1 + m, Ae, Ap, At, omega, dt, nx, ny, kxs, kys, depth);
    return sc;                                   // not live: all weights zero
  };
  const int g = L >> 2, q = L & 3;
  const SlotCoef s0 = coef(q);
  const float2 w0 = pick_w(s0, g);
  float2 w1;
  if (km == 8) {
    w1 = pick_w(coef(q + 4), g);
  } else {
    w1 = g == 2 ? make_float2(-w0.x, -w0.y) : w0;    // b half: w column changes sign
  }
  unsigned h0, l0, h1, l1;
  bf2_split(w0.x, -w0.y, h0, l0);
  bf2_split(w1.x, -w1.y, h1, l1);
  out[s].b[L] = make_uint4(h0, h1, l0, l1);
  if (L < 8) {
    float4 inf = make_float4(0.f, 1.f, 0.f, 0.f);
    if (L < km) {
      const SlotCoef sc = coef(L);
      if (sc.live) inf = make_float4(sc.k * 1.4426950408889634f, sc.invd, sc.we.x, sc.we.y);
    }
    out[s].info[L] = inf;
  }
}

struct SplitArgs {
  const SplitStep* steps;
  int nsteps, spr, ny;
  const float* pts;
  float *o_eta, *o_u, *o_v, *o_w, *o_p;
  int64_t np;
  double inv_lx, inv_ly;
  float depth;
  int p_mode;
  float rho, g;
  // points sorted by the tensor-core path: output i goes to perm[i], and only the tiles of
  // tile_pts points that tile_bad marks are written (NULL: caller's order, every point)
  const int32_t* perm;
  const uint8_t* tile_bad;
  int tile_pts;
};

template <bool FINITE>
__global__ void __launch_bounds__(kSplitThreads, 2) k_direct_split(SplitArgs a) {
  constexpr int KM = FINITE ? 4 : 8;
  constexpr int TT = kSplitTiles;
  constexpr int JN = FINITE ? 1 : 2;               // modes per lane per k-step
  __shared__ SplitStep stage[2][kSplitStage];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int64_t pbase = (int64_t(blockIdx.x) * (kSplitThreads / 32) + warp) * (16 * TT);
  bool write = true;
  if (a.tile_bad) {
    // the block's points span whole warps of one tile each; leave at once (before any barrier)
    // unless one of the block's tiles is marked
    const int64_t b0 = int64_t(blockIdx.x) * (kSplitThreads / 32) * (16 * TT);
    const int64_t t0 = b0 / a.tile_pts, t1 = (std::min(b0 + (kSplitThreads / 32) * (16 * TT), a.np) - 1) / a.tile_pts;
    bool any = false;
    for (int64_t tt = t0; tt <= t1; ++tt) any |= a.tile_bad[tt] != 0;
    if (!any) return;
    write = pbase < a.np && a.tile_bad[pbase / a.tile_pts] != 0;
  }

  unsigned X[TT][2], Y[TT][2];
  float z[TT][2], stc[TT][2], sts[TT][2];
  float pc[TT][2][JN], ps[TT][2][JN];
#pragma unroll
  for (int t = 0; t < TT; ++t)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = pbase + 16 * t + g + 8 * h;
      float x = 0.f, y = 0.f, zz = 0.f;
      if (i < a.np) {
        x = a.pts[3 * i];
        y = a.pts[3 * i + 1];
        zz = a.pts[3 * i + 2];
      }
      X[t][h] = turn_fraction(x, a.inv_lx);
      Y[t][h] = turn_fraction(y, a.inv_ly);
      z[t][h] = zz;
      // phase step for m -> m + KM
      sincospif(2.f * (float(int(unsigned(KM) * X[t][h])) * 2.3283064365386963e-10f), &sts[t][h], &stc[t][h]);
#pragma unroll
      for (int j = 0; j < JN; ++j) pc[t][h][j] = 1.f, ps[t][h][j] = 0.f;
    }
  float run[TT][4], eta_run[TT][2];
#pragma unroll
  for (int t = 0; t < TT; ++t) {
#pragma unroll
    for (int e = 0; e < 4; ++e) run[t][e] = 0.f;
    eta_run[t][0] = eta_run[t][1] = 0.f;
  }

  const int nchunks = (a.nsteps + kSplitStage - 1) / kSplitStage;
  auto load_chunk = [&](int c) {
    const int cnt = min(kSplitStage, a.nsteps - c * kSplitStage);
    const uint4* src = reinterpret_cast<const uint4*>(a.steps + size_t(c) * kSplitStage);
    uint4* dst = reinterpret_cast<uint4*>(stage[c & 1]);
    for (int v = threadIdx.x; v < cnt * 40; v += kSplitThreads) cp_async16(dst + v, src + v, 16);
    cp_async_commit();
  };
  load_chunk(0);
  int ri = 0, sidx = 0;                             // table row and step within it of step s
  for (int c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      load_chunk(c + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const SplitStep* st = stage[c & 1];
    const int cnt = min(kSplitStage, a.nsteps - c * kSplitStage);
    float acc[TT][4], eta_acc[TT][2];
#pragma unroll
    for (int t = 0; t < TT; ++t) {
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[t][e] = 0.f;
      eta_acc[t][0] = eta_acc[t][1] = 0.f;
    }
    for (int sl = 0; sl < cnt; ++sl) {
      if (sidx % kSplitAnchor == 0) {
        // exact phase (m X + n Y) mod 2^32 of this lane's modes
        const int r = (a.ny > 1 && ri >= a.ny / 2) ? ri + 1 : ri;
        const int n = a.ny > 1 ? (r < a.ny / 2 ? r : r - a.ny) : 0;
#pragma unroll
        for (int t = 0; t < TT; ++t)
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < JN; ++j) {
              const unsigned m = unsigned(sidx * KM + q + 4 * j);
              const unsigned ph = m * X[t][h] + unsigned(n) * Y[t][h];
              sincospif(2.f * (float(int(ph)) * 2.3283064365386963e-10f), &ps[t][h][j], &pc[t][h][j]);
            }
      } else {
#pragma unroll
        for (int t = 0; t < TT; ++t)
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < JN; ++j) {
              const float c2 = fmaf(pc[t][h][j], stc[t][h], -ps[t][h][j] * sts[t][h]);
              ps[t][h][j] = fmaf(ps[t][h][j], stc[t][h], pc[t][h][j] * sts[t][h]);
              pc[t][h][j] = c2;
            }
      }
      const uint4 bf = st[sl].b[lane];
      float4 inf[JN];
#pragma unroll
      for (int j = 0; j < JN; ++j) inf[j] = st[sl].info[q + 4 * j];
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        float v[2][2][2];                          // [register pair][h][cos/sin]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float zz = z[t][h];
          if constexpr (!FINITE) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const float f = ex2(inf[j].x * zz);
              v[j][h][0] = pc[t][h][j] * f;
              v[j][h][1] = ps[t][h][j] * f;
              eta_acc[t][h] = fmaf(inf[j].z, pc[t][h][j], fmaf(-inf[j].w, ps[t][h][j], eta_acc[t][h]));
            }
          } else {
            const float k = inf[0].x;
            const float fa = ex2(k * zz) * inf[0].y;
            const float fb = fa * ex2(-2.f * k * (zz + a.depth));
            v[0][h][0] = pc[t][h][0] * fa;
            v[0][h][1] = ps[t][h][0] * fa;
            v[1][h][0] = pc[t][h][0] * fb;
            v[1][h][1] = ps[t][h][0] * fb;
            eta_acc[t][h] = fmaf(inf[0].z, pc[t][h][0], fmaf(-inf[0].w, ps[t][h][0], eta_acc[t][h]));
          }
        }
        unsigned ahi[4], alo[4];
        bf2_split(v[0][0][0], v[0][0][1], ahi[0], alo[0]);   // (g, 2q..2q+1)
        bf2_split(v[0][1][0], v[0][1][1], ahi[1], alo[1]);   // (g+8, 2q..2q+1)
        bf2_split(v[1][0][0], v[1][0][1], ahi[2], alo[2]);   // (g, 2q+8..2q+9)
        bf2_split(v[1][1][0], v[1][1][1], ahi[3], alo[3]);   // (g+8, 2q+8..2q+9)
        mma16816(acc[t], ahi, bf.x, bf.y);
        mma16816(acc[t], ahi, bf.z, bf.w);
        mma16816(acc[t], alo, bf.x, bf.y);
      }
      if (++sidx == a.spr) {                       // next step: next table row
        sidx = 0;
        ++ri;
      }
    }
#pragma unroll
    for (int t = 0; t < TT; ++t) {
#pragma unroll
      for (int e = 0; e < 4; ++e) run[t][e] += acc[t][e];
      eta_run[t][0] += eta_acc[t][0];
      eta_run[t][1] += eta_acc[t][1];
    }
    __syncthreads();                               // stage (c & 1) is reloaded next iteration
  }

#pragma unroll
  for (int t = 0; t < TT; ++t) {
    float e0 = eta_run[t][0], e1 = eta_run[t][1];
    e0 += __shfl_xor_sync(0xffffffffu, e0, 1);
    e0 += __shfl_xor_sync(0xffffffffu, e0, 2);
    e1 += __shfl_xor_sync(0xffffffffu, e1, 1);
    e1 += __shfl_xor_sync(0xffffffffu, e1, 2);
    // lane q = 0 holds (u, v) of rows g and g + 8, lane q = 1 holds (w, phi_t)
    const float w0 = __shfl_down_sync(0xffffffffu, run[t][0], 1);
    const float t0 = __shfl_down_sync(0xffffffffu, run[t][1], 1);
    const float w1 = __shfl_down_sync(0xffffffffu, run[t][2], 1);
    const float t1 = __shfl_down_sync(0xffffffffu, run[t][3], 1);
    if (q != 0 || !write) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t ii = pbase + 16 * t + g + 8 * h;
      if (ii >= a.np) continue;
      const int64_t i = a.perm ? int64_t(a.perm[ii]) : ii;
      const float uu = run[t][2 * h], vv = run[t][2 * h + 1];
      const float ww = h ? w1 : w0, tt = h ? t1 : t0;
      if (a.o_eta) a.o_eta[i] = h ? e1 : e0;
      if (a.o_u) a.o_u[i] = uu;
      if (a.o_v) a.o_v[i] = vv;
      if (a.o_w) a.o_w[i] = ww;
      if (a.o_p) {
        float p;
        if (a.p_mode == SWENSE_P_PHIT) {
          p = tt;
        } else {
          p = -a.rho * (tt + 0.5f * (uu * uu + vv * vv + ww * ww));
          if (a.p_mode == SWENSE_P_TOTAL) p -= a.rho * a.g * z[t][h];
        }
        a.o_p[i] = p;
      }
    }
  }
}

}  // namespace
}  // namespace swense

using namespace swense;

namespace {

int direct_split_impl(const swense_modes* md, double t, const float* pts, const int32_t* perm,
                      const uint8_t* tile_bad, int tile_pts, int64_t np, float* eta, float* u,
                      float* v, float* w, float* p, int32_t p_mode, double rho, double grav,
                      cudaStream_t stream, size_t ws_offset) {
  const int nx = md->nx, ny = md->ny;
  const bool finite = md->depth > 0;
  const int km = finite ? 4 : 8;
  const int rm = ((nx / 2 + 7) / 8) * 8;        // modes per table row, padded to a multiple of 8
  const int spr = rm / km;
  const int nrows = ny > 1 ? ny - 1 : 1;        // Nyquist row skipped
  const int64_t nsteps = int64_t(nrows) * spr;
  if (nsteps * 32 >= (int64_t(1) << 31)) return fail(SWENSE_ERR_SIZE, "too many modes for the split table");
  void* ws = nullptr;
  int st = workspace(ws_offset + size_t(nsteps) * sizeof(SplitStep), stream, &ws);
  if (st) return st;
  SplitStep* steps = reinterpret_cast<SplitStep*>(static_cast<char*>(ws) + ws_offset);
  const float depth = finite ? float(md->depth) : 0.f;
  k_direct_prep_split<<<unsigned((nsteps * 32 + 255) / 256), 256, 0, stream>>>(
      reinterpret_cast<const float2*>(md->A_eta), reinterpret_cast<const float2*>(md->A_phi),
      reinterpret_cast<const float2*>(md->A_phit), md->omega, t - md->t_ref, nx, ny,
      float(6.283185307179586476925 / md->Lx), ny > 1 ? float(6.283185307179586476925 / md->Ly) : 0.f,
      depth, km, spr, int(nsteps), steps);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  SplitArgs a{};
  a.steps = steps;
  a.nsteps = int(nsteps);
  a.spr = spr;
  a.ny = ny;
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
  a.perm = perm;
  a.tile_bad = tile_bad;
  a.tile_pts = tile_pts;
  const int64_t per_cta = int64_t(kSplitThreads / 32) * 16 * kSplitTiles;
  const int64_t blocks = (np + per_cta - 1) / per_cta;
  if (blocks >= (int64_t(1) << 31)) return fail(SWENSE_ERR_SIZE, "too many points for one call");
  if (finite) k_direct_split<true><<<unsigned(blocks), kSplitThreads, 0, stream>>>(a);
  else k_direct_split<false><<<unsigned(blocks), kSplitThreads, 0, stream>>>(a);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

}  // namespace

namespace swense {

size_t split_table_bytes(const swense_modes* md) {
  const int km = md->depth > 0 ? 4 : 8;
  const int rm = ((md->nx / 2 + 7) / 8) * 8;
  const int nrows = md->ny > 1 ? md->ny - 1 : 1;
  return size_t(nrows) * (rm / km) * sizeof(SplitStep);
}

int direct_split_sorted(const swense_modes* md, double t, const float* srt, const int32_t* perm,
                        const uint8_t* tile_bad, int tile_pts, int64_t np, float* eta, float* u, float* v,
                        float* w, float* p, int32_t p_mode, double rho, double grav, cudaStream_t stream,
                        size_t ws_offset) {
  static_assert((kSplitThreads / 32) * 16 * kSplitTiles % 32 == 0, "warps of 32 points");
  if (tile_pts % (16 * kSplitTiles)) return fail(SWENSE_ERR_ARG, "tile size");
  // the workspace already holds the sorted points and the tensor-core path's tables, which this
  // launch reads: its own table goes at ws_offset, after them (the caller sized the workspace for
  // both, so that nothing here grows it and frees the buffers in use)
  return direct_split_impl(md, t, srt, perm, tile_bad, tile_pts, np, eta, u, v, w, p, p_mode, rho, grav,
                           stream, ws_offset);
}

}  // namespace swense

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
  if (precision != SWENSE_DIRECT_FP32 && precision != SWENSE_DIRECT_SPLIT_BF16 &&
      precision != SWENSE_DIRECT_SPLIT_BF16_PAIRWISE)
    return fail(SWENSE_ERR_ARG, "unknown precision");
  if (np == 0) return SWENSE_OK;
  if (precision == SWENSE_DIRECT_SPLIT_BF16)
    return direct_tc(md, t, pts, np, eta, u, v, w, p, p_mode, rho, grav, stream);
  if (precision == SWENSE_DIRECT_SPLIT_BF16_PAIRWISE)
    return direct_split_impl(md, t, pts, nullptr, nullptr, 0, np, eta, u, v, w, p, p_mode, rho, grav, stream, 0);
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
