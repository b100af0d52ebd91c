// Stage 1 of the reconstruction: modal amplitudes -> (zero-padded) grid at arbitrary levels.
//
// Paper: reconstruction section, step "IFFT" (one inverse transform per vertical level onto
// uniformly spaced nodes), the zero-padding refinement (spectrum extended n times with zero
// modes -> n times finer grid) and the extension of the solution above z = 0.
//
// Two passes per level chunk (3-D, ny > 1):
//   pass A  per (level, block of kx columns): form the four modal fields
//             U = i kx A^phi F, V = i ky A^phi F, W = |k| A^phi S, T = A^phit F
//           (depth factors F, S at the level), zero-pad along ky and inverse-transform along y;
//           writes G[level][field][y][m] (complex, one-sided in m) to the scratch workspace.
//   pass B  per (level, block of y rows): pack the two real-field pairs into one complex
//           spectrum each, Z1 = U + iV and Z2 = W + iT (Hermitian extension over m, zero-padded
//           to nx_r), inverse-transform along x and store float4 (u, v, w, dphi/dt) per node.
// Level chunks are sized so G stays L2-resident between the passes. eta is one extra transform
// per time level (pass A on A^eta; pass B packs two grid rows per complex transform).
// 2-D (ny == 1): pass B alone, reading the modes directly.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <string>

#include "fft.cuh"
#include "internal.cuh"
#include "tma.cuh"

namespace swense {
namespace {

struct Levels {
  float z[SWENSE_MAX_LEVELS];
};

struct PassAArgs {
  const float2* A_phi;   // [ny][nxh1] of this time level
  const float2* A_phit;
  const float2* A_eta;
  float2* G;             // [nlev][4][Nyr][Mh] (levels) or [Nyr][Mh] (eta)
  const float2* tw;
  int ny, nxh1, Mh, Nyr, log2Nyr;
  int cb, fp;            // kx columns per CTA, fields per shared-memory pass
  int lev0;              // first level of the chunk
  int eta_mode;
  float kxs, kys, depth;
  int Nxr, spline;       // spline: store cubic B-spline coefficients (modes prefiltered)
};

__global__ void __launch_bounds__(256) k_pass_a(PassAArgs a, Levels L) {
  extern __shared__ float2 sm[];
  const int c0 = blockIdx.x * a.cb;
  const int slot = blockIdx.y;
  const int ncol = min(a.cb, a.Mh - c0);
  const float z = a.eta_mode ? 0.f : L.z[a.lev0 + slot];
  const int nfield = a.eta_mode ? 1 : 4;
  const int nyh = a.ny >> 1;
  for (int f0 = 0; f0 < nfield; f0 += a.fp) {
    const int nf = min(a.fp, nfield - f0);
    const int narr = nf * a.cb;
    for (int i = threadIdx.x; i < narr * a.Nyr; i += blockDim.x) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = threadIdx.x; i < a.ny * a.cb; i += blockDim.x) {
      const int c = i % a.cb, r = i / a.cb;
      if (c >= ncol || r == nyh) continue;               // Nyquist row ignored
      const int m = c0 + c;
      const int n = r < nyh ? r : r - a.ny;
      const int pos = n >= 0 ? n : a.Nyr + n;            // zero-padding between +n and -n
      const unsigned br = bitrev(unsigned(pos), a.log2Nyr);
      const size_t gi = size_t(r) * a.nxh1 + m;
      const float pf = a.spline ? spline_prefilter(m, a.Nxr, n, a.Nyr) : 1.f;
      if (a.eta_mode) {
        const float2 e = __ldg(&a.A_eta[gi]);
        sm[c * a.Nyr + br] = make_float2(pf * e.x, pf * e.y);
        continue;
      }
      float2 Ap = __ldg(&a.A_phi[gi]);
      float2 At = __ldg(&a.A_phit[gi]);
      Ap = make_float2(pf * Ap.x, pf * Ap.y);
      At = make_float2(pf * At.x, pf * At.y);
      const float kx = float(m) * a.kxs, ky = float(n) * a.kys;
      const float k = sqrtf(kx * kx + ky * ky);
      float F, S;
      depth_factors(k, z, a.depth, F, S);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q < f0 || q >= f0 + nf) continue;
        float2 v;
        if (q == 0) v = make_float2(-kx * F * Ap.y, kx * F * Ap.x);        // i kx F A^phi
        else if (q == 1) v = make_float2(-ky * F * Ap.y, ky * F * Ap.x);   // i ky F A^phi
        else if (q == 2) v = make_float2(k * S * Ap.x, k * S * Ap.y);      // |k| S A^phi
        else v = make_float2(F * At.x, F * At.y);                          // F A^phit
        sm[((q - f0) * a.cb + c) * a.Nyr + br] = v;
      }
    }
    __syncthreads();
    fft_inv_inplace(sm, a.Nyr, a.log2Nyr, narr, a.tw);
    for (int i = threadIdx.x; i < nf * a.Nyr * a.cb; i += blockDim.x) {
      const int c = i % a.cb;
      const int rest = i / a.cb;
      const int y = rest % a.Nyr, q = rest / a.Nyr;
      if (c >= ncol) continue;
      const size_t go = ((size_t(slot) * nfield + f0 + q) * a.Nyr + y) * a.Mh + c0 + c;
      a.G[go] = sm[(q * a.cb + c) * a.Nyr + y];
    }
    __syncthreads();
  }
}

enum { B_LEVEL_G = 0, B_LEVEL_DIRECT = 1, B_ETA_G = 2, B_ETA_DIRECT = 3 };

struct PassBArgs {
  const float2* G;        // pass-A output (levels or eta)
  const float2* A_phi;    // direct mode (ny == 1): modes of this time level
  const float2* A_phit;
  const float2* A_eta;
  float4* nodes;          // [nz][Nyr][Nxr] of this time level
  float* eta;             // [Nyr][Nxr] of this time level
  const float2* tw;
  int Mh, Nxr, log2Nxr, Nyr;
  int rb;                 // rows (level modes) or row pairs (eta modes) per CTA
  int lev0;
  int mode;
  float kxs, depth;
  int spline;
};

// Hermitian packing of two one-sided spectra P, Q (coefficients of real fields p, q) into one
// full complex spectrum Z = P + iQ whose inverse transform is p + i q.
__device__ __forceinline__ void pack_pair(float2* Z, int m, int Nxr, int log2Nxr, float2 P, float2 Q) {
  if (m == 0) {
    Z[0] = make_float2(P.x, Q.x);                        // bitrev(0) == 0; real parts only
  } else {
    Z[bitrev(unsigned(m), log2Nxr)] = make_float2(P.x - Q.y, P.y + Q.x);
    Z[bitrev(unsigned(Nxr - m), log2Nxr)] = make_float2(P.x + Q.y, Q.x - P.y);
  }
}

__global__ void __launch_bounds__(256) k_pass_b(PassBArgs a, Levels L) {
  extern __shared__ float2 sm[];
  const int slot = blockIdx.y;
  const bool eta_mode = a.mode >= B_ETA_G;
  const int rows_per_cta = eta_mode ? 2 * a.rb : a.rb;
  const int y0 = blockIdx.x * rows_per_cta;
  const int narr = eta_mode ? a.rb : 2 * a.rb;
  for (int i = threadIdx.x; i < narr * a.Nxr; i += blockDim.x) sm[i] = make_float2(0.f, 0.f);
  __syncthreads();
  if (!eta_mode) {
    const float z = L.z[a.lev0 + slot];
    for (int i = threadIdx.x; i < a.rb * a.Mh; i += blockDim.x) {
      const int m = i % a.Mh, rr = i / a.Mh;
      const int y = y0 + rr;
      if (y >= a.Nyr) continue;
      float2 U, V, W, T;
      if (a.mode == B_LEVEL_G) {
        const size_t base = (size_t(slot) * 4 * a.Nyr + y) * a.Mh + m;
        const size_t fs = size_t(a.Nyr) * a.Mh;
        U = __ldcg(&a.G[base]);
        V = __ldcg(&a.G[base + fs]);
        W = __ldcg(&a.G[base + 2 * fs]);
        T = __ldcg(&a.G[base + 3 * fs]);
      } else {
        const float pf = a.spline ? spline_prefilter(m, a.Nxr, 0, 1) : 1.f;
        float2 Ap = __ldg(&a.A_phi[m]);
        float2 At = __ldg(&a.A_phit[m]);
        Ap = make_float2(pf * Ap.x, pf * Ap.y);
        At = make_float2(pf * At.x, pf * At.y);
        const float kx = float(m) * a.kxs;
        float F, S;
        depth_factors(kx, z, a.depth, F, S);
        U = make_float2(-kx * F * Ap.y, kx * F * Ap.x);
        V = make_float2(0.f, 0.f);
        W = make_float2(kx * S * Ap.x, kx * S * Ap.y);
        T = make_float2(F * At.x, F * At.y);
      }
      pack_pair(sm + size_t(2 * rr) * a.Nxr, m, a.Nxr, a.log2Nxr, U, V);
      pack_pair(sm + size_t(2 * rr + 1) * a.Nxr, m, a.Nxr, a.log2Nxr, W, T);
    }
  } else {
    for (int i = threadIdx.x; i < a.rb * a.Mh; i += blockDim.x) {
      const int m = i % a.Mh, pp = i / a.Mh;
      const int ya = y0 + 2 * pp, yb = ya + 1;
      if (ya >= a.Nyr) continue;
      float2 Ea, Eb = make_float2(0.f, 0.f);
      if (a.mode == B_ETA_G) {
        Ea = __ldcg(&a.G[size_t(ya) * a.Mh + m]);
        if (yb < a.Nyr) Eb = __ldcg(&a.G[size_t(yb) * a.Mh + m]);
      } else {
        const float pf = a.spline ? spline_prefilter(m, a.Nxr, 0, 1) : 1.f;
        Ea = __ldg(&a.A_eta[m]);
        Ea = make_float2(pf * Ea.x, pf * Ea.y);
      }
      pack_pair(sm + size_t(pp) * a.Nxr, m, a.Nxr, a.log2Nxr, Ea, Eb);
    }
  }
  __syncthreads();
  fft_inv_inplace(sm, a.Nxr, a.log2Nxr, narr, a.tw);
  if (!eta_mode) {
    float4* out = a.nodes + size_t(a.lev0 + slot) * a.Nyr * a.Nxr;
    for (int i = threadIdx.x; i < a.rb * a.Nxr; i += blockDim.x) {
      const int x = i % a.Nxr, rr = i / a.Nxr;
      const int y = y0 + rr;
      if (y >= a.Nyr) continue;
      const float2 z1 = sm[size_t(2 * rr) * a.Nxr + x];
      const float2 z2 = sm[size_t(2 * rr + 1) * a.Nxr + x];
      // 2-D: v is identically zero (the imaginary part of z1 holds only round-off)
      const float v = a.mode == B_LEVEL_DIRECT ? 0.f : z1.y;
      __stcs(&out[size_t(y) * a.Nxr + x], make_float4(z1.x, v, z2.x, z2.y));
    }
  } else {
    for (int i = threadIdx.x; i < a.rb * a.Nxr; i += blockDim.x) {
      const int x = i % a.Nxr, pp = i / a.Nxr;
      const int ya = y0 + 2 * pp, yb = ya + 1;
      if (ya >= a.Nyr) continue;
      const float2 zz = sm[size_t(pp) * a.Nxr + x];
      __stcs(&a.eta[size_t(ya) * a.Nxr + x], zz.x);
      if (yb < a.Nyr) __stcs(&a.eta[size_t(yb) * a.Nxr + x], zz.y);
    }
  }
}

// Linear propagation of stored modes: A(t) = A(t_ref) e^{-i omega (t - t_ref)}, every time level
// in one launch (blockIdx.y). The phase is reduced to turns in FP64 (exact enough for long
// simulated times); the rotation is FP32.
struct PropTimes {
  double dt[64];       // t_l - t_ref per time level (a grid request has at most 64)
};
__global__ void k_propagate(const float2* __restrict__ Ae, const float2* __restrict__ Ap,
                            const float2* __restrict__ At, const double* __restrict__ omega,
                            int nslot, PropTimes T, float2* __restrict__ out_all) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nslot) return;
  const double dt = T.dt[blockIdx.y];
  float2* out = out_all + size_t(blockIdx.y) * 3 * nslot;
  const double turns = omega[i] * dt * 0.15915494309189533577;  // theta / (2 pi)
  const double frac = turns - rint(turns);
  float s, c;
  sincospif(2.f * float(frac), &s, &c);
  const float2 src[3] = {Ae[i], Ap[i], At[i]};
#pragma unroll
  for (int q = 0; q < 3; ++q)
    out[size_t(q) * nslot + i] =
        make_float2(fmaf(src[q].x, c, src[q].y * s), fmaf(src[q].y, c, -src[q].x * s));
}

constexpr int kThreads = 256;
constexpr size_t kSmemBudget = 64 * 1024;
constexpr size_t kChunkBytes = size_t(64) << 20;
constexpr int kColBlock = 8;    // kx columns per column-transform CTA
constexpr int kColLevels = 2;   // levels per column-transform CTA
constexpr int kRowBlock = 8;    // grid rows per row-transform CTA (one per warp)

int set_smem(const void* fn, size_t bytes) {
  SWENSE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return SWENSE_OK;
}


// ------------------------------------------------------------------------------------------------
// Warp-register path for 32 <= ny_r, nx_r <= 1024 (one transform per warp, no shared-memory
// butterflies). Intermediate layout G2[level][field][m][y] (y contiguous): a column transform
// writes its warp's outputs as contiguous runs; the row kernel stages rb rows of all m.

// 8-byte asynchronous global -> shared copy (zero-filled when src_bytes == 0).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int src_bytes) {
  const unsigned d = unsigned(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

struct ColArgs {
  const float2* A_phi;   // [ny][nxh1] of this time level
  const float2* A_phit;
  float2* G;             // [nlev][4][Mh][Nyr]
  const float2* tw;
  int ny, nxh1, Mh, Nyr;
  int cb, lpc;           // kx columns and levels per CTA
  int lev0, nlev;        // chunk
  float kxs, kys, depth;
  int Nxr, spline;
  int ldG;               // m stride of the transposed intermediate (k_col_t)
};

// Modal field q at (kx, ky, |k|) with depth factors F, S: U = i kx F A, V = i ky F A,
// W = |k| S A, T = F A_t.
__device__ __forceinline__ float2 modal_field(int q, float kx, float ky, float k, float F, float S,
                                              float2 Ap, float2 At) {
  if (q == 0) return make_float2(-kx * F * Ap.y, kx * F * Ap.x);
  if (q == 1) return make_float2(-ky * F * Ap.y, ky * F * Ap.x);
  if (q == 2) return make_float2(k * S * Ap.x, k * S * Ap.y);
  return make_float2(F * At.x, F * At.y);
}

template <int E, int NF>
__global__ void __launch_bounds__(256, 2) k_col_fft(ColArgs a, Levels L) {
  extern __shared__ float2 sm[];                 // [2][ny][cb + 1]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * kColBlock;
  const int ncol = min(kColBlock, a.Mh - c0);
  const int ld = kColBlock + 1;
  for (int i = threadIdx.x; i < a.ny * kColBlock; i += blockDim.x) {
    const int c = i % kColBlock, r = i / kColBlock;
    const bool ok = c < ncol;
    const size_t gi = ok ? size_t(r) * a.nxh1 + c0 + c : 0;
    cp_async8(&sm[r * ld + c], &a.A_phi[gi], ok ? 8 : 0);
    cp_async8(&sm[(a.ny + r) * ld + c], &a.A_phit[gi], ok ? 8 : 0);
  }
  WarpFftTw<E> T;
  warp_fft_init<E>(T, a.tw, lane);
  cp_async_wait_all();
  __syncthreads();
  const int nyh = a.ny >> 1;
  const int groups = 4 / NF;
  const int ntask = a.lpc * kColBlock * groups;
  for (int task = warp; task < ntask; task += blockDim.x >> 5) {
    const int g = task % groups;
    const int rest = task / groups;
    const int c = rest % kColBlock;
    const int level = blockIdx.y * a.lpc + rest / kColBlock;
    if (c >= ncol || level >= a.nlev) continue;
    const float z = L.z[a.lev0 + level];
    const int m = c0 + c;
    const float kx = float(m) * a.kxs;
    float2 v[NF][E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int p = lane + 32 * k;
      int n;
      bool live = true;
      if (p < nyh) n = p;
      else if (p > a.Nyr - nyh) n = p - a.Nyr;
      else { n = 0; live = false; }
      float2 Ap = make_float2(0.f, 0.f), At = make_float2(0.f, 0.f);
      if (live) {
        const int r = n >= 0 ? n : a.ny + n;
        Ap = sm[r * ld + c];
        At = sm[(a.ny + r) * ld + c];
        if (a.spline) {
          const float pf = spline_prefilter(m, a.Nxr, n, a.Nyr);
          Ap = make_float2(pf * Ap.x, pf * Ap.y);
          At = make_float2(pf * At.x, pf * At.y);
        }
      }
      const float ky = float(n) * a.kys;
      const float kk = sqrtf(kx * kx + ky * ky);
      float F, S;
      depth_factors(kk, z, a.depth, F, S);
#pragma unroll
      for (int f = 0; f < NF; ++f) v[f][k] = modal_field(g * NF + f, kx, ky, kk, F, S, Ap, At);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      warp_fft<E>(v[f], T, lane);
      float2* out = a.G + ((size_t(level) * 4 + g * NF + f) * a.Mh + m) * a.Nyr +
                    E * int(bitrev(unsigned(lane), 5));
#pragma unroll
      for (int m2 = 0; m2 < E; m2 += 2) {
        if (E == 1) {
          out[0] = v[f][0];
        } else {
          __stcg(reinterpret_cast<float4*>(out + m2),
                 make_float4(v[f][m2].x, v[f][m2].y, v[f][m2 + 1].x, v[f][m2 + 1].y));
        }
      }
    }
  }
}

struct RowArgs {
  const float2* G;       // [nlev][4][Mh][Nyr]
  float4* nodes;         // [nz][Nyr][Nxr] of this time level
  const float2* tw;
  int Mh, Nxr, Nyr, rb, lev0;
  int ldG;               // m stride of the transposed intermediate (k_row_t)
  int polls;             // k_row_tma: polls of a bounded wait before it gives up
  int selftest;          // k_row_tma: 1 = issue no copy, so every wait runs out (self-test)
};

template <int E>
__global__ void __launch_bounds__(256, 2) k_row_fft(RowArgs a) {
  extern __shared__ float2 sm[];                 // [4][Mh][rb + 1]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y0 = blockIdx.x * kRowBlock;
  const int level = blockIdx.y;
  const int ld = kRowBlock + 1;
  const float2* G = a.G + size_t(level) * 4 * a.Mh * a.Nyr;
  for (int i = threadIdx.x; i < 4 * a.Mh * kRowBlock; i += blockDim.x) {
    const int rr = i % kRowBlock, qm = i / kRowBlock;
    const int y = y0 + rr;
    cp_async8(&sm[qm * ld + rr], &G[size_t(qm) * a.Nyr + (y < a.Nyr ? y : 0)], y < a.Nyr ? 8 : 0);
  }
  WarpFftTw<E> T;
  warp_fft_init<E>(T, a.tw, lane);
  cp_async_wait_all();
  __syncthreads();
  for (int rr = warp; rr < kRowBlock; rr += blockDim.x >> 5) {
    const int y = y0 + rr;
    if (y >= a.Nyr) break;
    float2 z1[E], z2[E];
    const size_t fs = size_t(a.Mh) * ld;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int p = lane + 32 * k;
      int m = -1;
      bool mirror = false;
      if (p < a.Mh) m = p;
      else if (p > a.Nxr - a.Mh) { m = a.Nxr - p; mirror = true; }
      float2 U = make_float2(0.f, 0.f), V = U, W = U, Tt = U;
      if (m >= 0) {
        const size_t o = size_t(m) * ld + rr;
        U = sm[o];
        V = sm[o + fs];
        W = sm[o + 2 * fs];
        Tt = sm[o + 3 * fs];
      }
      // Hermitian packing of two real fields into one complex spectrum (p + i q)
      if (p == 0) {
        z1[k] = make_float2(U.x, V.x);
        z2[k] = make_float2(W.x, Tt.x);
      } else if (!mirror) {
        z1[k] = make_float2(U.x - V.y, U.y + V.x);
        z2[k] = make_float2(W.x - Tt.y, W.y + Tt.x);
      } else {
        z1[k] = make_float2(U.x + V.y, V.x - U.y);
        z2[k] = make_float2(W.x + Tt.y, Tt.x - W.y);
      }
    }
    warp_fft<E>(z1, T, lane);
    warp_fft<E>(z2, T, lane);
    float4* out = a.nodes + (size_t(a.lev0 + level) * a.Nyr + y) * a.Nxr + E * int(bitrev(unsigned(lane), 5));
#pragma unroll
    for (int m2 = 0; m2 < E; ++m2)
      __stcs(&out[m2], make_float4(z1[m2].x, z1[m2].y, z2[m2].x, z2[m2].y));
  }
}

// Stockham per-warp variants of the two transform kernels (N = transform length >= 256): same
// inputs, outputs and layouts as k_col_fft / k_row_fft, with stk_fft (radix-8 register passes,
// exchanges through a warp-private shared buffer) in place of the shuffle-based transform.
template <int N, int NF>
__global__ void __launch_bounds__(256, N >= 1024 ? 1 : 2) k_col_stk(ColArgs a, Levels L) {
  extern __shared__ float2 sm[];                 // [2][ny][cb + 1] modes, then per-warp buffers
  constexpr int E = N / 32, RL = stk_radix(N, stk_npass(N) - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * kColBlock;
  const int ncol = min(kColBlock, a.Mh - c0);
  const int ld = kColBlock + 1;
  float2* wbuf = sm + 2 * a.ny * ld + warp * stk_buf(N);
  for (int i = threadIdx.x; i < a.ny * kColBlock; i += blockDim.x) {
    const int c = i % kColBlock, r = i / kColBlock;
    const bool ok = c < ncol;
    const size_t gi = ok ? size_t(r) * a.nxh1 + c0 + c : 0;
    cp_async8(&sm[r * ld + c], &a.A_phi[gi], ok ? 8 : 0);
    cp_async8(&sm[(a.ny + r) * ld + c], &a.A_phit[gi], ok ? 8 : 0);
  }
  float2 T[stk_twn(N)];
  stk_init<N>(T, a.tw, lane);
  cp_async_wait_all();
  __syncthreads();
  const int nyh = a.ny >> 1;
  const int groups = 4 / NF;
  const int ntask = a.lpc * kColBlock * groups;
  for (int task = warp; task < ntask; task += blockDim.x >> 5) {
    const int g = task % groups;
    const int rest = task / groups;
    const int c = rest % kColBlock;
    const int level = blockIdx.y * a.lpc + rest / kColBlock;
    if (c >= ncol || level >= a.nlev) continue;
    const float z = L.z[a.lev0 + level];
    const int m = c0 + c;
    const float kx = float(m) * a.kxs;
    float2 v[NF][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
      int n;
      bool live = true;
      if (p < nyh) n = p;
      else if (p > N - nyh) n = p - N;
      else { n = 0; live = false; }
      float2 Ap = make_float2(0.f, 0.f), At = make_float2(0.f, 0.f);
      if (live) {
        const int r = n >= 0 ? n : a.ny + n;
        Ap = sm[r * ld + c];
        At = sm[(a.ny + r) * ld + c];
        if (a.spline) {
          const float pf = spline_prefilter(m, a.Nxr, n, a.Nyr);
          Ap = make_float2(pf * Ap.x, pf * Ap.y);
          At = make_float2(pf * At.x, pf * At.y);
        }
      }
      const float ky = float(n) * a.kys;
      const float kk = sqrtf(kx * kx + ky * ky);
      float F, S;
      depth_factors(kk, z, a.depth, F, S);
#pragma unroll
      for (int f = 0; f < NF; ++f) v[f][e] = modal_field(g * NF + f, kx, ky, kk, F, S, Ap, At);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      stk_fft<N>(v[f], T, a.tw, wbuf, lane);
      float2* out = a.G + ((size_t(level) * 4 + g * NF + f) * a.Mh + m) * a.Nyr;
#pragma unroll
      for (int e = 0; e < E; ++e) __stcg(&out[lane + 32 * (e / RL) + (e % RL) * (N / RL)], v[f][e]);
    }
  }
}

// Hermitian packing of two real-output half spectra A, B (one column of the staged rows, stride
// ld) into z = A + i B over the full length-N spectrum, in the first-pass register layout of
// stk_fft; the upper half holds conj(A) + i conj(B) mirrored, the Nyquist slot stays zero.
template <int N>
__device__ __forceinline__ void row_pack(float2 (&z)[N / 32], const float2* A, const float2* B, int ld,
                                         int Mh, int lane) {
#pragma unroll
  for (int e = 0; e < N / 32; ++e) {
    const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
    const bool lo = p < Mh, hi = p > N - Mh;
    float2 a = make_float2(0.f, 0.f), b = a;
    if (lo || hi) {
      const int o = (lo ? p : N - p) * ld;
      a = A[o];
      b = B[o];
    }
    if (p == 0) z[e] = make_float2(a.x, b.x);
    else if (!hi) z[e] = make_float2(a.x - b.y, a.y + b.x);
    else z[e] = make_float2(a.x + b.y, b.x - a.y);
  }
}

template <int N>
__global__ void __launch_bounds__(256, N >= 1024 ? 1 : 2) k_row_stk(RowArgs a) {
  extern __shared__ float2 sm[];                 // [4][Mh][rb + 1] staging, then warp buffers
  constexpr int E = N / 32, RL = stk_radix(N, stk_npass(N) - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y0 = blockIdx.x * kRowBlock;
  const int level = blockIdx.y;
  const int ld = kRowBlock + 1;
  const float2* G = a.G + size_t(level) * 4 * a.Mh * a.Nyr;
  float2* wbuf = sm + 4 * a.Mh * ld + warp * stk_buf(N);
  for (int i = threadIdx.x; i < 4 * a.Mh * kRowBlock; i += blockDim.x) {
    const int rr = i % kRowBlock, qm = i / kRowBlock;
    const int y = y0 + rr;
    cp_async8(&sm[qm * ld + rr], &G[size_t(qm) * a.Nyr + (y < a.Nyr ? y : 0)], y < a.Nyr ? 8 : 0);
  }
  float2 T[stk_twn(N)];
  stk_init<N>(T, a.tw, lane);
  cp_async_wait_all();
  __syncthreads();
  const size_t fs = size_t(a.Mh) * ld;
  for (int rr = warp; rr < kRowBlock; rr += blockDim.x >> 5) {
    const int y = y0 + rr;
    if (y >= a.Nyr) break;
    float4* out = a.nodes + (size_t(a.lev0 + level) * a.Nyr + y) * N;
    if constexpr (N <= 256) {
      float2 z1[E], z2[E];
      row_pack<N>(z1, sm + rr, sm + fs + rr, ld, a.Mh, lane);
      row_pack<N>(z2, sm + 2 * fs + rr, sm + 3 * fs + rr, ld, a.Mh, lane);
      stk_fft<N>(z1, T, a.tw, wbuf, lane);
      stk_fft<N>(z2, T, a.tw, wbuf, lane);
#pragma unroll
      for (int e = 0; e < E; ++e)
        __stcs(&out[lane + 32 * (e / RL) + (e % RL) * (N / RL)],
               make_float4(z1[e].x, z1[e].y, z2[e].x, z2[e].y));
    } else {
      // one transform at a time (register budget): each half of a node's float4 is written by
      // its own pass; the two halves meet in L2 before the sector goes to DRAM
      float2* o2 = reinterpret_cast<float2*>(out);
#pragma unroll 1
      for (int q = 0; q < 2; ++q) {
        float2 z[E];
        row_pack<N>(z, sm + 2 * q * fs + rr, sm + (2 * q + 1) * fs + rr, ld, a.Mh, lane);
        stk_fft<N>(z, T, a.tw, wbuf, lane);
#pragma unroll
        for (int e = 0; e < E; ++e)
          __stcs(&o2[2 * (lane + 32 * (e / RL) + (e % RL) * (N / RL)) + q], z[e]);
      }
    }
  }
}

// Row pass, one field pair per CTA (blockIdx.z: 0 -> (U, V) into (u, v), 1 -> (W, T) into
// (w, dphi/dt)), one length-N transform per warp: half the registers of k_row_stk, so three CTAs
// fit on an SM. The staged rows are dead once every warp holds its row, and the same shared
// memory then serves as the per-warp exchange buffers. Each CTA writes one float2 half of the
// nodes' float4; the two halves meet in L2.
template <int N>
__global__ void __launch_bounds__(256, N >= 1024 ? 2 : 3) k_row_half(RowArgs a) {
  extern __shared__ float2 sm[];                 // [2][Mh][rb + 1] staging, then warp buffers
  constexpr int E = N / 32, RL = stk_radix(N, stk_npass(N) - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y0 = blockIdx.x * kRowBlock;
  const int level = blockIdx.y;
  const int q = blockIdx.z;
  constexpr int ld = kRowBlock + 1;
  const float2* G = a.G + (size_t(level) * 4 + 2 * q) * a.Mh * a.Nyr;
  for (int i = threadIdx.x; i < 2 * a.Mh * kRowBlock; i += blockDim.x) {
    const int rr = i % kRowBlock, fm = i / kRowBlock;
    const int y = y0 + rr;
    cp_async8(&sm[fm * ld + rr], &G[size_t(fm) * a.Nyr + (y < a.Nyr ? y : 0)], y < a.Nyr ? 8 : 0);
  }
  float2 T[stk_twn(N)];
  stk_init<N>(T, a.tw, lane);
  cp_async_wait_all();
  __syncthreads();
  const size_t fs = size_t(a.Mh) * ld;
  float2 z[E];
  row_pack<N>(z, sm + warp, sm + fs + warp, ld, a.Mh, lane);   // kRowBlock rows, one per warp
  __syncthreads();
  const int y = y0 + warp;
  if (y >= a.Nyr) return;
  stk_fft<N>(z, T, a.tw, sm + warp * stk_buf(N), lane);
  float2* o2 = reinterpret_cast<float2*>(a.nodes + (size_t(a.lev0 + level) * a.Nyr + y) * N) + q;
#pragma unroll
  for (int e = 0; e < E; ++e) __stcs(&o2[2 * (lane + 32 * (e / RL) + (e % RL) * (N / RL))], z[e]);
}

// m stride of the transposed intermediate: a whole number of 128-byte lines per field row, so
// the row pass can drop the rows it has consumed from L2 without touching a neighbour's data.
__host__ __device__ __forceinline__ int trans_ld(int Mh) { return (Mh + 15) & ~15; }

// Invalidate, without write-back, the L2 lines of nf field rows (stride fs float2) of ld float2
// each starting at row (128-byte aligned): their values are dead once the row pass has read
// them, so the column pass's writes need not reach DRAM. Lines spread over nt threads from t.
__device__ __forceinline__ void discard_rows(const float2* row, size_t fs, int nf, int ld, int t, int nt) {
  const int lines = ld / 16;
  for (int i = t; i < nf * lines; i += nt) {
    const float2* a = row + size_t(i / lines) * fs + size_t(i % lines) * 16;
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
  }
}

// Transposed-intermediate pair for 256- to 1024-point transforms. The column pass writes
// G[level][field][y][m] with the m stride padded to whole 128-byte lines (ldG), so a grid row's
// inputs are contiguous; the row pass then reads them straight into registers with coalesced
// loads, with no staging and no block-wide barrier.
//
// Column pass: the eight warps of a block own eight consecutive kx columns; each loads its
// column's modes once (reused over the block's levels), forms NF modal fields per depth-factor
// evaluation, transforms them, and the block writes the eight columns out row by row through a
// padded shared tile (64-byte segments).
// Position of (row, column) in the 8-column tiles through which the column passes transpose
// their output: a row's columns are XOR-swizzled by (row >> 1) & 7, so that a warp's column
// writes (16 consecutive rows a half-warp) and the row reads (two rows of 8 columns a
// half-warp) each hit 32 different banks.
static_assert(kColBlock == 8, "the tile swizzle spans 8 columns");
__device__ __forceinline__ int tile_pos(int row, int col) { return row * kColBlock + (col ^ ((row >> 1) & 7)); }

template <int N, int NF>
__global__ void __launch_bounds__(256, N >= 1024 ? 1 : 2) k_col_t(ColArgs a, Levels L) {
  extern __shared__ float2 sm[];                 // tile [N][kColBlock + 1], then warp buffers
  constexpr int E = N / 32, RL = stk_radix(N, stk_npass(N) - 1);
  constexpr int TLD = kColBlock + 1;
  static_assert(kColBlock * 32 == kThreads, "one column per warp");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * kColBlock;
  const int m = c0 + warp;
  const bool colok = m < a.Mh;
  float2* tile = sm;
  float2* wbuf = sm + N * TLD + warp * stk_buf(N);
  // depth factors of the current level, F and |k| S per element, made by the first field group
  // and reused by the second (short columns only; after the warp buffers)
  float* fks = reinterpret_cast<float*>(sm + N * TLD + (kThreads / 32) * stk_buf(N)) + warp * 2 * N;
  float2 T[stk_twn(N)];
  stk_init<N>(T, a.tw, lane);
  const int nyh = a.ny >> 1;
  const float kx = colok ? float(m) * a.kxs : 0.f;
  // modes of element e (zero in the padding and at the Nyquist row)
  auto load_mode = [&](int e, float2& ap, float2& at) {
    const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
    int n = 0;
    bool live = colok;
    if (p < nyh) n = p;
    else if (p > N - nyh) n = p - N;
    else live = false;
    ap = at = make_float2(0.f, 0.f);
    if (live) {
      const size_t gi = size_t(n >= 0 ? n : a.ny + n) * a.nxh1 + m;
      ap = __ldg(&a.A_phi[gi]);
      at = __ldg(&a.A_phit[gi]);
      if (a.spline) {
        const float pf = spline_prefilter(m, a.Nxr, n, a.Nyr);
        ap = make_float2(pf * ap.x, pf * ap.y);
        at = make_float2(pf * at.x, pf * at.y);
      }
    }
  };
  // short columns keep their modes in registers across levels; longer ones reload (L1)
  constexpr bool KEEP = N <= 256;
  float2 Ap[KEEP ? E : 1], At[KEEP ? E : 1];
  if constexpr (KEEP) {
#pragma unroll
    for (int e = 0; e < E; ++e) load_mode(e, Ap[e], At[e]);
  }
  for (int li = 0; li < a.lpc; ++li) {
    const int level = blockIdx.y * a.lpc + li;
    if (level >= a.nlev) break;                  // uniform over the block
    const float z = L.z[a.lev0 + level];
#pragma unroll 1
    for (int g = 0; g < 4 / NF; ++g) {
      float2 v[NF][E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
        // zero-padded and Nyquist positions carry no mode: evaluate their (unused) depth factor
        // at ky = 0, where it cannot overflow (e^{|k| z} at a padded |k| can reach inf, and
        // inf * 0 would be NaN)
        const int n = p < nyh ? p : (p > N - nyh ? p - N : 0);
        const float ky = float(n) * a.kys;
        float kk, F, S;
        float2 ap, at;
        if constexpr (KEEP) {
          ap = Ap[e];
          at = At[e];
          if (g == 0) {
            kk = sqrtf(kx * kx + ky * ky);
            depth_factors(kk, z, a.depth, F, S);
            S *= kk;                               // modal_field takes |k| S as one factor
            fks[e * 32 + lane] = F;
            fks[N + e * 32 + lane] = S;
          } else {
            F = fks[e * 32 + lane];
            S = fks[N + e * 32 + lane];
          }
          kk = 1.f;
        } else {
          kk = sqrtf(kx * kx + ky * ky);
          depth_factors(kk, z, a.depth, F, S);
          load_mode(e, ap, at);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f][e] = modal_field(g * NF + f, kx, ky, kk, F, S, ap, at);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        stk_fft<N>(v[f], T, a.tw, wbuf, lane);
#pragma unroll
        for (int e = 0; e < E; ++e) tile[tile_pos(lane + 32 * (e / RL) + (e % RL) * (N / RL), warp)] = v[f][e];
        __syncthreads();
        float2* out = a.G + (size_t(level) * 4 + g * NF + f) * a.Nyr * a.ldG + c0;
        // rows of 8 columns: 64 contiguous bytes of the intermediate per row
        for (int i = threadIdx.x; i < N * kColBlock; i += kThreads) {
          const int y = i / kColBlock, w = i % kColBlock;
          if (c0 + w < a.Mh) __stcg(&out[size_t(y) * a.ldG + w], tile[tile_pos(y, w)]);
        }
        __syncthreads();
      }
    }
  }
}

// Column pass of the transposed pair with the four modal fields in separate CTAs (blockIdx.z =
// field U, V, W, T): four times the CTAs of k_col_t per level and half its registers, so long
// columns fill the GPU even when a level chunk holds few levels (a 1024-point column pass has
// only Mh / 8 CTAs per level otherwise). The output tile and the warps' exchange buffers share
// the same shared memory (a barrier between the transforms and the tile writes).
template <int N>
__global__ void __launch_bounds__(256, N >= 1024 ? 1 : 2) k_col_tf(ColArgs a, Levels L) {
  extern __shared__ float2 sm[];                 // exchange buffers, then tile [N][kColBlock + 1]
  constexpr int E = N / 32, RL = stk_radix(N, stk_npass(N) - 1);
  static_assert(kColBlock * 32 == kThreads, "one column per warp");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * kColBlock;
  const int m = c0 + warp;
  const bool colok = m < a.Mh;
  const int q = blockIdx.z;
  float2* tile = sm;
  float2* wbuf = sm + warp * stk_buf(N);
  float2 T[stk_twn(N)];
  stk_init<N>(T, a.tw, lane);
  const int nyh = a.ny >> 1;
  const float kx = colok ? float(m) * a.kxs : 0.f;
  const float2* __restrict__ A = q == 3 ? a.A_phit : a.A_phi;
  // the column's modes of this field, loaded once and kept in registers over the CTA's levels
  // (zero in the padding and at the Nyquist row)
  float2 am[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
    int n = 0;
    bool live = colok;
    if (p < nyh) n = p;
    else if (p > N - nyh) n = p - N;
    else live = false;
    am[e] = make_float2(0.f, 0.f);
    if (live) {
      am[e] = __ldg(&A[size_t(n >= 0 ? n : a.ny + n) * a.nxh1 + m]);
      if (a.spline) {
        const float pf = spline_prefilter(m, a.Nxr, n, a.Nyr);
        am[e] = make_float2(pf * am[e].x, pf * am[e].y);
      }
    }
  }
  for (int li = 0; li < a.lpc; ++li) {
    const int level = blockIdx.y * a.lpc + li;
    if (level >= a.nlev) break;                  // uniform over the block
    const float z = L.z[a.lev0 + level];
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
      // zero-padded and Nyquist positions carry no mode: their (unused) depth factor is taken
      // at ky = 0, where it cannot overflow
      const int n = p < nyh ? p : (p > N - nyh ? p - N : 0);
      const float ky = float(n) * a.kys;
      const float kk = sqrtf(kx * kx + ky * ky);
      float F, S;
      depth_factors(kk, z, a.depth, F, S);
      v[e] = modal_field(q, kx, ky, kk, F, S, am[e], am[e]);
    }
    stk_fft<N>(v, T, a.tw, wbuf, lane);
    __syncthreads();                             // every warp is done with its exchange buffer
#pragma unroll
    for (int e = 0; e < E; ++e) tile[tile_pos(lane + 32 * (e / RL) + (e % RL) * (N / RL), warp)] = v[e];
    __syncthreads();
    float2* out = a.G + (size_t(level) * 4 + q) * a.Nyr * a.ldG + c0;
    // rows of 8 columns: 64 contiguous bytes of the intermediate per row
    for (int i = threadIdx.x; i < N * kColBlock; i += kThreads) {
      const int y = i / kColBlock, w = i % kColBlock;
      if (c0 + w < a.Mh) __stcg(&out[size_t(y) * a.ldG + w], tile[tile_pos(y, w)]);
    }
    __syncthreads();                             // the tile is read before the next transforms
  }
}

// The same column pass with two warps per column (1024-point columns): warp 2c + s transforms
// the rows p = 2 i + s of column c (a 512-point Stockham transform, 16 points a lane), the odd
// warp multiplies its result by e^{2 pi i k / N}, both halves go to the CTA's tile, and the
// radix-2 combine X[k] = E[k] + O'[k], X[k + N/2] = E[k] - O'[k] is done while the tile is
// written out (the operations of the one-warp transform's last pass, in the same order, so the
// results are identical). Half the points per lane (128 registers) and twice the warps per SM of
// k_col_tf<1024>, whose 244 registers leave one 8-warp CTA per SM; bank-conflict-free tile
// (XOR swizzle) and no separate exchange for the combine: stage 1 of the large sea 17.65 ->
// 16.67 ms.
template <int N>
__global__ void __launch_bounds__(2 * kThreads, 1) k_col_tf2(ColArgs a, Levels L) {
  extern __shared__ float2 sm[];                 // exchange buffers, then tile [N][kColBlock] (swizzled)
  constexpr int H = N / 2, E = H / 32, RL = stk_radix(H, stk_npass(H) - 1);
  static_assert(kColBlock == 8, "the tile swizzle spans 8 columns");
  static_assert(kColBlock * 64 == 2 * kThreads, "two warps per column");
  // e^{2 pi i k / N}, k < H: the factors of the N-point transform's last pass (radix 2, stride H),
  // read from its pass-major table (consecutive k in consecutive entries)
  static_assert(stk_radix(N, stk_npass(N) - 1) == 2 && stk_ns(N, stk_npass(N) - 1) == H,
                "the combine is the last radix-2 pass of the N-point transform");
  constexpr int kTwC = stk_twp(N, stk_npass(N) - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = warp >> 1, par = warp & 1;     // column of the CTA, parity of this warp's rows
  const int c0 = blockIdx.x * kColBlock;
  const int m = c0 + col;
  const bool colok = m < a.Mh;
  const int q = blockIdx.z;
  float2* tile = sm;
  float2* wbuf = sm + warp * stk_buf(H);
  float2 T[stk_twn(H)];
  stk_init<H>(T, a.tw, lane);
  const int nyh = a.ny >> 1;
  const float kx = colok ? float(m) * a.kxs : 0.f;
  const float2* __restrict__ A = q == 3 ? a.A_phit : a.A_phi;
  // this warp's modes (rows p = 2 i + par of the half-sequence position i), loaded once and kept
  // in registers over the CTA's levels (zero in the padding and at the Nyquist row)
  float2 am[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = 2 * (lane + 32 * (e / 8) + (e % 8) * (H / 8)) + par;
    int n = 0;
    bool live = colok;
    if (p < nyh) n = p;
    else if (p > N - nyh) n = p - N;
    else live = false;
    am[e] = make_float2(0.f, 0.f);
    if (live) {
      am[e] = __ldg(&A[size_t(n >= 0 ? n : a.ny + n) * a.nxh1 + m]);
      if (a.spline) {
        const float pf = spline_prefilter(m, a.Nxr, n, a.Nyr);
        am[e] = make_float2(pf * am[e].x, pf * am[e].y);
      }
    }
  }
  for (int li = 0; li < a.lpc; ++li) {
    const int level = blockIdx.y * a.lpc + li;
    if (level >= a.nlev) break;                  // uniform over the block
    const float z = L.z[a.lev0 + level];
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = 2 * (lane + 32 * (e / 8) + (e % 8) * (H / 8)) + par;
      // zero-padded and Nyquist positions carry no mode: their (unused) depth factor is taken
      // at ky = 0, where it cannot overflow
      const int n = p < nyh ? p : (p > N - nyh ? p - N : 0);
      const float ky = float(n) * a.kys;
      const float kk = sqrtf(kx * kx + ky * ky);
      float F, S;
      depth_factors(kk, z, a.depth, F, S);
      v[e] = modal_field(q, kx, ky, kk, F, S, am[e], am[e]);
    }
    stk_fft<H>(v, T, a.tw, wbuf, lane);
    __syncthreads();                             // every warp is done with its exchange buffer
    // element e holds output k = lane + 32 (e / RL) + (e % RL) (H / RL) of this half; the odd half,
    // twiddled, goes to tile row H + k. Tile rows hold the CTA's 8 columns with column c at
    // c ^ ((row >> 1) & 7): the column writes (16 consecutive rows a half-warp) and the row reads
    // (two rows of 8 columns a half-warp) both hit 32 different banks.
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * (e / RL) + (e % RL) * (H / RL);
      if (par) v[e] = cmul(v[e], __ldg(&a.tw[kTwC + k]));
      const int row = k + par * H;
      tile[tile_pos(row, col)] = v[e];
    }
    __syncthreads();
    float2* out = a.G + (size_t(level) * 4 + q) * a.Nyr * a.ldG + c0;
    // the radix-2 combine on the way out: X[y] = E[y] + O'[y], X[y + H] = E[y] - O'[y]
    for (int i = threadIdx.x; i < H * kColBlock; i += 2 * kThreads) {
      const int y = i / kColBlock, w = i % kColBlock;
      const float2 ev = tile[tile_pos(y, w)], od = tile[tile_pos(y + H, w)];
      if (c0 + w < a.Mh) {
        __stcg(&out[size_t(y) * a.ldG + w], cadd(ev, od));
        __stcg(&out[size_t(y + H) * a.ldG + w], csub(ev, od));
      }
    }
    __syncthreads();                             // the tile is read before the next transforms
  }
}

// Row pass over the transposed intermediate: one warp per grid row of one level, its four
// modal fields loaded straight from G (consecutive lanes read consecutive m), packed as
// Z1 = U + iV and Z2 = W + iT over the full x spectrum, transformed, stored as float4.
template <int N>
__global__ void __launch_bounds__(256, N >= 1024 ? 1 : 2) k_row_t(RowArgs a) {
  extern __shared__ float2 sm[];                 // warp exchange buffers
  constexpr int E = N / 32, RL = stk_radix(N, stk_npass(N) - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y = blockIdx.x * (kThreads / 32) + warp;
  const int level = blockIdx.y;
  if (y >= a.Nyr) return;                        // no block-wide barrier in this kernel
  float2 T[stk_twn(N)];
  stk_init<N>(T, a.tw, lane);
  float2* wbuf = sm + warp * stk_buf(N);
  const size_t fs = size_t(a.Nyr) * a.ldG;
  const float2* row = a.G + size_t(level) * 4 * fs + size_t(y) * a.ldG;
  float4* out = a.nodes + (size_t(a.lev0 + level) * a.Nyr + y) * N;
  float2 z1[E], z2[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
    const bool lo = p < a.Mh, hi = p > N - a.Mh;
    float2 U = make_float2(0.f, 0.f), V = U, W = U, Tt = U;
    if (lo || hi) {
      const int mm = lo ? p : N - p;
      U = __ldcg(&row[mm]);
      V = __ldcg(&row[fs + mm]);
      W = __ldcg(&row[2 * fs + mm]);
      Tt = __ldcg(&row[3 * fs + mm]);
    }
    if (p == 0) {
      z1[e] = make_float2(U.x, V.x);
      z2[e] = make_float2(W.x, Tt.x);
    } else if (!hi) {
      z1[e] = make_float2(U.x - V.y, U.y + V.x);
      z2[e] = make_float2(W.x - Tt.y, W.y + Tt.x);
    } else {
      z1[e] = make_float2(U.x + V.y, V.x - U.y);
      z2[e] = make_float2(W.x + Tt.y, Tt.x - W.y);
    }
  }
  stk_fft<N>(z1, T, a.tw, wbuf, lane);
  stk_fft<N>(z2, T, a.tw, wbuf, lane);
#pragma unroll
  for (int e = 0; e < E; ++e)
    __stcs(&out[lane + 32 * (e / RL) + (e % RL) * (N / RL)], make_float4(z1[e].x, z1[e].y, z2[e].x, z2[e].y));
  __syncwarp();                                  // every lane's reads of the row are done
  discard_rows(row, fs, 4, a.ldG, lane, 32);
}

// Same row pass with one transform per warp (warps 2r and 2r+1 of a block take Z1 and Z2 of
// row r): half the registers, so more warps per SM; each warp writes one float2 half of the
// nodes' float4 (the halves meet in L2).
template <int N>
__global__ void __launch_bounds__(256, N >= 2048 ? 1 : (N >= 1024 ? 2 : 3)) k_row_t2(RowArgs a) {
  extern __shared__ float2 sm[];                 // warp exchange buffers
  constexpr int E = N / 32, RL = stk_radix(N, stk_npass(N) - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y = blockIdx.x * (kThreads / 64) + (warp >> 1);
  const int q = warp & 1;                        // 0: Z1 = U + iV, 1: Z2 = W + iT
  const int level = blockIdx.y;
  if (y >= a.Nyr) return;                        // no block-wide barrier in this kernel
  float2 T[stk_twn(N)];
  stk_init<N>(T, a.tw, lane);
  float2* wbuf = sm + warp * stk_buf(N);
  const size_t fs = size_t(a.Nyr) * a.ldG;
  const float2* row = a.G + (size_t(level) * 4 + 2 * q) * fs + size_t(y) * a.ldG;
  float2 z[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
    const bool lo = p < a.Mh, hi = p > N - a.Mh;
    float2 A = make_float2(0.f, 0.f), B = A;
    if (lo || hi) {
      const int mm = lo ? p : N - p;
      A = __ldcg(&row[mm]);
      B = __ldcg(&row[fs + mm]);
    }
    if (p == 0) z[e] = make_float2(A.x, B.x);
    else if (!hi) z[e] = make_float2(A.x - B.y, A.y + B.x);
    else z[e] = make_float2(A.x + B.y, B.x - A.y);
  }
  stk_fft<N>(z, T, a.tw, wbuf, lane);
  float2* out = reinterpret_cast<float2*>(a.nodes + (size_t(a.lev0 + level) * a.Nyr + y) * N) + q;
#pragma unroll
  for (int e = 0; e < E; ++e) __stcs(&out[2 * (lane + 32 * (e / RL) + (e % RL) * (N / RL))], z[e]);
  __syncwarp();                                  // every lane's reads of the two rows are done
  discard_rows(row, fs, 2, a.ldG, lane, 32);
}

// Row pass for rows longer than a warp transform (2048..8192 points): one block of kThreads per
// grid row of one level, inputs from the transposed intermediate (coalesced), block-wide
// Stockham transforms of Z1 = U + iV and Z2 = W + iT. 2048-point rows: three blocks per SM (80
// registers) hide more of the intermediate's load latency than two (92): stage 1 of the large
// sea 16.64 -> 16.12 ms.
template <int N>
__global__ void __launch_bounds__(256, N >= 8192 ? 1 : (N >= 4096 ? 2 : 3)) k_row_tb(RowArgs a) {
  extern __shared__ float2 sm[];                 // one or two exchange buffers
  constexpr int E = N / kThreads, RL = stk_radix(N, stk_npass(N) - 1);
  constexpr bool BOTH = N <= 4096;               // both transforms' data in registers at once
  const int t = threadIdx.x;
  const int y = blockIdx.x;
  const int level = blockIdx.y;
  const size_t fs = size_t(a.Nyr) * a.ldG;
  const float2* row = a.G + size_t(level) * 4 * fs + size_t(y) * a.ldG;
  float4* out = a.nodes + (size_t(a.lev0 + level) * a.Nyr + y) * N;
  auto pack = [&](float2 (&z)[E], int q) {       // q = 0: U + iV, 1: W + iT
    const float2* A = row + 2 * q * fs;
    const float2* B = A + fs;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = t + kThreads * (e / 8) + (e % 8) * (N / 8);
      const bool lo = p < a.Mh, hi = p > N - a.Mh;
      float2 u = make_float2(0.f, 0.f), v = u;
      if (lo || hi) {
        const int mm = lo ? p : N - p;
        u = __ldcg(&A[mm]);
        v = __ldcg(&B[mm]);
      }
      if (p == 0) z[e] = make_float2(u.x, v.x);
      else if (!hi) z[e] = make_float2(u.x - v.y, u.y + v.x);
      else z[e] = make_float2(u.x + v.y, v.x - u.y);
    }
  };
  if constexpr (BOTH) {
    float2 z1[E], z2[E];
    pack(z1, 0);
    pack(z2, 1);
    stkb_fft2<N, kThreads>(z1, z2, a.tw, sm, sm + stk_buf(N), t);
#pragma unroll
    for (int e = 0; e < E; ++e)
      __stcs(&out[t + kThreads * (e / RL) + (e % RL) * (N / RL)], make_float4(z1[e].x, z1[e].y, z2[e].x, z2[e].y));
    __syncthreads();                             // every thread's reads of the rows are done
    discard_rows(row, fs, 4, a.ldG, t, kThreads);
  } else {
    float2* o2 = reinterpret_cast<float2*>(out);
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
      float2 z[E];
      pack(z, q);
      stkb_fft<N, kThreads>(z, a.tw, sm, t);
#pragma unroll
      for (int e = 0; e < E; ++e) __stcs(&o2[2 * (t + kThreads * (e / RL) + (e % RL) * (N / RL)) + q], z[e]);
      __syncthreads();                           // the buffer is reused by the second transform
    }
    discard_rows(row, fs, 4, a.ldG, t, kThreads);  // after the barrier: all reads are done
  }
}

// Row pass over the transposed intermediate with its inputs staged by bulk copies: each warp
// takes `rpw` consecutive rows of one level; lane 0 copies a row's four field segments
// (ldG complex values each, contiguous in G) into the warp's staging buffer with cp.async.bulk
// on the warp's mbarrier, and the next row's copy runs while the current row is transformed.
// A wait that does not complete within its bound sets the device error flag and ends the warp:
// the warp decides together (every lane must have seen its copy complete), waits, also bounded,
// for the copy it still has in flight, and leaves as one. The host reads and clears the flag
// with swense_async_status.
__device__ int g_async_timeout;

template <int N>
__global__ void __launch_bounds__(256, N >= 1024 ? 1 : 2) k_row_tma(RowArgs a, int rpw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int E = N / 32, RL = stk_radix(N, stk_npass(N) - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned span = unsigned(a.ldG) * unsigned(sizeof(float2));      // bytes per field row
  const size_t per_warp = 4 * size_t(span) + size_t(stk_buf(N)) * sizeof(float2);
  float2* stg = reinterpret_cast<float2*>(smraw + warp * per_warp);
  float2* xbuf = reinterpret_cast<float2*>(smraw + warp * per_warp + 4 * size_t(span));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + (kThreads / 32) * per_warp) + warp;
  const int level = blockIdx.y;
  const int y0 = (blockIdx.x * (kThreads / 32) + warp) * rpw;
  const int nrows = min(rpw, a.Nyr - y0);
  if (nrows <= 0) return;                        // no block-wide barrier in this kernel
  const size_t fs = size_t(a.Nyr) * a.ldG;
  const float2* Gl = a.G + size_t(level) * 4 * fs;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncwarp();
  auto issue = [&](int i) {
    if (lane == 0) {
      fence_proxy_async();                       // earlier reads of the buffer come first
      mbar_arrive_expect_tx(bar, 4 * span);
      const float2* src = Gl + size_t(y0 + i) * a.ldG;
      if (!a.selftest) {
#pragma unroll
        for (int f = 0; f < 4; ++f) bulk_g2s(stg + f * a.ldG, src + f * fs, span, bar);
      }
    }
  };
  issue(0);
  float2 T[stk_twn(N)];
  stk_init<N>(T, a.tw, lane);
  for (int i = 0; i < nrows; ++i) {
    const bool done = mbar_wait(bar, unsigned(i) & 1u, a.polls);
    if (!__all_sync(0xffffffffu, done)) {        // one lane gave up: the whole warp leaves
      if (lane == 0) atomicExch(&g_async_timeout, 1);
      // the copy waited on is the only one in flight (none in the self-test)
      mbar_wait(bar, unsigned(i) & 1u, a.polls);
      __syncwarp();
      return;
    }
    float2 z1[E], z2[E];
    const float2* U = stg;
    const float2* V = stg + a.ldG;
    const float2* W = stg + 2 * a.ldG;
    const float2* Tt = stg + 3 * a.ldG;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = lane + 32 * (e / 8) + (e % 8) * (N / 8);
      const bool lo = p < a.Mh, hi = p > N - a.Mh;
      float2 u = make_float2(0.f, 0.f), v = u, w = u, t = u;
      if (lo || hi) {
        const int mm = lo ? p : N - p;
        u = U[mm];
        v = V[mm];
        w = W[mm];
        t = Tt[mm];
      }
      if (p == 0) {
        z1[e] = make_float2(u.x, v.x);
        z2[e] = make_float2(w.x, t.x);
      } else if (!hi) {
        z1[e] = make_float2(u.x - v.y, u.y + v.x);
        z2[e] = make_float2(w.x - t.y, w.y + t.x);
      } else {
        z1[e] = make_float2(u.x + v.y, v.x - u.y);
        z2[e] = make_float2(w.x + t.y, t.x - w.y);
      }
    }
    __syncwarp();                                // every lane has read the staged row
    // the bulk copy that filled the staging buffer has completed: its global rows are dead
    discard_rows(Gl + size_t(y0 + i) * a.ldG, fs, 4, a.ldG, lane, 32);
    if (i + 1 < nrows) issue(i + 1);
    stk_fft<N>(z1, T, a.tw, xbuf, lane);
    stk_fft<N>(z2, T, a.tw, xbuf, lane);
    float4* out = a.nodes + (size_t(a.lev0 + level) * a.Nyr + y0 + i) * N;
#pragma unroll
    for (int e = 0; e < E; ++e)
      __stcs(&out[lane + 32 * (e / RL) + (e % RL) * (N / RL)], make_float4(z1[e].x, z1[e].y, z2[e].x, z2[e].y));
  }
}

// Launch-shape choices of the warp-register path, per grid shape (set by swense_autotune_grid;
// defaults otherwise).
struct Tune {
  int lpc = -1;                         // levels per column-transform CTA of the warp path;
                                        // 0: shared-memory path; -1: default for the shape
  size_t chunk_bytes = kChunkBytes;     // scratch per level chunk (L2-resident)
  int rowv = 0;                         // row pass: 0 both field pairs per warp (k_row_stk),
                                        // 1 one field pair per CTA (k_row_half)
  int colv = 0;                         // column pass of the transposed pair: 0 k_col_t,
                                        // 1 k_col_tf (one modal field per CTA)
};
std::mutex g_tune_mutex;
std::map<std::array<int64_t, 4>, Tune> g_tune;

Tune tuned(int nx, int ny, int pad, int nz) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune.find({nx, ny, pad, nz});
  return it == g_tune.end() ? Tune{} : it->second;
}

// Validated sizes and derived constants of one swense_fields_on_grid request.
struct GridPlan {
  int nx, ny, nz, n_tl, nxh1, Mh, pad, spline;
  int64_t Nxr, Nyr;
  size_t nslot, per_level, prop_bytes, geta_bytes;
  Levels lev;
};

template <int E, int NF>
int launch_col(const ColArgs& c, const Levels& L, dim3 grid, size_t smem, cudaStream_t stream) {
  int st = set_smem((const void*)k_col_fft<E, NF>, smem);
  if (st) return st;
  k_col_fft<E, NF><<<grid, kThreads, smem, stream>>>(c, L);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N, int NF>
int launch_col_stk(const ColArgs& c, const Levels& L, dim3 grid, size_t smem, cudaStream_t stream) {
  smem += size_t(8) * stk_buf(N) * sizeof(float2);
  int st = set_smem((const void*)k_col_stk<N, NF>, smem);
  if (st) return st;
  k_col_stk<N, NF><<<grid, kThreads, smem, stream>>>(c, L);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N>
int launch_row_stk(const RowArgs& r, dim3 grid, size_t smem, cudaStream_t stream) {
  smem += size_t(8) * stk_buf(N) * sizeof(float2);
  int st = set_smem((const void*)k_row_stk<N>, smem);
  if (st) return st;
  k_row_stk<N><<<grid, kThreads, smem, stream>>>(r);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N, int NF>
int launch_col_t(const ColArgs& c, const Levels& L, dim3 grid, cudaStream_t stream) {
  const size_t smem = (size_t(N) * (kColBlock + 1) + size_t(8) * stk_buf(N)) * sizeof(float2) +
                      (N <= 256 ? size_t(8) * 2 * N * sizeof(float) : 0);
  int st = set_smem((const void*)k_col_t<N, NF>, smem);
  if (st) return st;
  k_col_t<N, NF><<<grid, kThreads, smem, stream>>>(c, L);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N>
int launch_col_tf(const ColArgs& c, const Levels& L, dim3 grid, cudaStream_t stream) {
  const size_t smem = std::max(size_t(N) * (kColBlock + 1), size_t(8) * stk_buf(N)) * sizeof(float2);
  int st = set_smem((const void*)k_col_tf<N>, smem);
  if (st) return st;
  grid.z = 4;
  k_col_tf<N><<<grid, kThreads, smem, stream>>>(c, L);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N>
int launch_col_tf2(const ColArgs& c, const Levels& L, dim3 grid, cudaStream_t stream) {
  const size_t smem = std::max(size_t(N) * kColBlock, size_t(16) * stk_buf(N / 2)) * sizeof(float2);
  int st = set_smem((const void*)k_col_tf2<N>, smem);
  if (st) return st;
  grid.z = 4;
  k_col_tf2<N><<<grid, 2 * kThreads, smem, stream>>>(c, L);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N>
int launch_row_t(const RowArgs& r, dim3 grid, cudaStream_t stream) {
  const size_t smem = size_t(8) * stk_buf(N) * sizeof(float2);
  int st = set_smem((const void*)k_row_t<N>, smem);
  if (st) return st;
  k_row_t<N><<<grid, kThreads, smem, stream>>>(r);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N>
int launch_row_tb(const RowArgs& r, unsigned nl, cudaStream_t stream) {
  const size_t smem = size_t(N <= 4096 ? 2 : 1) * stk_buf(N) * sizeof(float2);
  int st = set_smem((const void*)k_row_tb<N>, smem);
  if (st) return st;
  k_row_tb<N><<<dim3(unsigned(r.Nyr), nl), kThreads, smem, stream>>>(r);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

constexpr int kRowsPerWarp = 2;     // rows a warp of the staged row pass takes in turn

template <int N>
int launch_row_tma(const RowArgs& r, unsigned nl, cudaStream_t stream) {
  const size_t per_warp = 4 * size_t(r.ldG) * sizeof(float2) + size_t(stk_buf(N)) * sizeof(float2);
  const size_t smem = (kThreads / 32) * per_warp + (kThreads / 32) * sizeof(uint64_t);
  int st = set_smem((const void*)k_row_tma<N>, smem);
  if (st) return st;
  const unsigned per_block = (kThreads / 32) * kRowsPerWarp;
  k_row_tma<N><<<dim3((unsigned(r.Nyr) + per_block - 1) / per_block, nl), kThreads, smem, stream>>>(r, kRowsPerWarp);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N>
int launch_row_t2(const RowArgs& r, dim3 grid, cudaStream_t stream) {
  const size_t smem = size_t(8) * stk_buf(N) * sizeof(float2);
  int st = set_smem((const void*)k_row_t2<N>, smem);
  if (st) return st;
  k_row_t2<N><<<grid, kThreads, smem, stream>>>(r);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

// Transposed-intermediate pair (row variants 2 and 3): both transform lengths in 256..1024;
// variant 3 runs one transform per warp in the row pass.
int launch_pair_t(const ColArgs& c, const RowArgs& r, const Levels& L, int nl, cudaStream_t s,
                  bool one_per_warp, bool staged = false, int which = 0, int colv = 0) {
  const dim3 gc(unsigned((c.Mh + kColBlock - 1) / kColBlock), unsigned((nl + c.lpc - 1) / c.lpc));
  const dim3 gr(unsigned((r.Nyr + 7) / 8), unsigned(nl));
  const dim3 gr2(unsigned((r.Nyr + 3) / 4), unsigned(nl));
  int st = SWENSE_OK;
  if (which != 2 && colv == 1) {
    switch (c.Nyr) {
      case 256: st = launch_col_tf<256>(c, L, gc, s); break;
      case 512: st = launch_col_tf<512>(c, L, gc, s); break;
      case 1024: st = launch_col_tf2<1024>(c, L, gc, s); break;
      default: return fail(SWENSE_ERR_UNSUPPORTED, "transposed pair: column length");
    }
  } else if (which != 2) {
    switch (c.Nyr) {
      case 256: st = launch_col_t<256, 2>(c, L, gc, s); break;
      case 512: st = launch_col_t<512, 1>(c, L, gc, s); break;
      case 1024: st = launch_col_t<1024, 1>(c, L, gc, s); break;
      default: return fail(SWENSE_ERR_UNSUPPORTED, "transposed pair: column length");
    }
  }
  if (st || which == 1) return st;
  if (one_per_warp && r.Nxr == 2048) return launch_row_t2<2048>(r, gr2, s);   // 64 elements a lane
  switch (r.Nxr) {                               // rows longer than a warp transform
    case 2048: return launch_row_tb<2048>(r, unsigned(nl), s);
    case 4096: return launch_row_tb<4096>(r, unsigned(nl), s);
    case 8192: return launch_row_tb<8192>(r, unsigned(nl), s);
    default: break;
  }
  if (staged) {
    switch (r.Nxr) {
      case 256: return launch_row_tma<256>(r, unsigned(nl), s);
      case 512: return launch_row_tma<512>(r, unsigned(nl), s);
      case 1024: return launch_row_tma<1024>(r, unsigned(nl), s);
      default: return fail(SWENSE_ERR_UNSUPPORTED, "staged row pass: row length");
    }
  }
  if (one_per_warp) {
    switch (r.Nxr) {
      case 256: return launch_row_t2<256>(r, gr2, s);
      case 512: return launch_row_t2<512>(r, gr2, s);
      case 1024: return launch_row_t2<1024>(r, gr2, s);
      default: return fail(SWENSE_ERR_UNSUPPORTED, "transposed pair: row length");
    }
  }
  switch (r.Nxr) {
    case 256: return launch_row_t<256>(r, gr, s);
    case 512: return launch_row_t<512>(r, gr, s);
    case 1024: return launch_row_t<1024>(r, gr, s);
    default: return fail(SWENSE_ERR_UNSUPPORTED, "transposed pair: row length");
  }
}

int launch_col_e(int E, const ColArgs& c, const Levels& L, dim3 grid, size_t smem, cudaStream_t s) {
  switch (E) {
    case 1: return launch_col<1, 4>(c, L, grid, smem, s);
    case 2: return launch_col<2, 4>(c, L, grid, smem, s);
    case 4: return launch_col<4, 4>(c, L, grid, smem, s);
    case 8: return launch_col_stk<256, 2>(c, L, grid, smem, s);
    case 16: return launch_col_stk<512, 1>(c, L, grid, smem, s);
    case 32: return launch_col_stk<1024, 1>(c, L, grid, smem, s);
    default: return fail(SWENSE_ERR_UNSUPPORTED, "column transform size");
  }
}

template <int E>
int launch_row(const RowArgs& r, dim3 grid, size_t smem, cudaStream_t stream) {
  int st = set_smem((const void*)k_row_fft<E>, smem);
  if (st) return st;
  k_row_fft<E><<<grid, kThreads, smem, stream>>>(r);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

template <int N>
int launch_row_half(const RowArgs& r, dim3 grid, cudaStream_t stream) {
  static_assert(kRowBlock * 32 == kThreads, "one staged row per warp");
  const size_t smem = std::max(size_t(2) * r.Mh * (kRowBlock + 1), size_t(8) * stk_buf(N)) * sizeof(float2);
  int st = set_smem((const void*)k_row_half<N>, smem);
  if (st) return st;
  grid.z = 2;
  k_row_half<N><<<grid, kThreads, smem, stream>>>(r);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

int launch_row_e(int E, const RowArgs& r, dim3 grid, size_t smem, cudaStream_t s, int rowv = 0) {
  if (rowv == 1) {
    switch (E) {
      case 8: return launch_row_half<256>(r, grid, s);
      case 16: return launch_row_half<512>(r, grid, s);
      case 32: return launch_row_half<1024>(r, grid, s);
      default: break;                   // shorter rows: the joint kernel
    }
  }
  switch (E) {
    case 1: return launch_row<1>(r, grid, smem, s);
    case 2: return launch_row<2>(r, grid, smem, s);
    case 4: return launch_row<4>(r, grid, smem, s);
    case 8: return launch_row_stk<256>(r, grid, smem, s);
    case 16: return launch_row_stk<512>(r, grid, smem, s);
    case 32: return launch_row_stk<1024>(r, grid, smem, s);
    default: return fail(SWENSE_ERR_UNSUPPORTED, "row transform size");
  }
}

// The warp-register path covers 32 <= ny_r, nx_r <= 1024 (3-D only); the transposed pair also
// takes rows of 2048..8192 points (block-wide row transforms) over 256..1024-point columns.
bool warp_path(int ny, int64_t Nxr, int64_t Nyr) {
  return ny > 1 && Nyr >= 32 && Nyr <= 1024 && Nxr >= 32 && Nxr <= 1024;
}
bool pair_path(int ny, int64_t Nxr, int64_t Nyr) {
  return ny > 1 && Nyr >= 256 && Nyr <= 1024 && Nxr >= 256 && Nxr <= SWENSE_MAX_FFT;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int plan_grid(const swense_modes* md, int32_t n_tl, const double* t, const swense_grid_desc* desc,
              const float* nodes, const float* eta, GridPlan* p) {
  if (!md || !desc || !nodes || !eta) return fail(SWENSE_ERR_ARG, "NULL modes, desc or output");
  if (!md->A_eta || !md->A_phi || !md->A_phit) return fail(SWENSE_ERR_ARG, "NULL modal amplitudes");
  const int nx = md->nx, ny = md->ny;
  if (!is_pow2(nx) || nx < 4 || !is_pow2(ny) || (ny != 1 && ny < 4))
    return fail(SWENSE_ERR_SIZE, "nx must be a power of two >= 4, ny 1 or a power of two >= 4");
  const int pad = desc->pad_n;
  if (pad < 1 || pad > 8) return fail(SWENSE_ERR_ARG, "pad_n must lie in 1..8");
  const int64_t Nxr = int64_t(pad) * nx, Nyr = ny > 1 ? int64_t(pad) * ny : 1;
  if (Nxr > SWENSE_MAX_FFT || Nyr > SWENSE_MAX_FFT)
    return fail(SWENSE_ERR_SIZE, "pad_n*nx and pad_n*ny must not exceed SWENSE_MAX_FFT");
  if (!(md->Lx > 0) || !std::isfinite(md->Lx) || (ny > 1 && (!(md->Ly > 0) || !std::isfinite(md->Ly))))
    return fail(SWENSE_ERR_ARG, "domain lengths must be finite and positive");
  if (!std::isfinite(md->depth)) return fail(SWENSE_ERR_ARG, "depth must be finite");
  if (n_tl < 1 || n_tl > 64) return fail(SWENSE_ERR_ARG, "n_tl must be in [1, 64]");
  if (md->omega) {
    if (md->n_snap != 1) return fail(SWENSE_ERR_ARG, "with omega, n_snap must be 1");
    if (!t) return fail(SWENSE_ERR_ARG, "with omega, t[n_tl] is required");
    for (int l = 0; l < n_tl; ++l)
      if (!std::isfinite(t[l])) return fail(SWENSE_ERR_ARG, "non-finite time");
  } else if (md->n_snap != n_tl) {
    return fail(SWENSE_ERR_ARG, "without omega, n_snap must equal n_tl");
  }
  const int nz = desc->nz;
  if (nz < 4 || nz > SWENSE_MAX_LEVELS || !desc->z_levels)
    return fail(SWENSE_ERR_LEVELS, "need 4 <= nz <= SWENSE_MAX_LEVELS levels");
  for (int l = 0; l < nz; ++l) {
    p->lev.z[l] = desc->z_levels[l];
    if (!std::isfinite(p->lev.z[l]) || (l > 0 && !(p->lev.z[l] > p->lev.z[l - 1])))
      return fail(SWENSE_ERR_LEVELS, "z_levels must be finite and strictly increasing");
  }
  if ((reinterpret_cast<uintptr_t>(nodes) & 15) || (reinterpret_cast<uintptr_t>(eta) & 3))
    return fail(SWENSE_ERR_ARG, "nodes must be 16-byte aligned, eta 4-byte aligned");
  if (desc->scheme != SWENSE_LAGRANGE3 && desc->scheme != SWENSE_SPLINE3)
    return fail(SWENSE_ERR_ARG, "unknown interpolation scheme");
  p->spline = desc->scheme == SWENSE_SPLINE3;
  p->nx = nx;
  p->ny = ny;
  p->pad = pad;
  p->nz = nz;
  p->n_tl = n_tl;
  p->nxh1 = nx / 2 + 1;
  p->Mh = nx / 2;
  p->Nxr = Nxr;
  p->Nyr = Nyr;
  p->nslot = size_t(ny) * p->nxh1;
  p->per_level = size_t(4) * Nyr * trans_ld(p->Mh) * sizeof(float2);
  p->prop_bytes = md->omega ? size_t(n_tl) * 3 * p->nslot * sizeof(float2) : 0;
  p->geta_bytes = ny > 1 ? size_t(Nyr) * p->Mh * sizeof(float2) : 0;
  return SWENSE_OK;
}

// Untuned column-pass variant of the transposed pair: one modal field per CTA (k_col_tf) for
// 1024-point columns, whose k_col_t runs one CTA per SM with only Mh / 8 CTAs per level.
int default_colv(const GridPlan& p) { return pair_path(p.ny, p.Nxr, p.Nyr) && p.Nyr >= 1024 ? 1 : 0; }

// Scratch bytes for a level chunk of `chunk` levels (0 when no scratch is needed).
size_t scratch_bytes(const GridPlan& p, int chunk, int nbuf = 1) {
  const size_t g_bytes = p.ny > 1 ? size_t(chunk) * p.per_level : 0;
  return align256(p.prop_bytes) + align256(p.geta_bytes) + size_t(nbuf) * align256(g_bytes);
}

// Library-internal second stream and events (per device) for the two-stream transform
// pipeline: chunk c's row pass runs on the second stream while chunk c+1's column pass runs on
// the caller's stream, with two intermediate buffers. Created on first use; recording, waiting
// and launching on them inside a stream capture joins them to the capture (fork/join).
struct Pipe {
  cudaStream_t side = nullptr;
  cudaEvent_t col_done[2] = {nullptr, nullptr}, row_done[2] = {nullptr, nullptr};
  // the eta transform runs beside the level transforms on a stream of its own
  cudaStream_t eta_side = nullptr;
  cudaEvent_t eta_fork = nullptr, eta_join = nullptr;
};
std::mutex g_pipe_mutex;
std::map<int, Pipe> g_pipe;

int get_pipe(Pipe** out) {
  int dev = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_pipe_mutex);
  Pipe& pp = g_pipe[dev];
  if (!pp.side) {
    SWENSE_CUDA_TRY(cudaStreamCreateWithFlags(&pp.side, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      SWENSE_CUDA_TRY(cudaEventCreateWithFlags(&pp.col_done[b], cudaEventDisableTiming));
      SWENSE_CUDA_TRY(cudaEventCreateWithFlags(&pp.row_done[b], cudaEventDisableTiming));
    }
    SWENSE_CUDA_TRY(cudaStreamCreateWithFlags(&pp.eta_side, cudaStreamNonBlocking));
    SWENSE_CUDA_TRY(cudaEventCreateWithFlags(&pp.eta_fork, cudaEventDisableTiming));
    SWENSE_CUDA_TRY(cudaEventCreateWithFlags(&pp.eta_join, cudaEventDisableTiming));
  }
  *out = &pp;
  return SWENSE_OK;
}

// Enqueue every kernel of the request; `ws` holds scratch_bytes(p, chunk) bytes. eta_side: run
// the eta transform of each time level on the per-device second stream, forked after that time
// level's propagated modes exist and joined back before the call returns (graph-capturable).
int launch_grid(const GridPlan& p, const swense_modes* md, const double* t, float* nodes, float* eta,
                void* ws, int chunk, cudaStream_t stream, int lpc = kColLevels, int rowv = 0,
                int overlap = 0, int eta_side = 0, int colv = 0) {
  const float2* tw = nullptr;
  {
    int st = twiddles(stream, &tw);
    if (st) return st;
  }
  const int ny = p.ny, nz = p.nz, Mh = p.Mh, nxh1 = p.nxh1;
  const int64_t Nxr = p.Nxr, Nyr = p.Nyr;
  const size_t nslot = p.nslot;
  float2* prop = static_cast<float2*>(ws);
  float2* g_eta = reinterpret_cast<float2*>(static_cast<char*>(ws) + align256(p.prop_bytes));
  float2* g_lev = reinterpret_cast<float2*>(static_cast<char*>(ws) + align256(p.prop_bytes) +
                                            align256(p.geta_bytes));
  // second intermediate buffer of the two-stream pipeline
  float2* g_lev2 = reinterpret_cast<float2*>(reinterpret_cast<char*>(g_lev) +
                                             align256(size_t(chunk) * p.per_level));
  Pipe* pipe = nullptr;
  const bool use_pipe = overlap && rowv == 2 && pair_path(p.ny, p.Nxr, p.Nyr);
  const bool eta_fork = eta_side && p.ny > 1;
  if (use_pipe || eta_fork) {
    int st = get_pipe(&pipe);
    if (st) return st;
  }
  struct EtaJoin {                               // the caller's stream waits for the eta stream
    Pipe* pp;
    cudaStream_t s;
    bool forked;
    ~EtaJoin() {
      if (!pp || !forked) return;
      cudaEventRecord(pp->eta_join, pp->eta_side);
      cudaStreamWaitEvent(s, pp->eta_join, 0);
    }
  } eta_join{eta_fork ? pipe : nullptr, stream, false};
  int chunk_no = 0;                              // chunks issued so far (over all time levels)
  struct Join {                                  // the caller's stream waits for the second one
    Pipe* pp;
    int* n;
    cudaStream_t s;
    ~Join() {
      if (!pp) return;
      for (int b = 0; b < 2 && b < *n; ++b) cudaStreamWaitEvent(s, pp->row_done[b], 0);
    }
  } join{use_pipe ? pipe : nullptr, &chunk_no, stream};

  const float kxs = float(6.283185307179586476925 / md->Lx);
  const float kys = ny > 1 ? float(6.283185307179586476925 / md->Ly) : 0.f;
  const float depth = md->depth > 0 ? float(md->depth) : 0.f;
  const int log2Nxr = ilog2(Nxr), log2Nyr = ilog2(Nyr);

  // launch shapes
  int fp = 4, cb = 1;
  while (fp > 1 && size_t(fp) * Nyr * sizeof(float2) > kSmemBudget) fp >>= 1;
  cb = int(std::max<size_t>(1, kSmemBudget / (size_t(fp) * Nyr * sizeof(float2))));
  cb = std::min(cb, std::min(64, Mh));
  int cb_eta = int(std::max<size_t>(1, kSmemBudget / (size_t(Nyr) * sizeof(float2))));
  cb_eta = std::min(cb_eta, std::min(64, Mh));
  // the eta transform is a single level: keep about two CTAs per SM busy rather than few wide ones
  cb_eta = std::min(cb_eta, std::max(1, (Mh + 303) / 304));
  const size_t rowb = size_t(2) * Nxr * sizeof(float2);
  int rb = int(std::max<size_t>(1, kSmemBudget / rowb));
  rb = int(std::min<int64_t>(rb, std::min<int64_t>(16, Nyr)));
  int rb_eta = int(std::max<size_t>(1, kSmemBudget / (size_t(Nxr) * sizeof(float2))));
  rb_eta = int(std::min<int64_t>(rb_eta, std::min<int64_t>(16, (Nyr + 1) / 2)));
  rb_eta = int(std::min<int64_t>(rb_eta, std::max<int64_t>(1, ((Nyr + 1) / 2 + 303) / 304)));
  const size_t smem_a = size_t(fp) * cb * Nyr * sizeof(float2);
  const size_t smem_a_eta = size_t(cb_eta) * Nyr * sizeof(float2);
  const size_t smem_b = size_t(rb) * rowb;
  const size_t smem_b_eta = size_t(rb_eta) * Nxr * sizeof(float2);
  {
    int st = set_smem((const void*)k_pass_a, std::max(smem_a, smem_a_eta));
    if (!st) st = set_smem((const void*)k_pass_b, std::max(smem_b, smem_b_eta));
    if (st) return st;
  }

  if (md->omega) {                                // all time levels' modes at once
    PropTimes T{};
    for (int l = 0; l < p.n_tl; ++l) T.dt[l] = t[l] - md->t_ref;
    k_propagate<<<dim3(unsigned((nslot + 255) / 256), unsigned(p.n_tl)), 256, 0, stream>>>(
        reinterpret_cast<const float2*>(md->A_eta), reinterpret_cast<const float2*>(md->A_phi),
        reinterpret_cast<const float2*>(md->A_phit), md->omega, int(nslot), T, prop);
    SWENSE_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  for (int l = 0; l < p.n_tl; ++l) {
    const float2 *Ae, *Ap, *At;
    if (md->omega) {
      float2* o = prop + size_t(l) * 3 * nslot;
      Ae = o;
      Ap = o + nslot;
      At = o + 2 * nslot;
    } else {
      Ae = reinterpret_cast<const float2*>(md->A_eta) + size_t(l) * nslot;
      Ap = reinterpret_cast<const float2*>(md->A_phi) + size_t(l) * nslot;
      At = reinterpret_cast<const float2*>(md->A_phit) + size_t(l) * nslot;
    }
    float4* nodes_l = reinterpret_cast<float4*>(nodes) + size_t(l) * nz * Nyr * Nxr;
    float* eta_l = eta + size_t(l) * Nyr * Nxr;

    PassBArgs b{};
    b.A_phi = Ap;
    b.A_phit = At;
    b.A_eta = Ae;
    b.nodes = nodes_l;
    b.eta = eta_l;
    b.tw = tw;
    b.Mh = Mh;
    b.Nxr = int(Nxr);
    b.log2Nxr = log2Nxr;
    b.Nyr = int(Nyr);
    b.kxs = kxs;
    b.depth = depth;
    b.spline = p.spline;

    if (ny == 1) {
      b.mode = B_ETA_DIRECT;
      b.rb = 1;
      b.lev0 = 0;
      k_pass_b<<<dim3(1, 1), kThreads, size_t(Nxr) * sizeof(float2), stream>>>(b, p.lev);
      SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
      b.mode = B_LEVEL_DIRECT;
      b.rb = 1;
      k_pass_b<<<dim3(1, nz), kThreads, rowb, stream>>>(b, p.lev);
      SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
      continue;
    }

    PassAArgs a{};
    a.A_phi = Ap;
    a.A_phit = At;
    a.A_eta = Ae;
    a.tw = tw;
    a.ny = ny;
    a.nxh1 = nxh1;
    a.Mh = Mh;
    a.Nyr = int(Nyr);
    a.log2Nyr = log2Nyr;
    a.kxs = kxs;
    a.kys = kys;
    a.depth = depth;
    a.Nxr = int(Nxr);
    a.spline = p.spline;

    // eta: pass A (eta mode) then pass B packing row pairs; on the eta stream when forked (the
    // time levels' eta transforms stay in order there, so they share one intermediate)
    cudaStream_t es = stream;
    if (eta_fork) {
      SWENSE_CUDA_TRY(cudaEventRecord(pipe->eta_fork, stream));
      SWENSE_CUDA_TRY(cudaStreamWaitEvent(pipe->eta_side, pipe->eta_fork, 0));
      eta_join.forked = true;
      es = pipe->eta_side;
    }
    a.G = g_eta;
    a.eta_mode = 1;
    a.fp = 1;
    a.cb = cb_eta;
    a.lev0 = 0;
    k_pass_a<<<dim3((Mh + cb_eta - 1) / cb_eta, 1), kThreads, smem_a_eta, es>>>(a, p.lev);
    SWENSE_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    b.G = g_eta;
    b.mode = B_ETA_G;
    b.rb = rb_eta;
    b.lev0 = 0;
    k_pass_b<<<dim3(unsigned((Nyr + 2 * rb_eta - 1) / (2 * rb_eta)), 1), kThreads, smem_b_eta,
               es>>>(b, p.lev);
    SWENSE_CUDA_TRY(cudaGetLastError());
    count_launches(1);

    if (lpc > 0 && (warp_path(ny, Nxr, Nyr) || (pair_path(ny, Nxr, Nyr) && rowv >= 2))) {
      ColArgs ca{};
      ca.A_phi = Ap;
      ca.A_phit = At;
      ca.G = g_lev;
      ca.tw = tw;
      ca.ny = ny;
      ca.nxh1 = nxh1;
      ca.Mh = Mh;
      ca.Nyr = int(Nyr);
      ca.cb = kColBlock;
      ca.lpc = lpc;
      ca.kxs = kxs;
      ca.kys = kys;
      ca.depth = depth;
      ca.Nxr = int(Nxr);
      ca.spline = p.spline;
      RowArgs ra{};
      ra.G = g_lev;
      ra.nodes = nodes_l;
      ra.tw = tw;
      ra.Mh = Mh;
      ra.Nxr = int(Nxr);
      ra.Nyr = int(Nyr);
      ra.rb = kRowBlock;
      ra.polls = kMbarPolls;
      ra.selftest = 0;
      const size_t smem_col = size_t(2) * ny * (kColBlock + 1) * sizeof(float2);
      const size_t smem_row = size_t(4) * Mh * (kRowBlock + 1) * sizeof(float2);
      ca.ldG = ra.ldG = trans_ld(Mh);
      const bool pair_t = (rowv == 2 || rowv == 3 || (rowv == 4 && Nxr <= 1024)) && pair_path(ny, Nxr, Nyr);
  
      for (int l0 = 0; l0 < nz; l0 += chunk) {
        if (pair_t && use_pipe) {
          const int nl = std::min(chunk, nz - l0);
          const int b = chunk_no & 1;
          ca.lev0 = l0;
          ca.nlev = nl;
          ra.lev0 = l0;
          ca.G = b ? g_lev2 : g_lev;
          ra.G = ca.G;
          if (chunk_no >= 2) SWENSE_CUDA_TRY(cudaStreamWaitEvent(stream, pipe->row_done[b], 0));
          int st = launch_pair_t(ca, ra, p.lev, nl, stream, false, false, 1, colv);   // column pass
          if (st) return st;
          SWENSE_CUDA_TRY(cudaEventRecord(pipe->col_done[b], stream));
          SWENSE_CUDA_TRY(cudaStreamWaitEvent(pipe->side, pipe->col_done[b], 0));
          st = launch_pair_t(ca, ra, p.lev, nl, pipe->side, false, false, 2);    // row pass
          if (st) return st;
          SWENSE_CUDA_TRY(cudaEventRecord(pipe->row_done[b], pipe->side));
          ++chunk_no;
          continue;
        }
        if (pair_t) {
          const int nl = std::min(chunk, nz - l0);
          ca.lev0 = l0;
          ca.nlev = nl;
          ra.lev0 = l0;
          int st = launch_pair_t(ca, ra, p.lev, nl, stream, rowv == 3, rowv == 4, 0, colv);
          if (st) return st;
          continue;
        }
        const int nl = std::min(chunk, nz - l0);
        ca.lev0 = l0;
        ca.nlev = nl;
        ra.lev0 = l0;
        int st = launch_col_e(int(Nyr / 32), ca, p.lev,
                              dim3((Mh + kColBlock - 1) / kColBlock, (nl + lpc - 1) / lpc),
                              smem_col, stream);
        if (!st) st = launch_row_e(int(Nxr / 32), ra,
                                   dim3(unsigned((Nyr + kRowBlock - 1) / kRowBlock), nl), smem_row, stream,
                                   rowv);
        if (st) return st;
      }
      continue;
    }
    a.eta_mode = 0;
    a.fp = fp;
    a.cb = cb;
    a.G = g_lev;
    b.G = g_lev;
    b.mode = B_LEVEL_G;
    b.rb = rb;
    for (int l0 = 0; l0 < nz; l0 += chunk) {
      const int nl = std::min(chunk, nz - l0);
      a.lev0 = l0;
      b.lev0 = l0;
      k_pass_a<<<dim3((Mh + cb - 1) / cb, nl), kThreads, smem_a, stream>>>(a, p.lev);
      SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
      k_pass_b<<<dim3(unsigned((Nyr + rb - 1) / rb), nl), kThreads, smem_b, stream>>>(b, p.lev);
      SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
    }
  }
  return SWENSE_OK;
}

}  // namespace
}  // namespace swense

namespace swense {
namespace {

// Zero-padding by a factor that is not a power of two, pad = q p2 with q odd: the refined node
// x_I, I = q J + s, is the p2-refined node x_J moved by s Lx / (pad nx), which is the p2-refined
// transform of the modes times e^{i k_x s Lx / (pad nx)} (the shift theorem; likewise in y).
// So the grid is q^2 (q in 2-D) power-of-two transforms of phase-shifted modes, each scattered
// to every q-th node. The spline prefilter, which depends on the final node spacing, is applied
// here, and the shifted transforms run as Lagrange grids.
__global__ void __launch_bounds__(256) k_shift_modes(const float2* __restrict__ ae, const float2* __restrict__ ap,
                                                     const float2* __restrict__ at, int nx, int ny, int64_t total,
                                                     int sx, int sy, int Nxr, int Nyr, int spline,
                                                     float2* __restrict__ oe, float2* __restrict__ op,
                                                     float2* __restrict__ ot) {
  const int nh1 = nx / 2 + 1;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int m = int(i % nh1);
    const int r = int((i / nh1) % ny);
    const int n = ny == 1 ? 0 : (r < ny / 2 ? r : r - ny);
    // phase in turns, reduced exactly in integers: m sx / Nxr + n sy / Nyr
    const int tx = int((int64_t(m) * sx) % Nxr);
    const int ty = ny == 1 ? 0 : int(((int64_t(n) * sy) % Nyr + Nyr) % Nyr);
    float tau = float(tx) / float(Nxr) + (ny == 1 ? 0.f : float(ty) / float(Nyr));
    tau -= floorf(tau);
    float sn, cs;
    sincospif(2.f * tau, &sn, &cs);
    const float f = spline ? spline_prefilter(m, Nxr, n, Nyr) : 1.f;
    const float c = f * cs, s2 = f * sn;
    const float2 e = __ldg(&ae[i]), p = __ldg(&ap[i]), t = __ldg(&at[i]);
    oe[i] = make_float2(c * e.x - s2 * e.y, c * e.y + s2 * e.x);
    op[i] = make_float2(c * p.x - s2 * p.y, c * p.y + s2 * p.x);
    ot[i] = make_float2(c * t.x - s2 * t.y, c * t.y + s2 * t.x);
  }
}

// Sub-grid node (tl, level, J_y, J_x) -> refined node (tl, level, qy J_y + sy, q J_x + sx).
__global__ void __launch_bounds__(256) k_scatter_grid(const float4* __restrict__ sn, const float* __restrict__ se,
                                                      int64_t n_nodes, int64_t n_eta, int nxs, int nys, int q,
                                                      int qy, int sx, int sy, int64_t Nxr, int64_t Nyr,
                                                      float4* __restrict__ nodes, float* __restrict__ eta) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_nodes + n_eta;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = i < n_nodes ? i : i - n_nodes;
    const int64_t jx = k % nxs, rest = k / nxs;
    const int64_t jy = rest % nys, slab = rest / nys;            // slab: (tl, level) or tl
    const int64_t o = (slab * Nyr + qy * jy + sy) * Nxr + q * jx + sx;
    if (i < n_nodes) nodes[o] = __ldg(&sn[k]);
    else eta[o] = __ldg(&se[k]);
  }
}

}  // namespace
}  // namespace swense

using namespace swense;

namespace swense {
namespace {

int fields_on_grid_shifted(const GridPlan& p, const swense_modes* md, const double* t, float* nodes,
                           float* eta, cudaStream_t stream) {
  int q = p.pad, p2 = 1;
  while (!(q & 1)) {
    q >>= 1;
    p2 <<= 1;
  }
  const int qy = p.ny > 1 ? q : 1;
  // the plan of one shifted power-of-two transform
  GridPlan sp = p;
  sp.pad = p2;
  sp.spline = 0;
  sp.Nxr = int64_t(p2) * p.nx;
  sp.Nyr = p.ny > 1 ? int64_t(p2) * p.ny : 1;
  sp.per_level = size_t(4) * sp.Nyr * trans_ld(sp.Mh) * sizeof(float2);
  sp.geta_bytes = p.ny > 1 ? size_t(sp.Nyr) * sp.Mh * sizeof(float2) : 0;
  const Tune tn = tuned(p.nx, p.ny, p2, p.nz);
  const int chunk = p.ny > 1 ? int(std::max<size_t>(1, std::min<size_t>(p.nz, tn.chunk_bytes / sp.per_level))) : 0;
  const bool pair = pair_path(sp.ny, sp.Nxr, sp.Nyr);
  const int lpc = tn.lpc >= 0 ? tn.lpc : (pair ? 4 : ((sp.Nxr <= 512 && sp.Nyr <= 512) ? kColLevels : 0));
  const int rowv0 = tn.lpc >= 0 ? tn.rowv : (pair ? 2 : 0);
  const int rowv = rowv0 == 5 ? 2 : rowv0;                    // one stream for the sub-grids
  const size_t scratch = align256(scratch_bytes(sp, chunk, 1));
  const int64_t sub_nodes = int64_t(p.n_tl) * p.nz * sp.Nyr * sp.Nxr;
  const int64_t sub_eta = int64_t(p.n_tl) * sp.Nyr * sp.Nxr;
  const int64_t nmodes = int64_t(md->n_snap) * p.ny * p.nxh1;
  const size_t b_nodes = align256(size_t(sub_nodes) * sizeof(float4));
  const size_t b_eta = align256(size_t(sub_eta) * sizeof(float));
  const size_t b_modes = align256(size_t(nmodes) * sizeof(float2));
  void* ws = nullptr;
  int st = workspace(scratch + b_nodes + b_eta + 3 * b_modes, stream, &ws);
  if (st) return st;
  char* base = static_cast<char*>(ws);
  float4* snodes = reinterpret_cast<float4*>(base + scratch);
  float* seta = reinterpret_cast<float*>(base + scratch + b_nodes);
  float2* sm = reinterpret_cast<float2*>(base + scratch + b_nodes + b_eta);
  swense_modes shifted = *md;
  shifted.A_eta = reinterpret_cast<const float*>(sm);
  shifted.A_phi = reinterpret_cast<const float*>(sm + b_modes / sizeof(float2));
  shifted.A_phit = reinterpret_cast<const float*>(sm + 2 * (b_modes / sizeof(float2)));
  const int threads = 256;
  for (int sy = 0; sy < qy; ++sy) {
    for (int sx = 0; sx < q; ++sx) {
      const int64_t mb = std::min<int64_t>((nmodes + threads - 1) / threads, int64_t(1) << 20);
      k_shift_modes<<<unsigned(mb), threads, 0, stream>>>(
          reinterpret_cast<const float2*>(md->A_eta), reinterpret_cast<const float2*>(md->A_phi),
          reinterpret_cast<const float2*>(md->A_phit), p.nx, p.ny, nmodes, sx, sy, int(p.Nxr), int(p.Nyr),
          p.spline, sm, sm + b_modes / sizeof(float2), sm + 2 * (b_modes / sizeof(float2)));
      SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
      st = launch_grid(sp, &shifted, t, reinterpret_cast<float*>(snodes), seta, ws, chunk, stream, lpc, rowv, 0, 0);
      if (st) return st;
      const int64_t tot = sub_nodes + sub_eta;
      const int64_t gb = std::min<int64_t>((tot + threads - 1) / threads, int64_t(152) * 64);
      k_scatter_grid<<<unsigned(gb), threads, 0, stream>>>(snodes, seta, sub_nodes, sub_eta, int(sp.Nxr),
                                                           int(sp.Nyr), q, qy, sx, sy, p.Nxr, p.Nyr,
                                                           reinterpret_cast<float4*>(nodes), eta);
      SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
    }
  }
  return SWENSE_OK;
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_fields_on_grid(const swense_modes* md, int32_t n_tl, const double* t,
                                     const swense_grid_desc* desc, float* nodes, float* eta,
                                     void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  GridPlan p;
  int st = plan_grid(md, n_tl, t, desc, nodes, eta, &p);
  if (st) return st;
  if (!is_pow2(p.pad)) return fields_on_grid_shifted(p, md, t, nodes, eta, stream);
  const Tune tn = tuned(p.nx, p.ny, p.pad, p.nz);
  const int chunk = p.ny > 1 ? int(std::max<size_t>(1, std::min<size_t>(p.nz, tn.chunk_bytes / p.per_level))) : 0;
  void* ws = nullptr;
  // untuned default: the transposed Stockham pair where both lengths are 256..1024, else the
  // warp path where its transforms stay in registers (n <= 512), else the shared-memory path
  const bool pair = pair_path(p.ny, p.Nxr, p.Nyr);
  const int lpc = tn.lpc >= 0 ? tn.lpc : (pair ? 4 : ((p.Nxr <= 512 && p.Nyr <= 512) ? kColLevels : 0));
  const int rowv = tn.lpc >= 0 ? tn.rowv : (pair ? 2 : 0);
  const int colv = tn.lpc >= 0 ? tn.colv : default_colv(p);
  // variant 5: variant 2 with its column and row passes pipelined over two streams
  const size_t ws_bytes = scratch_bytes(p, chunk, rowv == 5 ? 2 : 1);
  if (ws_bytes) {
    st = workspace(ws_bytes, stream, &ws);
    if (st) return st;
  }
  return launch_grid(p, md, t, nodes, eta, ws, chunk, stream, lpc, rowv == 5 ? 2 : rowv, rowv == 5, 1,
                     colv);
}

namespace swense {

// Scratch one swense_fields_on_grid call needs with its current launch shape, and the same call
// with that scratch supplied (no library stream: the eta transform and, for variant 5, the row
// passes stay on `stream`), for callers that run several reconstructions concurrently, each in
// its own part of the workspace (swense_batch_run).
int grid_scratch(const swense_modes* md, int32_t n_tl, const double* t, const swense_grid_desc* desc,
                 float* nodes, float* eta, size_t* bytes) {
  GridPlan p;
  int st = plan_grid(md, n_tl, t, desc, nodes, eta, &p);
  if (st) return st;
  if (!is_pow2(p.pad)) return fail(SWENSE_ERR_UNSUPPORTED, "batched grids take power-of-two padding factors");
  const Tune tn = tuned(p.nx, p.ny, p.pad, p.nz);
  const int chunk = p.ny > 1 ? int(std::max<size_t>(1, std::min<size_t>(p.nz, tn.chunk_bytes / p.per_level))) : 0;
  *bytes = scratch_bytes(p, chunk, 1);
  return SWENSE_OK;
}

int grid_with_scratch(const swense_modes* md, int32_t n_tl, const double* t, const swense_grid_desc* desc,
                      float* nodes, float* eta, void* ws, cudaStream_t stream) {
  GridPlan p;
  int st = plan_grid(md, n_tl, t, desc, nodes, eta, &p);
  if (st) return st;
  if (!is_pow2(p.pad)) return fail(SWENSE_ERR_UNSUPPORTED, "batched grids take power-of-two padding factors");
  const Tune tn = tuned(p.nx, p.ny, p.pad, p.nz);
  const int chunk = p.ny > 1 ? int(std::max<size_t>(1, std::min<size_t>(p.nz, tn.chunk_bytes / p.per_level))) : 0;
  const bool pair = pair_path(p.ny, p.Nxr, p.Nyr);
  const int lpc = tn.lpc >= 0 ? tn.lpc : (pair ? 4 : ((p.Nxr <= 512 && p.Nyr <= 512) ? kColLevels : 0));
  int rowv = tn.lpc >= 0 ? tn.rowv : (pair ? 2 : 0);
  if (rowv == 5) rowv = 2;
  const int colv = tn.lpc >= 0 ? tn.colv : default_colv(p);
  return launch_grid(p, md, t, nodes, eta, ws, chunk, stream, lpc, rowv, 0, 0, colv);
}

}  // namespace swense

extern "C" int swense_autotune_grid(const swense_modes* md, int32_t n_tl, const double* t,
                                    const swense_grid_desc* desc, float* nodes, float* eta,
                                    int32_t* lpc_out, int64_t* chunk_bytes_out, int32_t* row_variant_out,
                                    void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  GridPlan p;
  int st = plan_grid(md, n_tl, t, desc, nodes, eta, &p);
  if (st) return st;
  if (!is_pow2(p.pad))
    return fail(SWENSE_ERR_UNSUPPORTED, "autotune the power-of-two factor of the padding instead");
  Tune best{};
  if (p.ny > 1) {
    cudaEvent_t e0, e1;
    SWENSE_CUDA_TRY(cudaEventCreate(&e0));
    SWENSE_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    // Every timed repetition starts from a cold L2, as a solver's step does (its other work
    // evicts the grid): the workspace, sized for the largest candidate and at least twice the
    // L2, is overwritten before each repetition (its contents are scratch).
    constexpr size_t kFlushBytes = size_t(256) << 20;
    const size_t max_chunk = std::max<size_t>(1, std::min<size_t>(p.nz, (size_t(256) << 20) / p.per_level));
    const size_t ws_all = std::max(scratch_bytes(p, int(max_chunk), 2), kFlushBytes);
    {
      void* ws = nullptr;
      st = workspace(ws_all, stream, &ws);
      if (st) return st;
    }
    for (int lpc : {0, 1, 2, 4})
    for (int rv : {0, 1, 2, 3, 4, 5, 2 + 16, 3 + 16, 4 + 16, 5 + 16}) {
      const int rowv = rv & 15, colv = rv >> 4;
      const bool wp = warp_path(p.ny, p.Nxr, p.Nyr), pp = pair_path(p.ny, p.Nxr, p.Nyr);
      // beyond the warp path, the pair runs with row variant 2 (block rows) or, for 2048-point
      // rows, 3 (one 64-element-per-lane transform per warp)
      const bool pair_ok = pp && (rowv == 2 || (rowv == 3 && p.Nxr == 2048));
      if (lpc > 0 && !wp && !pair_ok) continue;
      if (rowv && (lpc == 0 || p.Nxr < 256)) continue;   // only the Stockham row sizes have variants
      if (rowv >= 2 && !pp) continue;
      if (colv && !(pp && rowv >= 2)) continue;
      if (!wp && !pair_ok && lpc > 0) continue;
      if (rowv == 4 && p.Nxr > 1024) continue;
      if (p.Nxr > 1024 && rowv != 2 && !(rowv == 3 && p.Nxr == 2048)) continue;
      for (size_t mb : {16, 32, 64, 96, 128, 256}) {
        const size_t cb = mb << 20;
        const int chunk = int(std::max<size_t>(1, std::min<size_t>(p.nz, cb / p.per_level)));
        void* ws = nullptr;
        st = workspace(ws_all, stream, &ws);
        const int rv2 = rowv == 5 ? 2 : rowv;
        if (!st) st = launch_grid(p, md, t, nodes, eta, ws, chunk, stream, lpc, rv2, rowv == 5, 1, colv);   // warm
        // best of five (the fastest repetition is the least disturbed one)
        float ms = 0.f, tot = 1e30f;
        for (int rep = 0; rep < 5 && !st; ++rep) {
          if (cudaMemsetAsync(ws, 0, kFlushBytes, stream) != cudaSuccess) { st = SWENSE_ERR_CUDA; break; }
          if (cudaEventRecord(e0, stream) != cudaSuccess) { st = SWENSE_ERR_CUDA; break; }
          st = launch_grid(p, md, t, nodes, eta, ws, chunk, stream, lpc, rv2, rowv == 5, 1, colv);
          if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = SWENSE_ERR_CUDA;
          tot = std::min(tot, ms);
        }
        if (st) break;
        if (tot < best_ms) {
          best_ms = tot;
          best.lpc = lpc;
          best.chunk_bytes = cb;
          best.rowv = rowv;
          best.colv = colv;
        }
      }
      if (st) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st == SWENSE_ERR_CUDA ? cuda_fail(cudaGetLastError(), "autotune timing") : st;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[{p.nx, p.ny, p.pad, p.nz}] = best;
  }
  if (lpc_out) *lpc_out = best.lpc;
  if (chunk_bytes_out) *chunk_bytes_out = int64_t(best.chunk_bytes);
  if (row_variant_out) *row_variant_out = best.rowv + 16 * best.colv;
  return SWENSE_OK;
}

extern "C" int swense_set_grid_tune(int32_t nx, int32_t ny, int32_t pad_n, int32_t nz, int32_t lpc,
                                    int64_t chunk_bytes, int32_t row_variant) {
  if (lpc != -1 && lpc != 0 && lpc != 1 && lpc != 2 && lpc != 4)
    return fail(SWENSE_ERR_ARG, "lpc must be -1 (default), 0, 1, 2 or 4");
  if (chunk_bytes < (int64_t(1) << 20) || chunk_bytes > (int64_t(1) << 30))
    return fail(SWENSE_ERR_ARG, "chunk_bytes must be in [1 MiB, 1 GiB]");
  if ((row_variant & 15) > 5 || (row_variant >> 4) > 1 || row_variant < 0)
    return fail(SWENSE_ERR_ARG, "row_variant must be 0..5, plus 16 for the one-field column pass");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  if (lpc == -1) {                      // back to the untuned defaults for this shape
    g_tune.erase({nx, ny, pad_n, nz});
    return SWENSE_OK;
  }
  Tune tn;
  tn.lpc = lpc;
  tn.chunk_bytes = size_t(chunk_bytes);
  tn.rowv = row_variant & 15;
  tn.colv = row_variant >> 4;
  g_tune[{nx, ny, pad_n, nz}] = tn;
  return SWENSE_OK;
}

// ---------------------------------------------------------------------------------------------
// Bounded device-side waits report here: the flag of this translation unit (k_row_tma).
namespace swense {

int grid_async_flag(bool reset, int* was_set) {
  int v = 0;
  SWENSE_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_async_timeout, sizeof(int)));
  if (reset && v) {
    const int zero = 0;
    SWENSE_CUDA_TRY(cudaMemcpyToSymbol(g_async_timeout, &zero, sizeof(int)));
  }
  *was_set = v;
  return SWENSE_OK;
}

}  // namespace swense

extern "C" int swense_selftest_wait_timeout(void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const float2* tw = nullptr;
  int st = twiddles(stream, &tw);
  if (st) return st;
  // one level of 256-point rows, 16 rows: the bulk copies are never issued, so the first wait of
  // every warp runs out after a few polls; nothing is read or written but the flag
  constexpr int N = 256, rows = 16;
  const size_t g_bytes = size_t(4) * rows * trans_ld(N / 2) * sizeof(float2);
  void* ws = nullptr;
  st = workspace(g_bytes + size_t(rows) * N * sizeof(float4), stream, &ws);
  if (st) return st;
  RowArgs r{};
  r.G = static_cast<const float2*>(ws);
  r.nodes = reinterpret_cast<float4*>(static_cast<char*>(ws) + g_bytes);
  r.tw = tw;
  r.Mh = N / 2;
  r.Nxr = N;
  r.Nyr = rows;
  r.rb = kRowBlock;
  r.ldG = trans_ld(N / 2);
  r.polls = 8;
  r.selftest = 1;
  return launch_row_tma<N>(r, 1u, stream);
}

// ---------------------------------------------------------------------------------------------
// swense_fields_on_grid_noalloc: the same kernels, with their scratch in a fixed device array
// that is part of the library image instead of the cudaMalloc'ed workspace.
namespace swense {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SWENSE_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64] = {};

// Device address of g_noalloc_scratch on the current device. The host-side symbol is only a
// stand-in, so the address is looked up once per device (with that device current) and cached.
int noalloc_scratch(void** out) {
  int dev = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SWENSE_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SWENSE_OK;
}

}  // namespace
}  // namespace swense

extern "C" int swense_fields_on_grid_noalloc(const swense_modes* md, int32_t n_tl, const double* t,
                                             const swense_grid_desc* desc, float* nodes,
                                             float* eta, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  GridPlan p;
  int st = plan_grid(md, n_tl, t, desc, nodes, eta, &p);
  if (st) return st;
  if (!is_pow2(p.pad))
    return fail(SWENSE_ERR_UNSUPPORTED, "padding factors that are not powers of two need the workspace (swense_fields_on_grid)");
  const size_t cap = size_t(SWENSE_NOALLOC_SCRATCH_BYTES);
  const size_t fixed = scratch_bytes(p, 0);
  int chunk = 0;
  if (p.ny > 1) {
    if (fixed + p.per_level > cap)
      return fail(SWENSE_ERR_SIZE,
                  "request needs " + std::to_string(fixed + p.per_level) +
                      " bytes of scratch for one level; swense_fields_on_grid_noalloc has " +
                      std::to_string(cap) + " (SWENSE_NOALLOC_SCRATCH_BYTES)");
    chunk = int(std::min<size_t>(size_t(p.nz), (cap - fixed) / p.per_level));
  } else if (fixed > cap) {
    return fail(SWENSE_ERR_SIZE, "request needs " + std::to_string(fixed) +
                                     " bytes of scratch; swense_fields_on_grid_noalloc has " +
                                     std::to_string(cap) + " (SWENSE_NOALLOC_SCRATCH_BYTES)");
  }
  void* ws = nullptr;
  st = noalloc_scratch(&ws);
  if (st) return st;
  // the launch shape swense_fields_on_grid would take (tuned, else its default), except that the
  // two-stream pipeline (variant 5) runs as variant 2: the fixed array holds one level chunk, not
  // two, and this call uses no library stream
  const Tune tn = tuned(p.nx, p.ny, p.pad, p.nz);
  const bool pair = pair_path(p.ny, p.Nxr, p.Nyr);
  const int lpc = tn.lpc >= 0 ? tn.lpc : (pair ? 4 : ((p.Nxr <= 512 && p.Nyr <= 512) ? kColLevels : 0));
  int rowv = tn.lpc >= 0 ? tn.rowv : (pair ? 2 : 0);
  if (rowv == 5) rowv = 2;
  const int colv = tn.lpc >= 0 ? tn.colv : default_colv(p);
  return launch_grid(p, md, t, nodes, eta, ws, chunk, stream, lpc, rowv, 0, 0, colv);
}
