// Near-body direct modal sums on the fifth-generation tensor cores (tcgen05, sm_100 family).
//
// Paper: reconstruction section, analytical evaluation of the incident fields (the modal sums
// of Eqs. whatIsSpectralMethod1 / whatIsSpectralMethod evaluated at the points themselves: no
// grid, no interpolation error; cost proportional to the number of Fourier components per point).
//
// The sum F_c(p) = Re sum_{m,n} W_c[m,n] e^{i (kx_m x + ky_n y)} D_c(|k|, z) is reorganised so
// that its bulk is a dense contraction, without approximating anything beyond FP32 rounding:
//   1. separable phase: e^{i(kx x + ky y)} = X_m(x) Y_n(y), X_m = e^{i m 2 pi x / Lx};
//   2. depth factor about a centre z0: the points are sorted by z and cut into tiles of 128, two
//      consecutive tiles per CTA pair sharing z0 (the middle of their z range); with D = cosh or
//      sinh ratio (finite depth) or e^{|k| z} (deep water) and d/dz F = |k| S, d/dz S = |k| F,
//      the Taylor series to second order in dz = z - z0 is F(z) = F0 + |k| dz S0 +
//      (|k| dz)^2 / 2 F0 (S likewise with F0, S0 exchanged); the pair's kappa = max|k| max|dz|
//      is bounded (kKappaMax) so the dropped third-order term stays below 2e-6 relative, under
//      the split products' own rounding;
//   3. for each row n of modes and each field c and order j, T_{c,j,n}(p) = sum_m X_m(p)
//      C_{c,j}[m,n] with C = W_c |k|^j / j! (F0 or S0); rows n and -n share X_m and |k|, and
//      with Y_{-n} = conj(Y_n) their two terms add up to Re(Y_n (T_n + conj(T_{-n}))), so the
//      pair needs only Re(T_n + T_{-n}) and Im(T_n - T_{-n}): a (points x 2 m) by (2 m x
//      columns) real GEMM per K-chunk of 64 modes and group of 8 row pairs (26 columns per pair:
//      those two for u, v, w, dphi/dt at orders 0..2, and eta);
//   4. F_c(p) = sum_j dz^j sum_{n >= 0} Re(Y_n(p) (T_{c,j,n} + conj T_{c,j,-n})(p)): the
//      epilogue of every group.
// The GEMM runs as split BF16 (A = hi + lo, B = hi + lo, three products hi.hi + hi.lo + lo.hi
// accumulated in FP32 in tensor memory; the order-2 columns of B have no lo half, and the hi.lo
// product covers only the 144 columns that have one: an M = 256 MMA takes N / 2 cycles). Each cluster
// of two CTAs (cta_group::2) takes a tile pair: the even CTA's thread issues M = 256 MMAs over
// both CTAs' A (hi in tensor memory, lo in shared memory) and B halves (each CTA's producer warps
// make the columns of 4 of the group's 8 row pairs straight into its shared memory in the MMA's
// K-major core-matrix layout); accumulators are double-buffered in tensor memory so the epilogue
// of one group overlaps the MMAs of the next, and the next chunk's A is made while the current
// chunk runs. The epilogue reads each accumulator once per 64 modes, which keeps it under the
// MMA time. Tile pairs whose kappa is too large (sparse z) are left to the per-pair split-BF16
// kernel (direct.cu), which handles them exactly.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "mma.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace swense {
namespace {

constexpr int kTcM = 128;                             // points per tile (one CTA of the pair)
constexpr int kTcRows = 8;                            // mode row pairs (n, -n) per group
constexpr int kTcTerms = 3;                           // Taylor orders in dz: 0, 1, 2
constexpr int kTcCj = 4 * kTcTerms + 1;               // 13 complex outputs per row
constexpr int kTcN = kTcRows * 2 * kTcCj;             // 208 MMA columns
constexpr int kTcHalfRows = kTcRows / 2;              // row pairs whose B columns a CTA makes
constexpr int kTcNh = kTcN / 2;                       // 104 B columns per CTA
constexpr int kTcModes = 64;                          // modes m per K-chunk (one group's K)
constexpr int kTcK = 2 * kTcModes;                    // 128 K (re, im per mode)
// B layout (each CTA's half, columns nc = 8 slot + 2 pair + {0: Re(T_n + T_-n), 1: Im(T_n - T_-n)}
// for its 4 row pairs): one core matrix (8 columns x 8 K, 128 bytes) per output cj, at the slot
// tc_hslot gives; k-blocks of 8 K are kTcLBO bytes apart (13 core matrices + 16 bytes, so that
// the 32 lanes of a producer warp, one mode each, hit 32 different banks). In the pair's
// accumulator, column c < 104 comes from the even CTA's row pairs 0..3 and column 104 + c from
// the odd CTA's 4..7. The lo half holds only the 9 outputs below order 2 (slot tc_li, kTcLBOlo
// bytes per k-block); the hi.lo MMA (N = 144) writes accumulator columns 32 .. 175: the even
// CTA's slots 4..12 (its order-2 outputs take slots 0..3), then the odd CTA's 0..8 (its order-2
// outputs take 9..12).
constexpr int kTcNoLo = 4;                            // order-2 outputs (u, v, w, dphi/dt)
constexpr int kTcLoCj = kTcCj - kTcNoLo;              // 9 outputs with a lo half
constexpr int kTcNlo = kTcRows * 2 * kTcLoCj;         // 144: N of the hi.lo MMA
constexpr int kColLo = 8 * kTcNoLo;                   // its first accumulator column
constexpr int kTcSBO = 128;
constexpr int kTcLBO = (kTcNh / 8) * 128 + 16;
constexpr int kTcLBOlo = (kTcNlo / 2 / 8) * 128 + 16;
constexpr int kTcBBytes = (kTcK / 8) * kTcLBO;        // B hi
constexpr int kTcBLoBytes = (kTcK / 8) * kTcLBOlo;    // B lo
constexpr int kTcStageBytes = kTcBBytes + kTcBLoBytes;
constexpr bool tc_nolo(int cj) { return cj < 4 * kTcTerms && cj % kTcTerms == 2; }
// lo slot of an output with a lo half (cj order)
constexpr int tc_li(int cj) { return cj < 4 * kTcTerms ? (cj / kTcTerms) * 2 + cj % kTcTerms : 2 * 4; }
// hi slot of output cj in the B half of CTA `rank`
constexpr int tc_hslot(int rank, int cj) {
  return tc_nolo(cj) ? (rank ? kTcLoCj : 0) + cj / kTcTerms : (rank ? 0 : kTcNoLo) + tc_li(cj);
}
// Every output of a CTA's half has its own hi slot; an output with a lo half sits at accumulator
// column kColLo + rank kTcNlo / 2 + 8 tc_li (where the hi.lo MMA writes its lo products), an
// order-2 output outside the hi.lo MMA's columns.
constexpr bool tc_slots_ok() {
  for (int r = 0; r < 2; ++r)
    for (int a = 0; a < kTcCj; ++a) {
      if (tc_hslot(r, a) < 0 || tc_hslot(r, a) >= kTcCj) return false;
      for (int b = a + 1; b < kTcCj; ++b)
        if (tc_hslot(r, a) == tc_hslot(r, b)) return false;
      const int col = r * kTcNh + 8 * tc_hslot(r, a);
      const bool in_lo = col >= kColLo && col < kColLo + kTcNlo;
      if (tc_nolo(a) == in_lo) return false;
      if (!tc_nolo(a) && col != kColLo + r * (kTcNlo / 2) + 8 * tc_li(a)) return false;
    }
  return true;
}
static_assert(tc_slots_ok(), "B column slots of the two CTAs and the hi.lo MMA's columns");
static_assert(kColLo + kTcNlo == kTcNh + 8 * kTcLoCj, "the lo columns: the even CTA's last 9 slots, the odd CTA's first 9");
constexpr int kTcStages = 2;
// A's lo half (this CTA's 128 points x K) in shared memory, K-major core matrices: 16 along M
// per k-block, k-blocks kTcALBO bytes apart; its hi half is in tensor memory (columns 0..63).
// Tensor memory then holds A hi and two accumulators (64 + 2 x 208 of 512 columns), and the
// epilogue reads each accumulator once per 64 modes.
constexpr int kTcALBO = (kTcM / 8) * 128 + 16;
constexpr int kTcABytes = (kTcK / 8) * kTcALBO;
// the next chunk's A is made while the current chunk's groups run: its lo half into the other of
// two lo buffers, its hi half into a staging area (word j of point t at [j][t]) that is copied
// into tensor memory once the current chunk's MMAs are done
constexpr int kTcAHiBytes = kTcModes * kTcM * 4;
constexpr int kTcASmem = 2 * kTcABytes + kTcAHiBytes;
// per point, the row anchors Y^(8 j) (j < kYLo) of its groups: one group's first row in 64
constexpr int kYLo = 16;
constexpr int kYTabBytes = kYLo * kTcM * 8;
// 13 warps per CTA: 4 epilogue warps (one point each), 8 producer warps (two per row pair of
// this CTA's half, one per 32 modes of a group), 1 MMA warp (the even CTA's lane 0 issues for the
// pair; the warp owns the tensor-memory allocation in both CTAs)
constexpr int kEpiWarps = 4, kProdWarps = 8;
constexpr int kModeHalves = kTcModes / 32;
static_assert(kProdWarps == kModeHalves * kTcHalfRows, "one (row pair, 32 modes) block per producer warp");
constexpr int kMmaWarp = kEpiWarps + kProdWarps;
constexpr int kTcThreads = (kMmaWarp + 1) * 32;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColAhi = 0, kColD0 = kTcK / 2, kColD1 = kTcK / 2 + kTcN;
constexpr float kKappaMax = 0.02f;
constexpr int kZBuckets = 1 << 16;
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(2 * kTcM, kTcN);
constexpr uint32_t kIdescLo = tc::idesc_bf16_f32(2 * kTcM, kTcNlo);
// more than half of an SM's shared memory, so that one CTA of the kernel runs per SM (two
// pairs' CTAs sharing an SM would wait on each other's tensor memory)
constexpr size_t kTcSmemMin = 120 * 1024;
static_assert(kTcN % 16 == 0 && kTcN <= 256 && kTcNh % 8 == 0 && kTcNlo % 16 == 0, "MMA N for M = 256");
static_assert(kColD1 + kTcN <= kTmemCols, "tensor-memory columns");
static_assert(kTcStages * kTcStageBytes + kTcASmem + kYTabBytes + 2048 <= 227 * 1024, "shared memory");

// Set when a bounded wait of k_direct_tc gave up (read by swense_async_status).
__device__ int g_direct_timeout;

struct TcArgs {
  const float4* tab;        // [rows_p][mp] x 4: row n then row -n, each (W_phi, W_phit),
                            // (W_eta, |k|, 1/(1+e^{-2kh}))
  int rows_p, mp, ny;
  const float* spts;        // points sorted by z, [np][3]
  const int32_t* perm;      // sorted position -> caller's index
  int64_t np;
  float *o_eta, *o_u, *o_v, *o_w, *o_p;
  double inv_lx, inv_ly;
  float kxs, kys, depth, kmax;
  int p_mode;
  float rho, g;
  uint8_t* tile_bad;        // [ntiles]: 1 = left to the per-pair kernel
  int64_t ntiles;
  int polls;                // polls of a bounded wait (kMbarPolls; a few for the self-test)
  int withhold_a;           // self-test: A's arrivals are withheld, so the MMA's first wait runs out
};

// Table row q holds the mode rows n = q and n = -q (q = 0 .. ny/2 - 1; row -0 and the rows past
// ny/2 - 1 are zero modes; the Nyquist row is not in the table), rows padded to a multiple of 8.
// 2-D seas (ny = 1): row 0 holds n = 0.

// e^{k z} with the product k z carried as hi + lo (compensated), as for the grid's depth factors.
__device__ __forceinline__ float exp_kz(float k, float z) {
  const float kz = k * z;
  const float lo = fmaf(k, z, -kz);
  const float e = expf(kz);
  return fmaf(e, lo, e);
}

// hi + lo BF16 split of a pair (as bf2_split), the residual taken with one packed subtraction.
__device__ __forceinline__ void bf2_split_p(float2 v, unsigned& hi, unsigned& lo) {
  hi = bf2(v.x, v.y);
  const float2 r = csub(v, make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u)));
  lo = bf2(r.x, r.y);
}

// F = cosh(k(z+h))/cosh(kh), S = sinh(k(z+h))/cosh(kh) (finite depth), both e^{kz} in deep water.
__device__ __forceinline__ void depth_fs(float k, float z, float h, float invd, float& F, float& S) {
  const float e1 = exp_kz(k, z);
  if (h <= 0.f) {
    F = S = e1;
    return;
  }
  const float e2 = expf(-k * (z + 2.f * h));
  F = (e1 + e2) * invd;
  S = (e1 - e2) * invd;
}

// Warp-collective bounded wait: every lane polls; the warp succeeds only together. A wait that
// gives up (or sees another role give up) sets the CTA's abort flag and the device flag. The
// waits acquire at cluster scope: arrivals come from both CTAs of the pair.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, unsigned parity, volatile int* abort_flag, int polls) {
  bool ok = false;
  for (int it = 0; it < polls; ++it) {
    if (mbar_try_wait_cluster(bar, parity)) {
      ok = true;
      break;
    }
    if ((it & 31) == 31 && (*abort_flag || *(volatile int*)&g_direct_timeout)) break;
  }
  ok = __all_sync(0xffffffffu, ok);
  if (!ok && (threadIdx.x & 31) == 0) {
    *abort_flag = 1;
    atomicExch(&g_direct_timeout, 1);
  }
  return ok;
}
__device__ __forceinline__ bool thread_wait(uint64_t* bar, unsigned parity, volatile int* abort_flag, int polls) {
  for (int it = 0; it < polls; ++it) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if ((it & 31) == 31 && (*abort_flag || *(volatile int*)&g_direct_timeout)) {
      *abort_flag = 1;
      return false;
    }
  }
  *abort_flag = 1;
  atomicExch(&g_direct_timeout, 1);
  return false;
}

// One arrival per warp (cluster-scope release) on the even CTA's copy of a pair barrier, after
// the whole warp's preceding accesses (each lane has fenced them).
__device__ __forceinline__ void pair_arrive(uint64_t* bar, int lane) {
  __syncwarp();
  if (lane == 0) mbar_arrive_cluster(cluster_addr(bar, 0u));
}

struct TcShared {
  uint64_t b_full[kTcStages], b_empty[kTcStages], d_full[2], d_empty[2], a_ready, fin;
  uint32_t tmem;
  int abort_flag;
  float zmin[kTcThreads / 32], zmax[kTcThreads / 32];
};

// One cluster of two CTAs per pair of z-sorted tiles (256 points): the pair shares one expansion
// centre z0 and one B per group, each CTA making the B columns of 4 of the group's 8 row pairs,
// and the even CTA issues M = 256 MMAs over both CTAs' A and B. The pair's mbarriers that count
// arrivals of both CTAs (b_full, d_empty, a_ready) are the even CTA's; the MMA completions
// (b_empty, d_full, fin) arrive in both CTAs.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTcThreads, 1) k_direct_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* bst = smraw;                                   // kTcStages x (B hi, B lo)
  unsigned char* alo = smraw + kTcStages * kTcStageBytes;        // A lo, two chunks (this CTA's points)
  uint32_t* ahs = reinterpret_cast<uint32_t*>(alo + 2 * kTcABytes);  // next chunk's A hi [kTcModes][kTcM]
  float2* ytab = reinterpret_cast<float2*>(alo + kTcASmem);        // [kYLo][kTcM]
  TcShared& sh = *reinterpret_cast<TcShared*>(alo + kTcASmem + kYTabBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned rank = cluster_rank();                          // 0: even CTA, 1: odd CTA
  const int64_t tile = blockIdx.x;                               // rank == blockIdx.x & 1
  const int64_t p0 = tile * kTcM, pp0 = (tile - rank) * kTcM;     // this tile's, the pair's first point

  // ---- the pair's z range (both CTAs compute it from the same 256 points; padding repeats the
  // last point)
  {
    float lo = 3.4e38f, hi = -3.4e38f;
    for (int j = threadIdx.x; j < 2 * kTcM; j += kTcThreads) {
      const float zt = a.spts[3 * std::min<int64_t>(pp0 + j, a.np - 1) + 2];
      lo = fminf(lo, zt);
      hi = fmaxf(hi, zt);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      sh.zmin[warp] = lo;
      sh.zmax[warp] = hi;
    }
  }
  if (threadIdx.x == 0) sh.abort_flag = 0;
  __syncthreads();
  float zmin = sh.zmin[0], zmax = sh.zmax[0];
  for (int w = 1; w < kTcThreads / 32; ++w) {
    zmin = fminf(zmin, sh.zmin[w]);
    zmax = fmaxf(zmax, sh.zmax[w]);
  }
  const float z0 = 0.5f * (zmin + zmax);
  const float half = 0.5f * (zmax - zmin);
  if (a.kmax * half > kKappaMax) {                  // the same decision in both CTAs of the pair
    if (threadIdx.x == 0 && tile < a.ntiles) a.tile_bad[tile] = 1;
    return;
  }
  if (threadIdx.x == 0) {
    if (tile < a.ntiles) a.tile_bad[tile] = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&sh.b_full[s], 2 * kProdWarps);     // one arrival per producer warp
      mbar_init(&sh.b_empty[s], 1);
    }
    for (int d = 0; d < 2; ++d) {
      mbar_init(&sh.d_full[d], 1);
      mbar_init(&sh.d_empty[d], 2 * kEpiWarps);
    }
    mbar_init(&sh.a_ready, 2 * kEpiWarps);
    mbar_init(&sh.fin, 1);
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    tc::alloc2(&sh.tmem, kTmemCols);
    tc::relinquish2();
  }
  tc::fence_before();
  cluster_sync();                                   // both CTAs' barriers exist before any arrival
  tc::fence_after();
  const uint32_t tbase = sh.tmem;
  volatile int* abort_flag = &sh.abort_flag;
  const int nkc = a.mp / kTcModes, ng = a.rows_p / kTcRows, ngi = nkc * ng;

  if (warp < kEpiWarps) {
    // ================================================================ epilogue: one point each
    const int t = threadIdx.x;
    const int64_t pi = p0 + t;
    const bool live = pi < a.np;
    const int64_t ps = live ? pi : a.np - 1;
    const float x = a.spts[3 * ps], y = a.spts[3 * ps + 1], z = a.spts[3 * ps + 2];
    const unsigned X = turn_fraction(x, a.inv_lx), Y = a.ny > 1 ? turn_fraction(y, a.inv_ly) : 0u;
    const float dz = z - z0;
    float sy, cy;                                   // e^{i 2 pi y / Ly}: row step n -> n + 1
    sincospif(2.f * (float(int(Y)) * 2.3283064365386963e-10f), &sy, &cy);
    const uint32_t lanebase = tbase + ((uint32_t(warp) * 32u) << 16);
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};       // u, v, w, dphi/dt, eta
    const float dzp[kTcTerms] = {1.f, dz, dz * dz};  // each order's sums enter times dz^j

    // this point's row anchors: ytab[j] = Y^(8 j) as (Re, -Im), j < kYLo (exact, one
    // sine/cosine each); a group g >= kYLo also takes Y^(8 kYLo (g / kYLo)), kept in yhi
    for (int j = 0; j < kYLo; ++j) {
      const unsigned ph = unsigned(kTcRows * j) * Y;
      float si, co;
      sincospif(2.f * (float(int(ph)) * 2.3283064365386963e-10f), &si, &co);
      ytab[j * kTcM + t] = make_float2(co, -si);
    }
    float2 yhi = make_float2(1.f, 0.f);             // (Re, Im) of Y^(8 kYLo (g / kYLo))

    auto consume = [&](int gi, int g) {
      const uint32_t dcol = (gi & 1) ? kColD1 : kColD0;
      // Y_n(p) of the group's eight rows (consecutive n) as (Re Y, -Im Y): the anchor, then one
      // step per row
      float2 yv[kTcRows];
      {
        const float2 lo = ytab[(g % kYLo) * kTcM + t];          // (Re, -Im) of Y^(8 (g % kYLo))
        // (Re, -Im) of yhi * Y^(8 (g % kYLo))
        yv[0] = make_float2(fmaf(yhi.x, lo.x, yhi.y * lo.y), fmaf(yhi.x, lo.y, -yhi.y * lo.x));
      }
#pragma unroll
      for (int r = 1; r < kTcRows; ++r)
        yv[r] = make_float2(fmaf(yv[r - 1].x, cy, yv[r - 1].y * sy), fmaf(yv[r - 1].y, cy, -yv[r - 1].x * sy));
      // output cj: columns 8 tc_hslot(0, cj) .. + 7 (row pairs 0..3) and 104 + 8 tc_hslot(1, cj)
      // .. + 7 (pairs 4..7), (Re, Im) of each pair adjacent
      constexpr int kB = kTcCj;                      // every output's loads in flight, one wait
#pragma unroll
      for (int b0 = 0; b0 < kTcCj; b0 += kB) {
        uint32_t r[kB][2][8];
#pragma unroll
        for (int q = 0; q < kB; ++q)
          if (b0 + q < kTcCj) {
            tc::ld_x8(lanebase + dcol + uint32_t(8 * tc_hslot(0, b0 + q)), r[q][0]);
            tc::ld_x8(lanebase + dcol + uint32_t(kTcNh + 8 * tc_hslot(1, b0 + q)), r[q][1]);
          }
        tc::wait_ld();
        if (b0 + kB >= kTcCj) {                      // every column of this buffer is read
          tc::fence_before();
          pair_arrive(&sh.d_empty[gi & 1], lane);
        }
#pragma unroll
        for (int q = 0; q < kB; ++q) {
          if (b0 + q >= kTcCj) break;
          // (Re Y, -Im Y) x (Re T, Im T) pair by pair, summed as one packed pair
          float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int rr = 0; rr < kTcRows; ++rr)
            s2 = pfma(yv[rr],
                      make_float2(__uint_as_float(r[q][rr >> 2][2 * (rr & 3)]),
                                  __uint_as_float(r[q][rr >> 2][2 * (rr & 3) + 1])),
                      s2);
          const int cj = b0 + q;
          acc[cj / kTcTerms] = fmaf(dzp[cj % kTcTerms], s2.x + s2.y, acc[cj / kTcTerms]);
        }
      }
    };

    // A = X_m(p) of a K-chunk's 64 modes: word j = (cos, sin) of mode j as BF16. make_a: modes
    // 16 h .. 16 h + 15 of chunk kc, the lo residuals into the chunk's lo buffer (K pair j:
    // k-block j / 4, word j % 4 of this point's 16-byte row), the hi halves into the staging
    // area; put_a: the staged hi halves into tensor memory (columns 0..63), then the chunk's A
    // is announced
    auto make_a = [&](int kc, int h) {
      unsigned char* arow = alo + (kc & 1) * kTcABytes + (t >> 3) * 128 + (t & 7) * 16;
      uint32_t whi[16], wlo[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const unsigned m = unsigned(kc * kTcModes + 16 * h + j);
        const unsigned ph = m * X;
        float s, c;
        sincospif(2.f * (float(int(ph)) * 2.3283064365386963e-10f), &s, &c);
        bf2_split(c, s, whi[j], wlo[j]);
        ahs[(16 * h + j) * kTcM + t] = whi[j];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(arow + (4 * h + q) * kTcALBO) =
            make_uint4(wlo[4 * q], wlo[4 * q + 1], wlo[4 * q + 2], wlo[4 * q + 3]);
    };
    auto put_a = [&]() {
#pragma unroll 1
      for (int h = 0; h < kTcModes / 16; ++h) {
        uint32_t whi[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) whi[j] = ahs[(16 * h + j) * kTcM + t];
        tc::st_x16(lanebase + kColAhi + 16u * h, whi);
      }
      tc::wait_st();
      fence_proxy_async();                          // A lo: generic-proxy stores -> the MMA's reads
      tc::fence_before();
      if (!a.withhold_a) pair_arrive(&sh.a_ready, lane);
    };
#pragma unroll 1
    for (int h = 0; h < kTcModes / 16; ++h) make_a(0, h);
    put_a();
    bool ok = true;
    int made = 0;                                   // blocks of 16 modes of the next chunk's A made
    for (int gi = 0, g = 0, kc = 0; gi < ngi; ++gi) {
      if (g % kYLo == 0) {
        if (g == 0) {
          yhi = make_float2(1.f, 0.f);
        } else {
          const unsigned ph = unsigned(kTcRows * g) * Y;
          sincospif(2.f * (float(int(ph)) * 2.3283064365386963e-10f), &yhi.y, &yhi.x);
        }
      }
      ok = warp_wait(&sh.d_full[gi & 1], unsigned(gi >> 1) & 1u, abort_flag, a.polls);
      if (!ok) break;
      tc::fence_after();
      // the last group of a chunk is done, so are all MMAs reading this chunk's A: the next
      // chunk's A (made during this chunk) goes in before this group's epilogue
      if (g + 1 == ng && kc + 1 < nkc) {
        while (made < kTcModes / 16) make_a(kc + 1, made++);
        put_a();
      }
      consume(gi, g);
      if (g + 1 < ng && kc + 1 < nkc) {             // the next chunk's A, spread over this chunk
        while (made < ((kTcModes / 16) * (g + 1)) / (ng - 1)) make_a(kc + 1, made++);   // all by g = ng - 2
      }
      if (++g == ng) {
        made = 0;
        g = 0;
        ++kc;
      }
    }
    if (ok && live) {
      const float uu = acc[0], vv = acc[1], ww = acc[2], tt = acc[3];
      const int64_t o = a.perm[pi];
      if (a.o_eta) a.o_eta[o] = acc[4];
      if (a.o_u) a.o_u[o] = uu;
      if (a.o_v) a.o_v[o] = vv;
      if (a.o_w) a.o_w[o] = ww;
      if (a.o_p) {
        float p;
        if (a.p_mode == SWENSE_P_PHIT) {
          p = tt;
        } else {
          p = -a.rho * (tt + 0.5f * (uu * uu + vv * vv + ww * ww));
          if (a.p_mode == SWENSE_P_TOTAL) p -= a.rho * a.g * z;
        }
        a.o_p[o] = p;
      }
    }
  } else if (warp < kMmaWarp) {
    // ================================================================ producers: B per group
    const int pw = (warp - kEpiWarps) % kTcHalfRows;   // this CTA's row pair of the group
    const int mh = (warp - kEpiWarps) / kTcHalfRows;   // this warp's 32 modes of the group's 64
    const int pr = int(rank) * kTcHalfRows + pw;    // the pair's row pair
    const float h = a.depth;
    // this lane's mode is K pair 32 mh + lane: k-block 8 mh + lane / 4, word lane % 4 of a
    // 16-byte row; this pair's two rows (Re, Im) in each output's core matrix
    const uint32_t inrow = uint32_t(2 * pw) * 16u + uint32_t(lane & 3) * 4u;
    const uint32_t offh = uint32_t(8 * mh + (lane >> 2)) * kTcLBO + inrow;
    const uint32_t offl = uint32_t(8 * mh + (lane >> 2)) * kTcLBOlo + inrow;
    int g = 0, kc = 0;
    for (int gi = 0; gi < ngi; ++gi) {
      const int s = gi % kTcStages;
      const int tr = g * kTcRows + pr;              // mode rows n = tr and -tr
      const int m = kc * kTcModes + 32 * mh + lane;
      const float4* tp = &a.tab[4 * (size_t(tr) * a.mp + size_t(m))];
      const float4 c0 = __ldg(tp), c1 = __ldg(tp + 1), d0 = __ldg(tp + 2), d1 = __ldg(tp + 3);
      if (gi >= kTcStages &&
          !warp_wait(&sh.b_empty[s], unsigned(gi / kTcStages - 1) & 1u, abort_flag, a.polls))
        break;
      const float kx = float(m) * a.kxs, ky = float(tr) * a.kys, k = c1.z;   // |k| is that of both rows
      float F0, S0;
      depth_fs(k, z0, h, c1.w, F0, S0);
      const float k2 = 0.5f * k * k;
      const float P[kTcTerms] = {F0, k * S0, k2 * F0};      // F(z0 + dz) orders 0..2 (u, v, phi_t)
      const float Q[kTcTerms] = {S0, k * F0, k2 * S0};      // S(z0 + dz) orders 0..2 (w)
      // rows n (c) and -n (d): sums and differences of A^phi, A^phit, A^eta. With
      // W_u = i kx A^phi, W_v = i ky A^phi (ky negated on row -n), W_w = |k| A^phi, W_t = A^phit,
      // U = W(n) + W(-n) and V = W(n) - W(-n), the column Re(T_n + T_-n) takes the K pair
      // (Re U, -Im U) and the column Im(T_n - T_-n) the pair (Im V, Re V); below, those pairs
      // per field before the depth factor.
      const float2 sp = make_float2(c0.x + d0.x, c0.y + d0.y), dp = make_float2(c0.x - d0.x, c0.y - d0.y);
      const float2 st = make_float2(c0.z + d0.z, c0.w + d0.w), df = make_float2(c0.z - d0.z, c0.w - d0.w);
      const float2 Rf[4] = {make_float2(-kx * sp.y, -kx * sp.x), make_float2(-ky * dp.y, -ky * dp.x),
                            make_float2(k * sp.x, -k * sp.y), make_float2(st.x, -st.y)};
      const float2 If[4] = {make_float2(kx * dp.x, -kx * dp.y), make_float2(ky * sp.x, -ky * sp.y),
                            make_float2(k * dp.y, k * dp.x), make_float2(df.y, df.x)};
      unsigned char* bhi = bst + size_t(s) * kTcStageBytes;
      unsigned char* blo = bhi + kTcBBytes;
      // the order-2 columns have no lo half (their hi halves alone are exact to 2^-9 relative,
      // times (kappa^2 / 2) < 2e-4 from the expansion: below 4e-7)
      auto put = [&](int cj, float2 re, float2 im) {
        const uint32_t oh = offh + uint32_t(rank ? tc_hslot(1, cj) : tc_hslot(0, cj)) * kTcSBO;
        if (tc_nolo(cj)) {
          *reinterpret_cast<unsigned*>(bhi + oh) = bf2(re.x, re.y);
          *reinterpret_cast<unsigned*>(bhi + oh + 16) = bf2(im.x, im.y);
          return;
        }
        const uint32_t ol = offl + uint32_t(tc_li(cj)) * kTcSBO;
        unsigned h0, l0, h1, l1;
        bf2_split_p(re, h0, l0);
        bf2_split_p(im, h1, l1);
        *reinterpret_cast<unsigned*>(bhi + oh) = h0;
        *reinterpret_cast<unsigned*>(blo + ol) = l0;
        *reinterpret_cast<unsigned*>(bhi + oh + 16) = h1;
        *reinterpret_cast<unsigned*>(blo + ol + 16) = l1;
      };
#pragma unroll
      for (int j = 0; j < kTcTerms; ++j) {
        const float2 pj = make_float2(P[j], P[j]), qj = make_float2(Q[j], Q[j]);
        put(0 * kTcTerms + j, pmul(Rf[0], pj), pmul(If[0], pj));
        put(1 * kTcTerms + j, pmul(Rf[1], pj), pmul(If[1], pj));
        put(2 * kTcTerms + j, pmul(Rf[2], qj), pmul(If[2], qj));
        put(3 * kTcTerms + j, pmul(Rf[3], pj), pmul(If[3], pj));
      }
      put(4 * kTcTerms, make_float2(c1.x + d1.x, -(c1.y + d1.y)), make_float2(c1.y - d1.y, c1.x - d1.x));
      fence_proxy_async();                          // generic-proxy stores -> the MMA's reads
      pair_arrive(&sh.b_full[s], lane);
      if (++g == ng) {
        g = 0;
        ++kc;
      }
    }
  } else if (rank == 0) {
    // ================================================================ MMA issue (one thread)
    if (lane == 0) {
      bool ok = true;
      for (int kc = 0; kc < nkc && ok; ++kc) {
        ok = thread_wait(&sh.a_ready, unsigned(kc) & 1u, abort_flag, a.polls);
        if (!ok) break;
        tc::fence_after();
        for (int g = 0; g < ng; ++g) {
          const int gi = kc * ng + g, s = gi % kTcStages, d = gi & 1;
          ok = thread_wait(&sh.b_full[s], unsigned(gi / kTcStages) & 1u, abort_flag, a.polls);
          if (ok && gi >= 2)
            ok = thread_wait(&sh.d_empty[d], unsigned((gi >> 1) - 1) & 1u, abort_flag, a.polls);
          if (!ok) break;
          tc::fence_after();
          const uint32_t dacc = tbase + (d ? kColD1 : kColD0);
          unsigned char* bhi = bst + size_t(s) * kTcStageBytes;
          unsigned char* blo = bhi + kTcBBytes;
#pragma unroll
          for (int ks = 0; ks < kTcK / 16; ++ks) {
            const uint64_t dh = tc::smem_desc(bhi + 2 * ks * kTcLBO, kTcLBO, kTcSBO);
            const uint64_t dl = tc::smem_desc(blo + 2 * ks * kTcLBOlo, kTcLBOlo, kTcSBO);
            tc::mma2_ts(dacc, tbase + kColAhi + 8u * ks, dh, kIdesc, ks > 0 ? 1u : 0u);
            tc::mma2_ts(dacc + kColLo, tbase + kColAhi + 8u * ks, dl, kIdescLo, 1u);
            tc::mma2_ss(dacc, tc::smem_desc(alo + (kc & 1) * kTcABytes + 2 * ks * kTcALBO, kTcALBO, 128u), dh,
                        kIdesc, 1u);
          }
          tc::commit2(&sh.b_empty[s], uint16_t(3));
          tc::commit2(&sh.d_full[d], uint16_t(3));
        }
      }
      tc::commit2(&sh.fin, uint16_t(3));            // every MMA issued above has completed
    }
    __syncwarp();
  }

  // ---- teardown: once every MMA of the pair has completed (fin, in both CTAs) and both CTAs
  // are done with each other's barriers (cluster barrier), each frees its tensor memory
  if (warp == kMmaWarp) {
    bool done = false;
    for (int it = 0; it < kMbarPolls && !done; ++it) done = mbar_try_wait_cluster(&sh.fin, 0u);
    done = __all_sync(0xffffffffu, done);
    if (!done && lane == 0) atomicExch(&g_direct_timeout, 1);
  }
  tc::fence_before();
  cluster_sync();
  if (warp == kMmaWarp) {
    tc::fence_after();
    tc::dealloc2(tbase, kTmemCols);
  }
}

// ------------------------------------------------------------------------------------------------
// Mode table of the tensor-core path: entry (q, m, s) for row n = q (s = 0) and n = -q (s = 1),
// q < ny/2 (the Nyquist row is not in the table; row -0 is zero), rows padded to a multiple of 8
// and m = 0 .. nx/2 - 1 to a multiple of 32 with zero modes.
__global__ void k_tc_table(const float2* __restrict__ Ae, const float2* __restrict__ Ap,
                           const float2* __restrict__ At, const double* __restrict__ omega, double dt,
                           int nx, int ny, int rows_p, int mp, float kxs, float kys, float depth,
                           float4* __restrict__ tab) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(rows_p) * mp * 2) return;
  const int sgn = int(i & 1);
  const int64_t qm = i >> 1;
  const int tr = int(qm / mp), m = int(qm - int64_t(tr) * mp);
  float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = make_float4(0.f, 0.f, 0.f, 1.f);
  const int n = sgn ? -tr : tr;
  const bool live_row = ny > 1 ? (tr < ny / 2 && !(sgn && tr == 0)) : (tr == 0 && !sgn);
  if (live_row && m < nx / 2) {
    const int r = n >= 0 ? n : n + ny;                   // storage row of the half spectrum
    const size_t si = size_t(r) * (nx / 2 + 1) + m;
    float2 e = Ae[si], p = Ap[si], t = At[si];
    if (omega) {
      const double turns = omega[si] * dt * 0.15915494309189533577;
      const double frac = turns - rint(turns);
      float s, c;
      sincospif(2.f * float(frac), &s, &c);
      e = make_float2(fmaf(e.x, c, e.y * s), fmaf(e.y, c, -e.x * s));
      p = make_float2(fmaf(p.x, c, p.y * s), fmaf(p.y, c, -p.x * s));
      t = make_float2(fmaf(t.x, c, t.y * s), fmaf(t.y, c, -t.x * s));
    }
    const float kx = float(m) * kxs, ky = float(n) * kys;
    const float k = sqrtf(kx * kx + ky * ky);
    const float wgt = m == 0 ? 1.f : 2.f;
    c0 = make_float4(wgt * p.x, wgt * p.y, wgt * t.x, wgt * t.y);
    c1 = make_float4(wgt * e.x, wgt * e.y, k, depth > 0.f ? 1.f / (1.f + expf(-2.f * k * depth)) : 1.f);
  }
  tab[2 * i] = c0;
  tab[2 * i + 1] = c1;
}

// ------------------------------------------------------------------------------------------------
// Counting sort of the points by z (buckets over [min z, max z]); the order inside a bucket is
// unspecified (atomics), so a tile's composition, hence its z0, can differ between calls: results
// then differ at the level of the split products' rounding, never more.
__device__ __forceinline__ unsigned fkey(float z) {
  const unsigned u = __float_as_uint(z);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_z_range(const float* __restrict__ pts, int64_t np, unsigned* __restrict__ mm) {
  unsigned lo = 0xffffffffu, hi = 0u;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += int64_t(gridDim.x) * blockDim.x) {
    const unsigned k = fkey(pts[3 * i + 2]);
    lo = min(lo, k);
    hi = max(hi, k);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&mm[0], lo);
    atomicMax(&mm[1], hi);
  }
}

__device__ __forceinline__ int z_bucket(float z, float zlo, float scale) {
  return min(kZBuckets - 1, max(0, int((z - zlo) * scale)));
}

__global__ void k_z_count(const float* __restrict__ pts, int64_t np, const unsigned* __restrict__ mm,
                          unsigned* __restrict__ count) {
  const float zlo = fkey_inv(mm[0]), zhi = fkey_inv(mm[1]);
  const float scale = zhi > zlo ? float(kZBuckets) / (zhi - zlo) : 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += int64_t(gridDim.x) * blockDim.x)
    atomicAdd(&count[z_bucket(pts[3 * i + 2], zlo, scale)], 1u);
}

// Exclusive scan of the kZBuckets counts by one block (64 per thread).
__global__ void __launch_bounds__(1024) k_z_scan(unsigned* __restrict__ count) {
  __shared__ unsigned s[1024];
  constexpr int per = kZBuckets / 1024;
  unsigned v[per], tot = 0;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    v[j] = count[threadIdx.x * per + j];
    tot += v[j];
  }
  s[threadIdx.x] = tot;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned add = threadIdx.x >= unsigned(o) ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  unsigned run = s[threadIdx.x] - tot;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    count[threadIdx.x * per + j] = run;
    run += v[j];
  }
}

__global__ void k_z_scatter(const float* __restrict__ pts, int64_t np, const unsigned* __restrict__ mm,
                            unsigned* __restrict__ cursor, int32_t* __restrict__ perm, float* __restrict__ sorted) {
  const float zlo = fkey_inv(mm[0]), zhi = fkey_inv(mm[1]);
  const float scale = zhi > zlo ? float(kZBuckets) / (zhi - zlo) : 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += int64_t(gridDim.x) * blockDim.x) {
    const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    const unsigned pos = atomicAdd(&cursor[z_bucket(z, zlo, scale)], 1u);
    perm[pos] = int32_t(i);
    sorted[3 * size_t(pos)] = x;
    sorted[3 * size_t(pos) + 1] = y;
    sorted[3 * size_t(pos) + 2] = z;
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// ------------------------------------------------------------------------------------------------
// Self-test of the tensor-core data path: D (128 x N) = A (128 x K) x B^T (B: N x K), BF16 inputs
// (rounded from FP32), FP32 result, A from tensor memory (variant 0) or shared memory (variant 1),
// B from shared memory in the K-major core-matrix layout used above (k-blocks lbo bytes apart).
__global__ void __launch_bounds__(128, 1) k_tc_selftest(const float* __restrict__ A, const float* __restrict__ B,
                                                        float* __restrict__ D, int N, int K, int variant) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tm;
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t lbo = uint32_t(N / 8) * 128u + 16u;
  const uint32_t lboa = (kTcM / 8) * 128u + 16u;
  unsigned char* bs = smraw;                                    // B: (K / 8) k-blocks
  unsigned char* as = smraw + size_t(K / 8) * lbo;              // A (variant 1)
  for (int i = t; i < N * K / 2; i += 128) {
    const int nn = i / (K / 2), kp = i % (K / 2), k = 2 * kp;
    const uint32_t off = uint32_t(k / 8) * lbo + uint32_t(nn / 8) * 128u + uint32_t(nn % 8) * 16u + uint32_t(k % 8) * 2u;
    *reinterpret_cast<unsigned*>(bs + off) = bf2(B[size_t(nn) * K + k], B[size_t(nn) * K + k + 1]);
  }
  if (variant == 1) {
    for (int i = t; i < kTcM * K / 2; i += 128) {
      const int mm = i / (K / 2), kp = i % (K / 2), k = 2 * kp;
      const uint32_t off = uint32_t(k / 8) * lboa + uint32_t(mm / 8) * 128u + uint32_t(mm % 8) * 16u + uint32_t(k % 8) * 2u;
      *reinterpret_cast<unsigned*>(as + off) = bf2(A[size_t(mm) * K + k], A[size_t(mm) * K + k + 1]);
    }
  }
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tc::alloc(&tm, kTmemCols);
    tc::relinquish();
  }
  fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tb = tm;
  const uint32_t lanebase = tb + ((uint32_t(warp) * 32u) << 16);
  const uint32_t dcol = 256;
  if (variant == 0) {                               // A row t into columns 0 .. K/2 - 1
    for (int c0 = 0; c0 < K / 2; c0 += 16) {
      uint32_t w[16];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        w[j] = c0 + j < K / 2 ? bf2(A[size_t(t) * K + 2 * (c0 + j)], A[size_t(t) * K + 2 * (c0 + j) + 1]) : 0u;
      tc::st_x16(lanebase + uint32_t(c0), w);
    }
    tc::wait_st();
  }
  tc::fence_before();
  __syncthreads();
  if (t == 0) {
    tc::fence_after();
    const uint32_t idesc = tc::idesc_bf16_f32(kTcM, N);
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t bd = tc::smem_desc(bs + 2 * ks * lbo, lbo, 128u);
      if (variant == 0) {
        tc::mma_ts(tb + dcol, tb + 8u * ks, bd, idesc, ks > 0 ? 1u : 0u);
      } else {
        const uint64_t ad = tc::smem_desc(as + 2 * ks * lboa, lboa, 128u);
        tc::mma_ss(tb + dcol, ad, bd, idesc, ks > 0 ? 1u : 0u);
      }
    }
    tc::commit(&bar);
  }
  __syncwarp();
  bool done = false;
  for (int it = 0; it < kMbarPolls && !done; ++it) done = mbar_try_wait(&bar, 0u);
  done = __all_sync(0xffffffffu, done);
  tc::fence_after();
  if (done) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      tc::ld_x16(lanebase + dcol + uint32_t(c0), r);
      tc::wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) D[size_t(t) * N + c0 + j] = __uint_as_float(r[j]);
    }
  } else if ((t & 31) == 0) {
    atomicExch(&g_direct_timeout, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::dealloc(tb, kTmemCols);
  }
}

}  // namespace

int direct_async_flag(bool reset, int* was_set) {
  int v = 0;
  SWENSE_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_direct_timeout, sizeof(int)));
  if (reset && v) {
    const int zero = 0;
    SWENSE_CUDA_TRY(cudaMemcpyToSymbol(g_direct_timeout, &zero, sizeof(int)));
  }
  *was_set = v;
  return SWENSE_OK;
}

// Per device: the tile flags of the last tensor-core call (for swense_direct_stats).
struct TcLast {
  const uint8_t* bad = nullptr;
  int64_t ntiles = 0;
};
TcLast g_tc_last[64];
// self-test of the bounded waits, per device (swense_selftest_direct_wait_timeout)
bool g_tc_selftest[64];

// The tensor-core path of swense_direct (precision SWENSE_DIRECT_SPLIT_BF16): z sort, mode table,
// k_direct_tc over tiles of 128 sorted points, and the per-pair split kernel for the tiles it
// leaves (direct_split_sorted, direct.cu).
int direct_tc(const swense_modes* md, double t, const float* pts, int64_t np, float* eta, float* u,
              float* v, float* w, float* p, int32_t p_mode, double rho, double grav, cudaStream_t stream) {
  const int nx = md->nx, ny = md->ny;
  const int rows_p = ny > 1 ? (ny / 2 + kTcRows - 1) / kTcRows * kTcRows : kTcRows;   // row pairs
  const int mp = (nx / 2 + kTcModes - 1) / kTcModes * kTcModes;
  const int64_t ntiles = (np + kTcM - 1) / kTcM;
  if (ntiles >= (int64_t(1) << 31) || np >= (int64_t(1) << 31))
    return fail(SWENSE_ERR_SIZE, "too many points for one call of the tensor-core path");
  const size_t tab_b = align256(size_t(rows_p) * mp * 4 * sizeof(float4));
  const size_t mm_b = 256, cnt_b = align256(size_t(kZBuckets) * sizeof(unsigned));
  const size_t perm_b = align256(size_t(np) * sizeof(int32_t)), srt_b = align256(size_t(np) * 3 * sizeof(float));
  const size_t bad_b = align256(size_t(ntiles));
  const size_t split_off = tab_b + mm_b + cnt_b + perm_b + srt_b + bad_b;
  void* ws = nullptr;
  int st = workspace(split_off + split_table_bytes(md), stream, &ws);
  if (st) return st;
  char* base = static_cast<char*>(ws);
  float4* tab = reinterpret_cast<float4*>(base);
  unsigned* mm = reinterpret_cast<unsigned*>(base + tab_b);
  unsigned* cnt = reinterpret_cast<unsigned*>(base + tab_b + mm_b);
  int32_t* perm = reinterpret_cast<int32_t*>(base + tab_b + mm_b + cnt_b);
  float* srt = reinterpret_cast<float*>(base + tab_b + mm_b + cnt_b + perm_b);
  uint8_t* bad = reinterpret_cast<uint8_t*>(base + tab_b + mm_b + cnt_b + perm_b + srt_b);

  const float kxs = float(6.283185307179586476925 / md->Lx);
  const float kys = ny > 1 ? float(6.283185307179586476925 / md->Ly) : 0.f;
  const float depth = md->depth > 0 ? float(md->depth) : 0.f;
  {
    const int64_t n = int64_t(rows_p) * mp * 2;
    k_tc_table<<<unsigned((n + 255) / 256), 256, 0, stream>>>(
        reinterpret_cast<const float2*>(md->A_eta), reinterpret_cast<const float2*>(md->A_phi),
        reinterpret_cast<const float2*>(md->A_phit), md->omega, t - md->t_ref, nx, ny, rows_p, mp,
        kxs, kys, depth, tab);
    SWENSE_CUDA_TRY(cudaGetLastError());
  }
  SWENSE_CUDA_TRY(cudaMemsetAsync(mm, 0xff, sizeof(unsigned), stream));          // running min
  SWENSE_CUDA_TRY(cudaMemsetAsync(mm + 1, 0, sizeof(unsigned), stream));         // running max
  SWENSE_CUDA_TRY(cudaMemsetAsync(cnt, 0, size_t(kZBuckets) * sizeof(unsigned), stream));
  const unsigned gs = unsigned(std::min<int64_t>((np + 255) / 256, 152 * 8));
  k_z_range<<<gs, 256, 0, stream>>>(pts, np, mm);
  k_z_count<<<gs, 256, 0, stream>>>(pts, np, mm, cnt);
  k_z_scan<<<1, 1024, 0, stream>>>(cnt);
  k_z_scatter<<<gs, 256, 0, stream>>>(pts, np, mm, cnt, perm, srt);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(5);

  TcArgs a{};
  a.tab = tab;
  a.rows_p = rows_p;
  a.mp = mp;
  a.ny = ny;
  a.spts = srt;
  a.perm = perm;
  a.np = np;
  a.o_eta = eta;
  a.o_u = u;
  a.o_v = v;
  a.o_w = w;
  a.o_p = p;
  a.inv_lx = 1.0 / md->Lx;
  a.inv_ly = ny > 1 ? 1.0 / md->Ly : 0.0;
  a.kxs = kxs;
  a.kys = kys;
  a.depth = depth;
  {
    const double kx = double(nx / 2 - 1) * kxs, ky = ny > 1 ? double(ny / 2 - 1) * kys : 0.0;
    a.kmax = float(std::sqrt(kx * kx + ky * ky));
  }
  a.p_mode = p_mode;
  a.rho = float(rho);
  a.g = float(grav);
  a.tile_bad = bad;
  a.polls = kMbarPolls;
  a.withhold_a = 0;
  {
    int dev = 0;
    SWENSE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && g_tc_selftest[dev]) {
      a.polls = 8;
      a.withhold_a = 1;
    }
  }
  a.ntiles = ntiles;
  const size_t smem =
      std::max(size_t(kTcStages) * kTcStageBytes + kTcASmem + kYTabBytes + sizeof(TcShared), kTcSmemMin);
  SWENSE_CUDA_TRY(cudaFuncSetAttribute(k_direct_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  // clusters of two CTAs: one per pair of tiles (the odd CTA of a last, unpaired tile has no points)
  k_direct_tc<<<unsigned((ntiles + 1) / 2 * 2), kTcThreads, smem, stream>>>(a);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  {
    int dev = 0;
    SWENSE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64) g_tc_last[dev] = TcLast{bad, ntiles};
  }
  // tiles whose z range is too wide for the expansion: the per-pair kernel
  return direct_split_sorted(md, t, srt, perm, bad, kTcM, np, eta, u, v, w, p, p_mode, rho, grav, stream,
                             split_off);
}

}  // namespace swense

using namespace swense;

extern "C" int swense_direct_stats(int64_t* tiles, int64_t* fallback_tiles, void* stream) {
  if (!tiles || !fallback_tiles) return fail(SWENSE_ERR_ARG, "NULL output");
  int dev = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  *tiles = *fallback_tiles = 0;
  if (dev < 0 || dev >= 64 || !g_tc_last[dev].bad) return SWENSE_OK;
  SWENSE_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  std::vector<uint8_t> h(size_t(g_tc_last[dev].ntiles));
  SWENSE_CUDA_TRY(cudaMemcpy(h.data(), g_tc_last[dev].bad, h.size(), cudaMemcpyDeviceToHost));
  *tiles = g_tc_last[dev].ntiles;
  int64_t nb = 0;
  for (uint8_t b : h) nb += b != 0;
  *fallback_tiles = nb;
  return SWENSE_OK;
}

extern "C" int swense_selftest_tc_gemm(const float* A, const float* B, float* D, int32_t N, int32_t K,
                                       int32_t variant, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!A || !B || !D) return fail(SWENSE_ERR_ARG, "NULL operand");
  if (N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16 || (variant != 0 && variant != 1))
    return fail(SWENSE_ERR_ARG, "N in 16..256 (multiple of 16), K in 16..256 (multiple of 16), variant 0 or 1");
  const size_t smem = size_t(K / 8) * ((N / 8) * 128 + 16) + size_t(K / 8) * ((kTcM / 8) * 128 + 16);
  SWENSE_CUDA_TRY(cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  k_tc_selftest<<<1, 128, smem, stream>>>(A, B, D, N, K, variant);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}

extern "C" int swense_selftest_direct_wait_timeout(int32_t on) {
  int dev = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SWENSE_ERR_UNSUPPORTED, "device index too large");
  g_tc_selftest[dev] = on != 0;
  return SWENSE_OK;
}
