// Shared-memory inverse DFT (sign +, unnormalised) used by the grid reconstruction kernels.
//
// Iterative Cooley-Tukey decimation in time, in place: the caller scatters each length-n input
// into bit-reversed positions; the stages then combine sub-transforms of length h into 4h
// (two radix-2 stages fused in registers, three twiddle products), preceded by one radix-2 stage
// when log2(n) is odd. Output is in natural order. `batch` arrays of length n lie back to back.
#pragma once

#include "internal.cuh"

namespace swense {

// tw[j] = e^{+2 pi i j / SWENSE_MAX_FFT}
__device__ __forceinline__ void fft_inv_inplace(float2* data, int n, int log2n, int batch,
                                                const float2* __restrict__ tw) {
  const int nthr = blockDim.x;
  int h = 1;
  if (log2n & 1) {
    const int half = n >> 1;
    for (int t = threadIdx.x; t < batch * half; t += nthr) {
      const int b = t / half, j = t - b * half;
      float2* a = data + size_t(b) * n + 2 * j;
      const float2 x0 = a[0], x1 = a[1];
      a[0] = cadd(x0, x1);
      a[1] = csub(x0, x1);
    }
    h = 2;
    __syncthreads();
  }
  const int quarter = n >> 2;
  for (; h < n; h <<= 2) {
    const int s1 = SWENSE_MAX_FFT / (2 * h);  // twiddle stride of the length-2h stage
    const int s2 = s1 >> 1;                   // ... of the length-4h stage
    for (int t = threadIdx.x; t < batch * quarter; t += nthr) {
      const int b = t / quarter, r = t - b * quarter;
      const int g = r / h, j = r - g * h;
      float2* a = data + size_t(b) * n + g * 4 * h + j;
      const float2 w1 = __ldg(&tw[j * s1]);
      const float2 w2 = __ldg(&tw[j * s2]);
      const float2 x0 = a[0], x1 = a[h], x2 = a[2 * h], x3 = a[3 * h];
      const float2 t1 = cmul(w1, x1);
      const float2 a0 = cadd(x0, t1), a1 = csub(x0, t1);
      const float2 t3 = cmul(w1, x3);
      const float2 a2 = cadd(x2, t3), a3 = csub(x2, t3);
      const float2 t2 = cmul(w2, a2);
      const float2 u = cmul_i(cmul(w2, a3));
      a[0] = cadd(a0, t2);
      a[2 * h] = csub(a0, t2);
      a[h] = cadd(a1, u);
      a[3 * h] = csub(a1, u);
    }
    __syncthreads();
  }
}

// Depth factors of the spectral decomposition at vertical position z for |k| = k:
//   finite depth h > 0: F = cosh(k(z+h))/cosh(kh), S = sinh(k(z+h))/cosh(kh), written as
//     (e^{kz} +- e^{-k(z+2h)}) / (1 + e^{-2kh}) so that no term overflows;
//   deep water (h <= 0): F = S = e^{kz}.
// k*z is formed as an unevaluated sum hi + lo (fma residual) so the factor keeps FP32 accuracy
// for the large |k z| of the levels above z = 0.
__device__ __forceinline__ void depth_factors(float k, float z, float h, float& F, float& S) {
  const float kz = k * z;
  const float kz_lo = fmaf(k, z, -kz);
  float e1 = expf(kz);
  e1 = fmaf(e1, kz_lo, e1);
  if (h <= 0.f) {
    F = e1;
    S = e1;
    return;
  }
  const float e2 = expf(-k * (z + 2.f * h));
  const float d = 1.f + expf(-2.f * k * h);
  F = (e1 + e2) / d;
  S = (e1 - e2) / d;
}

// Prefilter of the periodic cubic-spline scheme. The spline interpolating grid values f_i is
// sum_j c_j B3(x/h - j) with (c_{i-1} + 4 c_i + c_{i+1}) / 6 = f_i; for one Fourier mode this
// divides its amplitude by the symbol (2 + cos(2 pi j / N)) / 3 of that averaging, per axis. So
// B-spline coefficients on the grid are the inverse transform of the modes divided by the
// symbols: 1 / prod over the horizontal axes, for signed mode j on an axis of N refined nodes.
__device__ __forceinline__ float spline_prefilter(int m, int Nx, int n, int Ny) {
  float f = 3.f / (2.f + cospif(2.f * float(m) / float(Nx)));
  if (Ny > 1) f *= 3.f / (2.f + cospif(2.f * float(n) / float(Ny)));
  return f;
}

}  // namespace swense

namespace swense {

// ------------------------------------------------------------------------------------------------
// Warp-register inverse DFT of length N = 32 * E (E <= 32), one transform per warp.
//
// With n = n1 + 32 n2 (n1 = lane, n2 < E) and m = m2 + E m1 (m2 < E, m1 < 32):
//   X[m] = sum_{n1} e^{2 pi i n1 m1 / 32} [ e^{2 pi i n1 m2 / N} sum_{n2} x[n1 + 32 n2] e^{2 pi i n2 m2 / E} ]
// so each lane does a length-E DFT over its own elements in registers, multiplies by the
// lane's twiddles, and the warp does E length-32 DFTs across lanes (radix-2 decimation in
// frequency with shuffles). Lane l ends up with X[m2 + E * bitrev5(l)], m2 = 0 .. E-1: E
// consecutive outputs, ready for a contiguous store.

constexpr int ct_log2(int v) { return v <= 1 ? 0 : 1 + ct_log2(v >> 1); }
constexpr int ct_rev(int v, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
  return r;
}

// Per-lane constants of one transform size (kernel-lifetime registers).
template <int E>
struct WarpFftTw {
  float2 wE[E > 1 ? E / 2 : 1];   // e^{2 pi i j / E}, j < E/2
  float2 w2[E];                   // e^{2 pi i lane m2 / N}
  float2 ws[5];                   // e^{2 pi i (lane mod s) / (2 s)}, s = 16, 8, 4, 2, 1
};

template <int E>
__device__ __forceinline__ void warp_fft_init(WarpFftTw<E>& T, const float2* __restrict__ tw, int lane) {
  constexpr int N = 32 * E;
#pragma unroll
  for (int j = 0; j < (E > 1 ? E / 2 : 1); ++j) T.wE[j] = __ldg(&tw[j * (SWENSE_MAX_FFT / (E > 1 ? E : 2))]);
#pragma unroll
  for (int m2 = 0; m2 < E; ++m2) T.w2[m2] = __ldg(&tw[(lane * m2) * (SWENSE_MAX_FFT / N)]);
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int s = 16 >> st;
    T.ws[st] = __ldg(&tw[(lane % s) * (SWENSE_MAX_FFT / (2 * s))]);
  }
}

// In-register length-E inverse DFT, natural order in and out (iterative radix-2 DIT).
template <int E>
__device__ __forceinline__ void dft_reg(float2 (&v)[E], const float2 (&wE)[E > 1 ? E / 2 : 1]) {
  constexpr int B = ct_log2(E);
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int j = ct_rev(i, B);
    if (j > i) {
      const float2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= E; len <<= 1) {
    const int half = len >> 1;
#pragma unroll
    for (int i = 0; i < E; i += len) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float2 b = v[i + j + half];
        const float2 t = j == 0 ? b : cmul(wE[j * (E / len)], b);
        v[i + j + half] = csub(v[i + j], t);
        v[i + j] = cadd(v[i + j], t);
      }
    }
  }
}

// Full warp transform: register DFT, lane twiddles, cross-lane length-32 DFT.
template <int E>
__device__ __forceinline__ void warp_fft(float2 (&v)[E], const WarpFftTw<E>& T, int lane) {
  dft_reg<E>(v, T.wE);
#pragma unroll
  for (int m2 = 1; m2 < E; ++m2) v[m2] = cmul(v[m2], T.w2[m2]);
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int s = 16 >> st;
    // lower lane: v + o; upper lane: (o - v) * w. Written as (o + sgn v) * w with sgn = -1 and
    // w = ws on upper lanes, sgn = +1 and w = 1 on lower lanes (no branch, no select per element)
    const bool upper = (lane & s) != 0;
    const float sgn = upper ? -1.f : 1.f;
    const float2 w = upper ? T.ws[st] : make_float2(1.f, 0.f);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      float2 o;
      o.x = __shfl_xor_sync(0xffffffffu, v[m].x, s);
      o.y = __shfl_xor_sync(0xffffffffu, v[m].y, s);
      const float2 r = make_float2(fmaf(sgn, v[m].x, o.x), fmaf(sgn, v[m].y, o.y));
      v[m] = s > 1 ? cmul(r, w) : r;
    }
  }
}

}  // namespace swense

namespace swense {

// ------------------------------------------------------------------------------------------------
// Per-warp Stockham inverse DFT of length N = 32 E (8 <= E <= 64), radix-8 passes followed by one
// radix-4 or radix-2 pass when log2 N is not a multiple of 3 (Stockham autosort: natural order in
// and out). Butterfly j of a pass with radix R after NS points have been combined reads
// x[j + r N/R], multiplies by e^{2 pi i (j mod NS) r / (NS R)}, takes the length-R DFT and writes
// y[(j / NS) NS R + (j mod NS) + r NS]. Lane l owns butterflies j = l + 32 b. Between passes the
// data go through a warp-private shared buffer with one pad element per 16 (index i + i/16),
// which keeps every exchange at the 2-wavefront minimum; the first pass reads registers filled
// by the caller (element b*8 + r holds position l + 32 b + r N/8) and the last pass leaves
// element b*R + r holding output position l + 32 b + r N/R (coalesced stores).

constexpr int stk_l2(int n) { return n <= 1 ? 0 : 1 + stk_l2(n >> 1); }
constexpr int stk_npass(int n) { return stk_l2(n) / 3 + (stk_l2(n) % 3 != 0 ? 1 : 0); }
constexpr int stk_radix(int n, int p) {
  return p < stk_l2(n) / 3 ? 8 : (stk_l2(n) % 3 == 1 ? 2 : 4);
}
constexpr int stk_ns(int n, int p) { return p == 0 ? 1 : stk_ns(n, p - 1) * stk_radix(n, p - 1); }
// distinct values of (j mod NS) among one lane's butterflies of pass p
constexpr int stk_dist(int n, int p) {
  return stk_ns(n, p) <= 32 ? 1
                            : (stk_ns(n, p) / 32 < n / 32 / stk_radix(n, p) ? stk_ns(n, p) / 32
                                                                            : n / 32 / stk_radix(n, p));
}
constexpr int stk_twoff(int n, int p) {
  return p <= 1 ? 0 : stk_twoff(n, p - 1) + stk_dist(n, p - 1) * (stk_radix(n, p - 1) - 1);
}
// passes 1 .. stk_regpass - 1 keep their twiddles in registers; later passes read the pass-major
// tables below (L1)
constexpr int stk_regpass(int n) { return n <= 256 ? stk_npass(n) : 2; }
constexpr int stk_twn(int n) { return stk_twoff(n, stk_regpass(n)) > 0 ? stk_twoff(n, stk_regpass(n)) : 1; }
constexpr int stk_buf(int n) { return n + n / 16; }   // padded buffer length (float2)

// Pass-major twiddles. Pass p >= 1 of an N-point transform (stride NS, radix R) multiplies by
// e^{+2 pi i jm r / (NS R)}, jm < NS, 0 < r < R. In the plain table that factor sits at
// jm r SWENSE_MAX_FFT / (NS R), so the lanes of a warp (consecutive jm) read entries r
// SWENSE_MAX_FFT / (NS R) apart: up to one L1 wavefront per lane. The twiddle array therefore also
// holds each factor at stk_twp(N, p) + (r - 1) NS + jm, where consecutive lanes read consecutive
// entries (2 wavefronts a warp). The tables of an N-point transform fill [SWENSE_MAX_FFT + N,
// SWENSE_MAX_FFT + 2 N): pass q holds NS_q (R_q - 1) = NS_{q+1} - NS_q entries, so pass p starts
// NS_p - NS_1 entries in.
constexpr int stk_twp(int n, int p) { return SWENSE_MAX_FFT + n + stk_ns(n, p) - stk_ns(n, 1); }
constexpr int kTwiddleLen = 3 * SWENSE_MAX_FFT;       // plain table + pass-major tables

// Exponent e of entry j of the twiddle array (the entry is e^{+2 pi i e / SWENSE_MAX_FFT}): j in
// the plain table; in the pass-major tables, jm r SWENSE_MAX_FFT / (NS R) of the transform size,
// pass, r and jm that slot j stands for; 0 in the slots no pass uses.
__host__ __device__ constexpr int twiddle_exponent(int j) {
  if (j < SWENSE_MAX_FFT) return j;
  const int i = j - SWENSE_MAX_FFT;
  int n = 1;
  while (2 * n <= i) n *= 2;                       // slot i lies in [n, 2n): the tables of size n
  int ns = stk_radix(n, 0);                        // stride NS_1 of pass 1
  const int o = i - n + ns;                        // pass p holds NS_p <= o < NS_{p+1}
  for (int p = 1; p < stk_npass(n); ++p) {
    const int R = stk_radix(n, p);
    if (o < ns * R) {
      const int q = o - ns;                        // (r - 1) NS + jm
      return (q % ns) * (q / ns + 1) * (SWENSE_MAX_FFT / (ns * R));
    }
    ns *= R;
  }
  return 0;
}

__device__ __forceinline__ int stk_pad(int i) { return i + (i >> 4); }

// Per-lane twiddles of the register-held passes (kernel-lifetime registers).
// (one template instance per pass, so every register index is a compile-time constant)
template <int N, int P = 1>
__device__ __forceinline__ void stk_init(float2 (&T)[stk_twn(N)], const float2* __restrict__ tw, int lane) {
  if constexpr (P < stk_regpass(N)) {
    constexpr int R = stk_radix(N, P), NS = stk_ns(N, P), D = stk_dist(N, P), OFF = stk_twoff(N, P);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int jm = NS <= 32 ? lane % NS : lane + 32 * d;
#pragma unroll
      for (int r = 1; r < R; ++r) T[OFF + d * (R - 1) + r - 1] = __ldg(&tw[jm * r * (SWENSE_MAX_FFT / (NS * R))]);
    }
    stk_init<N, P + 1>(T, tw, lane);
  }
}

// Inverse DFTs of length 2, 4, 8 in registers (natural order), constants folded.
__device__ __forceinline__ void stk_dft2(float2* v) {
  const float2 a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}
__device__ __forceinline__ void stk_dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
  const float2 t3 = cmul_i(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}
__device__ __forceinline__ void stk_dft8(float2* v) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  stk_dft4(e0, e1, e2, e3);
  stk_dft4(o0, o1, o2, o3);
  const float c = 0.70710678118654752f;                         // e^{i pi/4} = c (1 + i)
  o1 = make_float2(c * (o1.x - o1.y), c * (o1.x + o1.y));
  o2 = cmul_i(o2);
  o3 = make_float2(-c * (o3.x + o3.y), c * (o3.x - o3.y));      // e^{3 i pi/4} = c (-1 + i)
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

template <int N, int P>
__device__ __forceinline__ void stk_pass(float2 (&v)[N / 32], const float2 (&T)[stk_twn(N)],
                                         const float2* __restrict__ tw, float2* buf, int lane) {
  constexpr int E = N / 32, R = stk_radix(N, P), NS = stk_ns(N, P), B = E / R;
  if constexpr (P > 0 && P < stk_regpass(N)) {
    constexpr int OFF = stk_twoff(N, P);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int d = NS <= 32 ? 0 : b % (NS / 32);
#pragma unroll
      for (int r = 1; r < R; ++r)
        v[b * R + r] = cmul(v[b * R + r], T[OFF + d * (R - 1) + r - 1]);
    }
  } else if constexpr (P > 0) {
    constexpr int TP = stk_twp(N, P);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int jm = NS <= 32 ? lane % NS : lane + 32 * (b % (NS / 32));
#pragma unroll
      for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], __ldg(&tw[TP + (r - 1) * NS + jm]));
    }
  }
#pragma unroll
  for (int b = 0; b < B; ++b) {
    if constexpr (R == 8) stk_dft8(&v[b * 8]);
    else if constexpr (R == 4) stk_dft4(v[b * 4], v[b * 4 + 1], v[b * 4 + 2], v[b * 4 + 3]);
    else stk_dft2(&v[b * 2]);
  }
  if constexpr (P + 1 < stk_npass(N)) {
    // Output index of (b, r) = lane part + constant part with disjoint bits, so the padded index
    // splits the same way and every access is a per-pass base plus an immediate offset.
    const int lst = NS <= 32 ? (lane / NS) * NS * R + lane % NS : lane;
    float2* bst = buf + stk_pad(lst);
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = NS <= 32 ? 32 * b * R + r * NS
                               : (b / (NS / 32)) * NS * R + 32 * (b % (NS / 32)) + r * NS;
        bst[c + (c >> 4)] = v[b * R + r];
      }
    __syncwarp();
    constexpr int R2 = stk_radix(N, P + 1), B2 = E / R2;
    const float2* bld = buf + stk_pad(lane);
#pragma unroll
    for (int b = 0; b < B2; ++b)
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        const int c = 32 * b + r * (N / R2);
        v[b * R2 + r] = bld[c + (c >> 4)];
      }
    __syncwarp();
    stk_pass<N, P + 1>(v, T, tw, buf, lane);
  }
}

// Full transform; see the block comment above for the register layouts in and out.
template <int N>
__device__ __forceinline__ void stk_fft(float2 (&v)[N / 32], const float2 (&T)[stk_twn(N)],
                                        const float2* __restrict__ tw, float2* buf, int lane) {
  static_assert(N >= 256 && N <= 2048, "per-warp Stockham sizes");
  stk_pass<N, 0>(v, T, tw, buf, lane);
}

}  // namespace swense

namespace swense {

// ------------------------------------------------------------------------------------------------
// Block-wide Stockham inverse DFT of length N by TH threads (E = N / TH >= 8 elements each), the
// same radix-8 (then 4 or 2) passes as stk_fft with "lane" generalised to the thread index and
// the exchange through a padded block-shared buffer under __syncthreads. Twiddles come from the
// pass-major tables (L1). Layouts: on entry element b*8 + r of thread t holds position
// t + TH b + r N/8; on exit element b*R + r holds t + TH b + r N/R (R = radix of the last pass).
template <int N, int TH, int P>
__device__ __forceinline__ void stkb_pass(float2 (&v)[N / TH], const float2* __restrict__ tw,
                                          float2* buf, int t) {
  constexpr int E = N / TH, R = stk_radix(N, P), NS = stk_ns(N, P), B = E / R;
  static_assert(B >= 1, "each thread holds at least one butterfly per pass");
  if constexpr (P > 0) {
    constexpr int TP = stk_twp(N, P);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int jm = NS <= TH ? t % NS : t + TH * (b % (NS / TH));
#pragma unroll
      for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], __ldg(&tw[TP + (r - 1) * NS + jm]));
    }
  }
#pragma unroll
  for (int b = 0; b < B; ++b) {
    if constexpr (R == 8) stk_dft8(&v[b * 8]);
    else if constexpr (R == 4) stk_dft4(v[b * 4], v[b * 4 + 1], v[b * 4 + 2], v[b * 4 + 3]);
    else stk_dft2(&v[b * 2]);
  }
  if constexpr (P + 1 < stk_npass(N)) {
    // thread part and constant part of each index have disjoint bits (as in stk_pass)
    const int lst = NS <= TH ? (t / NS) * NS * R + t % NS : t;
    float2* bst = buf + stk_pad(lst);
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = NS <= TH ? TH * b * R + r * NS
                               : (b / (NS / TH)) * NS * R + TH * (b % (NS / TH)) + r * NS;
        bst[c + (c >> 4)] = v[b * R + r];
      }
    __syncthreads();
    constexpr int R2 = stk_radix(N, P + 1), B2 = E / R2;
    const float2* bld = buf + stk_pad(t);
#pragma unroll
    for (int b = 0; b < B2; ++b)
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        const int c = TH * b + r * (N / R2);
        v[b * R2 + r] = bld[c + (c >> 4)];
      }
    __syncthreads();
    stkb_pass<N, TH, P + 1>(v, tw, buf, t);
  }
}

template <int N, int TH>
__device__ __forceinline__ void stkb_fft(float2 (&v)[N / TH], const float2* __restrict__ tw, float2* buf,
                                         int t) {
  static_assert(N / TH >= 8 && N <= SWENSE_MAX_FFT && (TH & 15) == 0, "block Stockham sizes");
  static_assert(N / 8 >= TH, "constant index parts are multiples of the thread count");
  stkb_pass<N, TH, 0>(v, tw, buf, t);
}

// Two block-wide transforms of the same length side by side (buffers buf1, buf2): each pass
// applies to both before the shared barriers, so the pair takes the barriers of one transform
// and twice the independent work between them.
template <int N, int TH, int P>
__device__ __forceinline__ void stkb_pass2(float2 (&v1)[N / TH], float2 (&v2)[N / TH],
                                           const float2* __restrict__ tw, float2* buf1, float2* buf2, int t) {
  constexpr int E = N / TH, R = stk_radix(N, P), NS = stk_ns(N, P), B = E / R;
  if constexpr (P > 0) {
    constexpr int TP = stk_twp(N, P);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int jm = NS <= TH ? t % NS : t + TH * (b % (NS / TH));
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = __ldg(&tw[TP + (r - 1) * NS + jm]);
        v1[b * R + r] = cmul(v1[b * R + r], w);
        v2[b * R + r] = cmul(v2[b * R + r], w);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < B; ++b) {
    if constexpr (R == 8) {
      stk_dft8(&v1[b * 8]);
      stk_dft8(&v2[b * 8]);
    } else if constexpr (R == 4) {
      stk_dft4(v1[b * 4], v1[b * 4 + 1], v1[b * 4 + 2], v1[b * 4 + 3]);
      stk_dft4(v2[b * 4], v2[b * 4 + 1], v2[b * 4 + 2], v2[b * 4 + 3]);
    } else {
      stk_dft2(&v1[b * 2]);
      stk_dft2(&v2[b * 2]);
    }
  }
  if constexpr (P + 1 < stk_npass(N)) {
    const int lst = NS <= TH ? (t / NS) * NS * R + t % NS : t;
    float2* bst1 = buf1 + stk_pad(lst);
    float2* bst2 = buf2 + stk_pad(lst);
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = NS <= TH ? TH * b * R + r * NS
                               : (b / (NS / TH)) * NS * R + TH * (b % (NS / TH)) + r * NS;
        bst1[c + (c >> 4)] = v1[b * R + r];
        bst2[c + (c >> 4)] = v2[b * R + r];
      }
    __syncthreads();
    constexpr int R2 = stk_radix(N, P + 1), B2 = E / R2;
    const float2* bld1 = buf1 + stk_pad(t);
    const float2* bld2 = buf2 + stk_pad(t);
#pragma unroll
    for (int b = 0; b < B2; ++b)
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        const int c = TH * b + r * (N / R2);
        v1[b * R2 + r] = bld1[c + (c >> 4)];
        v2[b * R2 + r] = bld2[c + (c >> 4)];
      }
    __syncthreads();
    stkb_pass2<N, TH, P + 1>(v1, v2, tw, buf1, buf2, t);
  }
}

template <int N, int TH>
__device__ __forceinline__ void stkb_fft2(float2 (&v1)[N / TH], float2 (&v2)[N / TH],
                                          const float2* __restrict__ tw, float2* buf1, float2* buf2, int t) {
  static_assert(N / TH >= 8 && N <= SWENSE_MAX_FFT && (TH & 15) == 0, "block Stockham sizes");
  static_assert(N / 8 >= TH, "constant index parts are multiples of the thread count");
  stkb_pass2<N, TH, 0>(v1, v2, tw, buf1, buf2, t);
}

}  // namespace swense
