// Stream-function regular waves: the host solve of the modal amplitudes and the GPU evaluation
// of the incident fields at points.
//
// Paper: subsection on regular waves by stream-function theory (Rienecker & Fenton): basis
// functions psi_i(x - ct), so the amplitudes do not depend on time, found from the kinematic and
// dynamic free-surface conditions; and the "analytical evaluation" of such waves at the cells,
// affordable because N ~ 10 components suffice (ka = 0.24 converges with N = 9).
//
// Frame moving with the wave (crest at X = 0, z up from the mean level, depth h):
//   psi(X, z) = -ubar (z + h) + sum_j B_j S_j(z) cos(j k X)
//   S_j(z) = sinh(j k (z + h)) / cosh(j k h),  C_j(z) = cosh(j k (z + h)) / cosh(j k h)
//   U = -ubar + sum_j j k B_j C_j cos(j k X),  W = sum_j j k B_j S_j sin(j k X)
// Collocation at X_m = m pi / (N k), m = 0..N, with unknowns v = (k, eta_0..eta_N, B_1..B_N,
// ubar, Q, R):  psi(X_m, eta_m) + Q = 0;  (U^2 + W^2)/2 + g eta_m - R = 0;  trapezoidal mean of
// eta_m = 0;  eta_0 - eta_N = H;  ubar = 2 pi / (k T) (no mean Eulerian current, so c = ubar).
// Newton's method with the analytic Jacobian (k X_m = m pi / N does not depend on k), the height
// raised in steps from the linear wave. All in FP64 on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace swense {
namespace {

constexpr double kPi = 3.141592653589793238462643;

// Ratios C_j, S_j at s = z + h and tanh(j k h), without overflow for deep water.
struct Hyp {
  double C, S, T;
};
inline Hyp hyp(int j, double k, double z, double h) {
  const double a = std::exp(-2.0 * j * k * (z + h)), b = std::exp(-2.0 * j * k * h);
  const double e = std::exp(j * k * z) / (1.0 + b);
  return {e * (1.0 + a), e * (1.0 - a), (1.0 - b) / (1.0 + b)};
}

struct Problem {
  int n;
  double T, H, h, g;
  int nv() const { return 2 * n + 5; }
};

// Residuals r and Jacobian J (row-major nv x nv) at v.
void eval(const Problem& P, const std::vector<double>& v, std::vector<double>& r, std::vector<double>* J) {
  const int n = P.n, nv = P.nv();
  const double k = v[0], ubar = v[2 * n + 2], Q = v[2 * n + 3], R = v[2 * n + 4];
  const double* eta = &v[1];
  const double* B = &v[n + 2];
  r.assign(nv, 0.0);
  if (J) J->assign(size_t(nv) * nv, 0.0);
  auto Jr = [&](int row, int col) -> double& { return (*J)[size_t(row) * nv + col]; };
  for (int m = 0; m <= n; ++m) {
    const double z = eta[m], s = z + P.h;
    double psi = -ubar * s, U = -ubar, W = 0.0;
    double dpsi_dk = 0.0, dU_dz = 0.0, dW_dz = 0.0, dU_dk = 0.0, dW_dk = 0.0;
    std::vector<double> dU_dB(n), dW_dB(n), dpsi_dB(n);
    for (int j = 1; j <= n; ++j) {
      const Hyp q = hyp(j, k, z, P.h);
      const double cm = std::cos(j * m * kPi / n), sm = std::sin(j * m * kPi / n);
      const double jk = j * k, b = B[j - 1];
      const double dS_dk = j * (s * q.C - P.h * q.S * q.T), dC_dk = j * (s * q.S - P.h * q.C * q.T);
      psi += b * q.S * cm;
      U += jk * b * q.C * cm;
      W += jk * b * q.S * sm;
      dpsi_dk += b * cm * dS_dk;
      dU_dz += jk * b * jk * q.S * cm;
      dW_dz += jk * b * jk * q.C * sm;
      dU_dk += j * b * cm * (q.C + k * dC_dk);
      dW_dk += j * b * sm * (q.S + k * dS_dk);
      dpsi_dB[j - 1] = q.S * cm;
      dU_dB[j - 1] = jk * q.C * cm;
      dW_dB[j - 1] = jk * q.S * sm;
    }
    r[m] = psi + Q;                                         // kinematic
    r[n + 1 + m] = 0.5 * (U * U + W * W) + P.g * z - R;      // dynamic
    if (J) {
      Jr(m, 0) = dpsi_dk;
      Jr(m, 1 + m) = U;                                      // d psi / d eta_m
      for (int j = 0; j < n; ++j) Jr(m, n + 2 + j) = dpsi_dB[j];
      Jr(m, 2 * n + 2) = -s;
      Jr(m, 2 * n + 3) = 1.0;
      const int d = n + 1 + m;
      Jr(d, 0) = U * dU_dk + W * dW_dk;
      Jr(d, 1 + m) = U * dU_dz + W * dW_dz + P.g;
      for (int j = 0; j < n; ++j) Jr(d, n + 2 + j) = U * dU_dB[j] + W * dW_dB[j];
      Jr(d, 2 * n + 2) = -U;
      Jr(d, 2 * n + 4) = -1.0;
    }
  }
  const int rm = 2 * n + 2, rh = 2 * n + 3, rc = 2 * n + 4;
  double mean = 0.0;
  for (int m = 0; m <= n; ++m) mean += (m == 0 || m == n ? 0.5 : 1.0) * eta[m];
  r[rm] = mean / n;
  r[rh] = eta[0] - eta[n] - P.H;
  r[rc] = ubar - 2.0 * kPi / (k * P.T);
  if (J) {
    for (int m = 0; m <= n; ++m) Jr(rm, 1 + m) = (m == 0 || m == n ? 0.5 : 1.0) / n;
    Jr(rh, 1) = 1.0;
    Jr(rh, 1 + n) = -1.0;
    Jr(rc, 0) = 2.0 * kPi / (k * k * P.T);
    Jr(rc, 2 * n + 2) = 1.0;
  }
}

// Solve A x = b in place (A row-major n x n) by Gaussian elimination with partial pivoting.
bool solve_dense(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(A[size_t(i) * n + c]) > std::fabs(A[size_t(p) * n + c])) p = i;
    if (!(std::fabs(A[size_t(p) * n + c]) > 0.0)) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(A[size_t(p) * n + j], A[size_t(c) * n + j]);
      std::swap(b[p], b[c]);
    }
    for (int i = c + 1; i < n; ++i) {
      const double f = A[size_t(i) * n + c] / A[size_t(c) * n + c];
      if (f == 0.0) continue;
      for (int j = c; j < n; ++j) A[size_t(i) * n + j] -= f * A[size_t(c) * n + j];
      b[i] -= f * b[c];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double acc = b[i];
    for (int j = i + 1; j < n; ++j) acc -= A[size_t(i) * n + j] * b[j];
    b[i] = acc / A[size_t(i) * n + i];
  }
  return true;
}

// Root of (2 pi / T)^2 = g k tanh(k h) by bisection (the left side of g k tanh(k h) is monotone).
double linear_k(double T, double h, double g) {
  const double om2 = std::pow(2.0 * kPi / T, 2);
  double lo = 0.0, hi = om2 / g + 1.0 / h + 1.0;
  while (g * hi * std::tanh(hi * h) < om2) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    (g * mid * std::tanh(mid * h) < om2 ? lo : hi) = mid;
  }
  return 0.5 * (lo + hi);
}

struct StreamArgs {
  int n;
  float kt_hi, kt_lo;          // k / (2 pi) as an unevaluated sum: phase in turns = x k / (2 pi)
  float turn0;                 // (k (x0 + c t) / (2 pi)) mod 1
  float k, h, c, cu;           // cu = c - ubar (0 with no mean current)
  float R, g, rho;
  int p_mode;
  float ajk[SWENSE_STREAM_MAX_N];      // j k B_j / (1 + e^{-2 j k h})
  float E[SWENSE_STREAM_MAX_N + 1];
};

__global__ void __launch_bounds__(256) k_stream_eval(StreamArgs a, const float* __restrict__ pts, int64_t np,
                                                     float* __restrict__ o_eta, float* __restrict__ o_u,
                                                     float* __restrict__ o_v, float* __restrict__ o_w,
                                                     float* __restrict__ o_p) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float x = __ldg(&pts[3 * i]), z = __ldg(&pts[3 * i + 2]);
    // phase k (x - x0 - c t) in turns, x k / (2 pi) carried as hi + lo and reduced mod 1
    const float th = x * a.kt_hi;
    const float tl = fmaf(x, a.kt_hi, -th) + x * a.kt_lo;
    const float tau = (th - floorf(th)) + tl - a.turn0;
    float s1, c1;
    sincospif(2.f * tau, &s1, &c1);
    const float e1 = expf(a.k * z), f1 = expf(-2.f * a.k * (z + a.h));
    float cj = c1, sj = s1, ej = e1, fj = f1;
    float eta = a.E[0], u = a.cu, w = 0.f;
#pragma unroll 4
    for (int j = 1; j <= a.n; ++j) {
      // j k B_j C_j = ajk_j (e^{jkz} + e^{jkz} e^{-2jk(z+h)}), and the sinh ratio with a minus
      const float g = ej * fj;
      eta = fmaf(a.E[j], cj, eta);
      u = fmaf(a.ajk[j - 1] * (ej + g), cj, u);
      w = fmaf(a.ajk[j - 1] * (ej - g), sj, w);
      const float cn = cj * c1 - sj * s1;
      sj = fmaf(sj, c1, cj * s1);
      cj = cn;
      ej *= e1;
      fj *= f1;
    }
    if (o_eta) o_eta[i] = eta;
    if (o_u) o_u[i] = u;
    if (o_v) o_v[i] = 0.f;
    if (o_w) o_w[i] = w;
    if (o_p) {
      const float U = u - a.c;                                   // wave-frame horizontal velocity
      const float pdyn = a.rho * (a.R - 0.5f * (U * U + w * w)); // steady Bernoulli, p = 0 on the surface
      float p;
      if (a.p_mode == SWENSE_P_DYN) p = pdyn;
      else if (a.p_mode == SWENSE_P_TOTAL) p = pdyn - a.rho * a.g * z;
      else p = -pdyn / a.rho - 0.5f * (u * u + w * w);          // dphi/dt
      o_p[i] = p;
    }
  }
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_stream_solve(double period, double height, double depth, double g, int32_t n,
                                   int32_t height_steps, swense_stream_wave* out) {
  if (!out) return fail(SWENSE_ERR_ARG, "NULL output");
  if (n < 1 || n > SWENSE_STREAM_MAX_N) return fail(SWENSE_ERR_SIZE, "n must lie in 1..SWENSE_STREAM_MAX_N");
  if (!(period > 0.0 && height > 0.0 && depth > 0.0 && g > 0.0) || !std::isfinite(period + height + depth + g))
    return fail(SWENSE_ERR_ARG, "period, height, depth and g must be positive and finite");
  if (height_steps < 1 || height_steps > 1000) return fail(SWENSE_ERR_ARG, "height_steps must lie in 1..1000");
  Problem P{n, period, 0.0, depth, g};
  const int nv = P.nv();
  const double k0 = linear_k(period, depth, g), c0 = 2.0 * kPi / (k0 * period);
  std::vector<double> v(nv, 0.0), r, J;
  for (int s = 1; s <= height_steps; ++s) {
    P.H = height * s / height_steps;
    if (s == 1) {                                             // linear wave of the first height
      const double a = P.H / 2;
      v[0] = k0;
      for (int m = 0; m <= n; ++m) v[1 + m] = a * std::cos(m * kPi / n);
      v[n + 2] = c0 * a / std::tanh(k0 * depth);
      v[2 * n + 2] = c0;
      v[2 * n + 3] = c0 * depth;
      v[2 * n + 4] = 0.5 * c0 * c0;
    } else {                                                  // previous wave, surface rescaled
      const double f = double(s) / (s - 1);
      for (int m = 0; m <= n; ++m) v[1 + m] *= f;
    }
    const double scale = std::max({c0 * depth, c0 * c0, g * height, 1e-300});
    bool done = false;
    for (int it = 0; it < 80 && !done; ++it) {
      eval(P, v, r, &J);
      double rmax = 0.0;
      for (double x : r) rmax = std::max(rmax, std::fabs(x));
      if (rmax <= 1e-14 * scale) {
        done = true;
        break;
      }
      std::vector<double> dv = r;
      if (!solve_dense(J, dv, nv)) return fail(SWENSE_ERR_CONVERGENCE, "singular Newton system");
      double dmax = 0.0;
      for (int i = 0; i < nv; ++i) {
        v[i] -= dv[i];
        dmax = std::max(dmax, std::fabs(dv[i]) / std::max(std::fabs(v[i]), 1e-12 * scale));
      }
      if (!(v[0] > 0.0) || !std::isfinite(v[0])) return fail(SWENSE_ERR_CONVERGENCE, "wavenumber left (0, inf)");
      if (dmax < 1e-15) done = true;
    }
    eval(P, v, r, nullptr);
    double rmax = 0.0;
    for (double x : r) rmax = std::max(rmax, std::fabs(x));
    if (!(rmax <= 1e-9 * scale))
      return fail(SWENSE_ERR_CONVERGENCE, "no convergence (wave too steep for n, or too few height steps)");
  }
  swense_stream_wave& o = *out;
  o = swense_stream_wave{};
  o.n = n;
  o.k = v[0];
  o.ubar = v[2 * n + 2];
  o.c = o.ubar;
  o.Q = v[2 * n + 3];
  o.R = v[2 * n + 4];
  o.depth = depth;
  o.g = g;
  o.period = period;
  o.height = height;
  for (int j = 0; j < n; ++j) o.B[j] = v[n + 2 + j];
  for (int m = 0; m <= n; ++m) o.eta_m[m] = v[1 + m];
  for (int j = 0; j <= n; ++j) {                               // cosine coefficients of eta_m
    double acc = 0.0;
    for (int m = 0; m <= n; ++m) acc += (m == 0 || m == n ? 0.5 : 1.0) * v[1 + m] * std::cos(j * m * kPi / n);
    o.E[j] = (j == 0 || j == n ? 1.0 : 2.0) / n * acc;
  }
  return SWENSE_OK;
}

extern "C" int swense_stream_eval(const swense_stream_wave* wave, double t, double x0, const float* pts,
                                  int64_t np, float* eta, float* u, float* v, float* w, float* p,
                                  int32_t p_mode, double rho, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!wave) return fail(SWENSE_ERR_ARG, "NULL wave");
  if (wave->n < 1 || wave->n > SWENSE_STREAM_MAX_N) return fail(SWENSE_ERR_SIZE, "wave->n outside 1..SWENSE_STREAM_MAX_N");
  if (!(wave->k > 0.0 && wave->depth > 0.0) || !std::isfinite(wave->k + wave->c + wave->R))
    return fail(SWENSE_ERR_ARG, "wave not solved (k, depth must be positive)");
  if (p_mode < SWENSE_P_DYN || p_mode > SWENSE_P_TOTAL) return fail(SWENSE_ERR_ARG, "bad p_mode");
  if (np < 0) return fail(SWENSE_ERR_ARG, "negative point count");
  if (!std::isfinite(t) || !std::isfinite(x0)) return fail(SWENSE_ERR_ARG, "t and x0 must be finite");
  if (np == 0) return SWENSE_OK;
  if (!pts) return fail(SWENSE_ERR_ARG, "NULL points");
  StreamArgs a{};
  a.n = wave->n;
  const double kt = wave->k / (2.0 * kPi);
  a.kt_hi = float(kt);
  a.kt_lo = float(kt - double(a.kt_hi));
  double t0 = kt * (x0 + wave->c * t);
  t0 -= std::floor(t0);
  a.turn0 = float(t0);
  a.k = float(wave->k);
  a.h = float(wave->depth);
  a.c = float(wave->c);
  a.cu = float(wave->c - wave->ubar);
  a.R = float(wave->R);
  a.g = float(wave->g);
  a.rho = float(rho);
  a.p_mode = p_mode;
  for (int j = 1; j <= wave->n; ++j)
    a.ajk[j - 1] = float(j * wave->k * wave->B[j - 1] / (1.0 + std::exp(-2.0 * j * wave->k * wave->depth)));
  for (int j = 0; j <= wave->n; ++j) a.E[j] = float(wave->E[j]);
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((np + threads - 1) / threads, int64_t(1) << 30);
  k_stream_eval<<<unsigned(blocks), threads, 0, stream>>>(a, pts, np, eta, u, v, w, p);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return SWENSE_OK;
}
