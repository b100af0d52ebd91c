// Point binning for scattered point sets (no counterpart in the paper, whose CFD points come in
// mesh order): a counting sort of the points by grid tile (4 x 4 cells horizontally, one level
// stencil vertically, x fastest), so that consecutive points share grid stencils and the
// box-staged gather can keep them in shared memory. Produces the sorted coordinates and the
// permutation back to the caller's order; the order inside one tile is unspecified (atomics),
// which does not change any result (every point is evaluated on its own).
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace swense {
namespace {

constexpr int kTileX = 4, kTileY = 4;
constexpr int kScanBlock = 1024;

struct BinArgs {
  const float* pts;
  int64_t np;
  int Nxr, Nyr, nz, tx, ty;        // grid sizes; tiles per row / column
  float sx_hi, sx_lo, sy_hi, sy_lo;
  float z[SWENSE_MAX_LEVELS];
};

__device__ __forceinline__ int cell_of(float x, float hi, float lo, int n) {
  const float p = x * hi;
  const float e = fmaf(x, hi, -p);
  const float l = fmaf(x, lo, e);
  const float fl = floorf(p);
  const float f = (p - fl) + l;
  int i = int(fl);
  if (f < 0.f) i -= 1;
  else if (f >= 1.f) i += 1;
  if ((n & (n - 1)) == 0) return i & (n - 1);       // power-of-two node count
  const int r = i % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ unsigned tile_key(const BinArgs& a, int64_t i) {
  const float x = a.pts[3 * i], y = a.pts[3 * i + 1], zz = a.pts[3 * i + 2];
  const int ix = cell_of(x, a.sx_hi, a.sx_lo, a.Nxr);
  const int iy = a.Nyr > 1 ? cell_of(y, a.sy_hi, a.sy_lo, a.Nyr) : 0;
  int lo = 0, hi = a.nz;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a.z[mid] <= zz) lo = mid + 1; else hi = mid;
  }
  const int j = min(max(lo - 1, 0), a.nz - 2);
  const int j0 = min(max(j - 1, 0), a.nz - 4);
  return (unsigned(j0) * a.ty + unsigned(iy / kTileY)) * a.tx + unsigned(ix / kTileX);
}

__global__ void k_bin_count(BinArgs a, unsigned* __restrict__ key, unsigned* __restrict__ count) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.np;
       i += int64_t(gridDim.x) * blockDim.x) {
    const unsigned k = tile_key(a, i);
    key[i] = k;
    atomicAdd(&count[k], 1u);
  }
}

// Exclusive scan, pass 1: per-block scan (in place) and block totals.
__global__ void __launch_bounds__(kScanBlock) k_scan_blocks(unsigned* __restrict__ v, int64_t n,
                                                            unsigned* __restrict__ sums) {
  __shared__ unsigned s[kScanBlock];
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  const unsigned x = i < n ? v[i] : 0u;
  s[threadIdx.x] = x;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {          // Hillis-Steele inclusive scan
    const unsigned add = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  if (i < n) v[i] = s[threadIdx.x] - x;                 // exclusive
  if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = s[threadIdx.x];
}

// Pass 2: exclusive scan of the block totals by one block (serial chunks per thread).
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(unsigned* __restrict__ sums, int nb) {
  __shared__ unsigned s[kScanBlock];
  const int per = (nb + kScanBlock - 1) / kScanBlock;
  const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  unsigned tot = 0;
  for (int b = b0; b < b1; ++b) tot += sums[b];
  s[threadIdx.x] = tot;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    const unsigned add = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  unsigned run = s[threadIdx.x] - tot;
  for (int b = b0; b < b1; ++b) {
    const unsigned x = sums[b];
    sums[b] = run;
    run += x;
  }
}

__global__ void k_scan_add(unsigned* __restrict__ v, int64_t n, const unsigned* __restrict__ sums) {
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  if (i < n) v[i] += sums[blockIdx.x];
}

__global__ void k_bin_scatter(const float* __restrict__ pts, int64_t np,
                              const unsigned* __restrict__ key, unsigned* __restrict__ cursor,
                              int32_t* __restrict__ perm, float* __restrict__ sorted) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np;
       i += int64_t(gridDim.x) * blockDim.x) {
    const unsigned pos = atomicAdd(&cursor[key[i]], 1u);
    perm[pos] = int32_t(i);
    sorted[3 * size_t(pos)] = pts[3 * i];
    sorted[3 * size_t(pos) + 1] = pts[3 * i + 1];
    sorted[3 * size_t(pos) + 2] = pts[3 * i + 2];
  }
}

void split2(double v, float& hi, float& lo) {
  hi = float(v);
  lo = float(v - double(hi));
}

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_bin_points(const swense_grid* g, const float* pts, int64_t np, int32_t* perm,
                                 float* pts_sorted, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (!g || !g->z_levels) return fail(SWENSE_ERR_ARG, "NULL grid or levels");
  if (np < 0 || np > int64_t(0x7fffffff)) return fail(SWENSE_ERR_SIZE, "np must be in [0, 2^31)");
  if (np == 0) return SWENSE_OK;
  if (!pts || !perm || !pts_sorted) return fail(SWENSE_ERR_ARG, "NULL points or outputs");
  if ((g->nx_r & 1) || g->nx_r < 4 || g->nx_r > SWENSE_MAX_FFT ||
      (g->ny_r != 1 && ((g->ny_r & 1) || g->ny_r < 4)) || g->ny_r > SWENSE_MAX_FFT)
    return fail(SWENSE_ERR_SIZE, "grid sizes");
  if (g->nz < 4 || g->nz > SWENSE_MAX_LEVELS) return fail(SWENSE_ERR_LEVELS, "need 4 <= nz <= SWENSE_MAX_LEVELS");
  if (!(g->Lx > 0) || (g->ny_r > 1 && !(g->Ly > 0))) return fail(SWENSE_ERR_ARG, "domain lengths");
  BinArgs a{};
  for (int l = 0; l < g->nz; ++l) {
    a.z[l] = g->z_levels[l];
    if (!std::isfinite(a.z[l]) || (l > 0 && !(a.z[l] > a.z[l - 1])))
      return fail(SWENSE_ERR_LEVELS, "z_levels must be finite and strictly increasing");
  }
  a.pts = pts;
  a.np = np;
  a.Nxr = g->nx_r;
  a.Nyr = g->ny_r;
  a.nz = g->nz;
  a.tx = std::max(1, (g->nx_r + kTileX - 1) / kTileX);
  a.ty = std::max(1, (g->ny_r + kTileY - 1) / kTileY);
  split2(double(g->nx_r) / g->Lx, a.sx_hi, a.sx_lo);
  if (g->ny_r > 1) split2(double(g->ny_r) / g->Ly, a.sy_hi, a.sy_lo);
  const int64_t nkeys = int64_t(g->nz - 3) * a.ty * a.tx;
  const int64_t nblk = (nkeys + kScanBlock - 1) / kScanBlock;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t bytes = al(size_t(nkeys) * 4) + al(size_t(nblk) * 4) + al(size_t(np) * 4);
  void* ws = nullptr;
  int st = workspace(bytes, stream, &ws);
  if (st) return st;
  unsigned* count = static_cast<unsigned*>(ws);
  unsigned* sums = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + al(size_t(nkeys) * 4));
  unsigned* key = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + al(size_t(nkeys) * 4) + al(size_t(nblk) * 4));
  SWENSE_CUDA_TRY(cudaMemsetAsync(count, 0, size_t(nkeys) * 4, stream));
  const unsigned grid_pts = unsigned(std::min<int64_t>((np + 255) / 256, 152 * 32));
  k_bin_count<<<grid_pts, 256, 0, stream>>>(a, key, count);
  SWENSE_CUDA_TRY(cudaGetLastError());
  k_scan_blocks<<<unsigned(nblk), kScanBlock, 0, stream>>>(count, nkeys, sums);
  SWENSE_CUDA_TRY(cudaGetLastError());
  k_scan_sums<<<1, kScanBlock, 0, stream>>>(sums, int(nblk));
  SWENSE_CUDA_TRY(cudaGetLastError());
  k_scan_add<<<unsigned(nblk), kScanBlock, 0, stream>>>(count, nkeys, sums);
  SWENSE_CUDA_TRY(cudaGetLastError());
  k_bin_scatter<<<grid_pts, 256, 0, stream>>>(pts, np, key, count, perm, pts_sorted);
  SWENSE_CUDA_TRY(cudaGetLastError());
  count_launches(5);
  return SWENSE_OK;
}
