// Many independent sea states in one call (workload of uneven instances). The reconstructions
// run concurrently on library streams forked from the caller's stream (largest instance first,
// round robin, each stream with its own part of the workspace, so small grids that cannot fill
// the GPU alone run side by side); after the join, every instance's gather goes through one
// planning launch and one persistent gather launch over a device queue of all the instances'
// point chunks (interp_batch). The fork and join are events, so a whole call can be captured as
// one CUDA graph and replayed as one launch. The first call (outside any capture) sizes the
// workspace and uploads the gather tables.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace swense {
namespace {

constexpr int kBatchStreams = 4;

struct BatchStreams {
  cudaStream_t s[kBatchStreams] = {};
  cudaEvent_t fork = nullptr, done[kBatchStreams] = {};
};
std::mutex g_bs_mutex;
BatchStreams g_bs[64];

int batch_streams(BatchStreams** out) {
  int dev = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SWENSE_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_bs_mutex);
  BatchStreams& b = g_bs[dev];
  if (!b.fork) {
    for (int k = 0; k < kBatchStreams; ++k) {
      SWENSE_CUDA_TRY(cudaStreamCreateWithFlags(&b.s[k], cudaStreamNonBlocking));
      SWENSE_CUDA_TRY(cudaEventCreateWithFlags(&b.done[k], cudaEventDisableTiming));
    }
    SWENSE_CUDA_TRY(cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming));
  }
  *out = &b;
  return SWENSE_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace swense

using namespace swense;

extern "C" int swense_batch_run(const swense_instance* inst, int32_t n, int32_t p_mode, double rho,
                                double g, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (n < 0) return fail(SWENSE_ERR_ARG, "negative instance count");
  if (n == 0) return SWENSE_OK;
  if (!inst) return fail(SWENSE_ERR_ARG, "NULL instance array");
  // scratch of each reconstruction (its tuned launch shape) and the gather items
  size_t slice = 0;
  std::vector<GatherItem> items(static_cast<size_t>(n));
  std::vector<double> weight(static_cast<size_t>(n));
  for (int32_t i = 0; i < n; ++i) {
    const swense_instance& c = inst[i];
    size_t b = 0;
    int st = grid_scratch(&c.modes, c.n_tl, c.t_levels, &c.desc, c.nodes, c.eta, &b);
    if (st) return st;
    slice = std::max(slice, align256(b));
    GatherItem& it = items[size_t(i)];
    it.grid = swense_grid{};
    it.grid.nodes = c.nodes;
    it.grid.eta = c.eta;
    it.grid.nx_r = c.desc.pad_n * c.modes.nx;
    it.grid.ny_r = c.modes.ny > 1 ? c.desc.pad_n * c.modes.ny : 1;
    it.grid.nz = c.desc.nz;
    it.grid.n_tl = c.n_tl;
    it.grid.Lx = c.modes.Lx;
    it.grid.Ly = c.modes.Ly;
    it.grid.z_levels = c.desc.z_levels;
    it.grid.t_levels = c.t_levels;
    it.grid.scheme = c.desc.scheme;
    it.t = c.t;
    it.pts = c.pts;
    it.perm = c.perm;
    it.np = c.np;
    it.eta = c.out_eta;
    it.u = c.out_u;
    it.v = c.out_v;
    it.w = c.out_w;
    it.p = c.out_p;
    weight[size_t(i)] = double(it.grid.nx_r) * it.grid.ny_r * c.desc.nz * c.n_tl;
  }
  size_t gbytes = 0;
  int st = interp_batch_bytes(items.data(), n, &gbytes);
  if (st) return st;
  void* ws = nullptr;
  st = workspace(size_t(kBatchStreams) * slice + gbytes, stream, &ws);
  if (st) return st;
  BatchStreams* bs = nullptr;
  st = batch_streams(&bs);
  if (st) return st;
  std::vector<int> order(static_cast<size_t>(n));
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return weight[size_t(a)] > weight[size_t(b)]; });
  // fork: every library stream starts after the work already on the caller's stream
  SWENSE_CUDA_TRY(cudaEventRecord(bs->fork, stream));
  const int used = std::min(kBatchStreams, int(n));
  for (int k = 0; k < used; ++k) SWENSE_CUDA_TRY(cudaStreamWaitEvent(bs->s[k], bs->fork, 0));
  int first_err = SWENSE_OK;
  for (int j = 0; j < n && !first_err; ++j) {
    const int i = order[size_t(j)], k = j % kBatchStreams;
    const swense_instance& c = inst[i];
    first_err = grid_with_scratch(&c.modes, c.n_tl, c.t_levels, &c.desc, c.nodes, c.eta,
                                  static_cast<char*>(ws) + size_t(k) * slice, bs->s[k]);
  }
  // join (also after an error, so that no stream is left forked from a capture)
  for (int k = 0; k < used; ++k) {
    SWENSE_CUDA_TRY(cudaEventRecord(bs->done[k], bs->s[k]));
    SWENSE_CUDA_TRY(cudaStreamWaitEvent(stream, bs->done[k], 0));
  }
  if (first_err) return first_err;
  return interp_batch(items.data(), n, p_mode, rho, g, static_cast<char*>(ws) + size_t(kBatchStreams) * slice,
                      stream);
}
