// Per-device scratch workspace, twiddle table and error reporting.
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>

#include "fft.cuh"
#include "internal.cuh"

namespace swense {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int status, const std::string& msg) {
  g_last_error = std::string(swense_strerror(status)) + ": " + msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string("SWENSE_ERR_CUDA: ") + what + ": " + cudaGetErrorString(e);
  return SWENSE_ERR_CUDA;
}

namespace {

constexpr int kMaxDevices = 64;

struct DeviceState {
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool tw_ready = false;
};

std::mutex g_mutex;
DeviceState g_dev[kMaxDevices];

// Entry j holds e^{+2 pi i e / SWENSE_MAX_FFT}, e = twiddle_exponent(j): the plain table, then the
// pass-major tables (layout at stk_twp). Computed in FP64 with sincospi (exact argument scaling)
// and rounded once, so each pass-major entry equals the plain entry of the same e bit for bit.
__device__ float2 g_twiddle[kTwiddleLen];

__global__ void k_fill_twiddles() {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kTwiddleLen) return;
  const int e = twiddle_exponent(j);
  double s, c;
  sincospi(2.0 * double(e) / double(SWENSE_MAX_FFT), &s, &c);
  g_twiddle[j] = make_float2(float(c), float(s));
}

int current_device(int* dev) {
  SWENSE_CUDA_TRY(cudaGetDevice(dev));
  if (*dev < 0 || *dev >= kMaxDevices) return fail(SWENSE_ERR_UNSUPPORTED, "device index too large");
  return SWENSE_OK;
}

}  // namespace

int workspace(size_t bytes, cudaStream_t stream, void** out) {
  int dev;
  int st = current_device(&dev);
  if (st) return st;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& d = g_dev[dev];
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes <= d.ws_bytes) {
    *out = d.ws;
    return SWENSE_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SWENSE_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(SWENSE_ERR_ARG, "scratch workspace must grow, which is not allowed during stream "
                                "capture; make one call with the same sizes before capturing");
  if (d.ws) {
    SWENSE_CUDA_TRY(cudaDeviceSynchronize());
    SWENSE_CUDA_TRY(cudaFree(d.ws));
    d.ws = nullptr;
    d.ws_bytes = 0;
  }
  size_t want = bytes + bytes / 4;  // headroom so small growth does not reallocate
  cudaError_t e = cudaMalloc(&d.ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    d.ws = nullptr;
    return fail(SWENSE_ERR_OOM, "cudaMalloc of the scratch workspace (" + std::to_string(want) +
                                    " bytes) failed: " + cudaGetErrorString(e));
  }
  d.ws_bytes = want;
  *out = d.ws;
  return SWENSE_OK;
}

int twiddles(cudaStream_t stream, const float2** out) {
  int dev;
  int st = current_device(&dev);
  if (st) return st;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_dev[dev].tw_ready) {
      // Filled once per device and waited for, so that every later stream sees it.
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      SWENSE_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
      if (cap != cudaStreamCaptureStatusNone)
        return fail(SWENSE_ERR_ARG, "the first call on a device must not be inside a stream "
                                    "capture (it fills the twiddle table)");
      k_fill_twiddles<<<(kTwiddleLen + 255) / 256, 256, 0, stream>>>();
      SWENSE_CUDA_TRY(cudaGetLastError());
      count_launches(1);
      SWENSE_CUDA_TRY(cudaStreamSynchronize(stream));
      g_dev[dev].tw_ready = true;
    }
  }
  void* p = nullptr;
  SWENSE_CUDA_TRY(cudaGetSymbolAddress(&p, g_twiddle));
  *out = static_cast<const float2*>(p);
  return SWENSE_OK;
}

}  // namespace swense

extern "C" {

int64_t swense_workspace_bytes(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= swense::kMaxDevices) return 0;
  std::lock_guard<std::mutex> lock(swense::g_mutex);
  return int64_t(swense::g_dev[dev].ws_bytes);
}

int swense_release(void) {
  int dev = 0;
  SWENSE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= swense::kMaxDevices) return SWENSE_OK;
  std::lock_guard<std::mutex> lock(swense::g_mutex);
  swense::DeviceState& d = swense::g_dev[dev];
  if (d.ws) {
    SWENSE_CUDA_TRY(cudaDeviceSynchronize());
    SWENSE_CUDA_TRY(cudaFree(d.ws));
  }
  d.ws = nullptr;
  d.ws_bytes = 0;
  return SWENSE_OK;
}

const char* swense_last_error(void) { return swense::g_last_error.c_str(); }

const char* swense_strerror(int status) {
  switch (status) {
    case SWENSE_OK: return "SWENSE_OK";
    case SWENSE_ERR_ARG: return "SWENSE_ERR_ARG";
    case SWENSE_ERR_SIZE: return "SWENSE_ERR_SIZE";
    case SWENSE_ERR_LEVELS: return "SWENSE_ERR_LEVELS";
    case SWENSE_ERR_OOM: return "SWENSE_ERR_OOM";
    case SWENSE_ERR_CUDA: return "SWENSE_ERR_CUDA";
    case SWENSE_ERR_TIMEOUT: return "SWENSE_ERR_TIMEOUT";
    case SWENSE_ERR_UNSUPPORTED: return "SWENSE_ERR_UNSUPPORTED";
    case SWENSE_ERR_CONVERGENCE: return "SWENSE_ERR_CONVERGENCE";
    default: return "SWENSE_ERR_UNKNOWN";
  }
}

int swense_async_status(int32_t reset, void* stream) {
  SWENSE_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int grid = 0, direct = 0;
  int st = swense::grid_async_flag(reset != 0, &grid);
  if (!st) st = swense::direct_async_flag(reset != 0, &direct);
  if (st) return st;
  if (grid)
    return swense::fail(SWENSE_ERR_TIMEOUT, "a bounded wait of the staged row pass (k_row_tma) gave "
                                            "up; the grid rows of that warp were not written");
  if (direct)
    return swense::fail(SWENSE_ERR_TIMEOUT, "a bounded wait of the tensor-core direct sum "
                                            "(k_direct_tc) gave up; the outputs of that tile were "
                                            "not written");
  return SWENSE_OK;
}

int swense_version(void) { return SWENSE_VERSION; }

int64_t swense_launches(void) { return swense::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
