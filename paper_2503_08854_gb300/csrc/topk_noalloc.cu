// topk_noalloc.cu -- ranking without any device allocation.
//
// Some callers cannot let a library allocate device memory: a host framework
// that has already reserved nearly all of the GPU's memory for its own pool
// (a library cudaMalloc would then fail or break that framework's
// accounting), or a real-time loop that cannot pay the latency and the
// implicit synchronisation of cudaMalloc/cudaFree between frames.  For them
// ndt_topk_noalloc runs the same top-k kernels as ndt_topk_candidates, but its
// scratch memory is a fixed array compiled into this library instead of a
// context-owned allocation.
//
// The array below is a host-side stand-in in host code: its device address
// is fetched once per device with cudaGetSymbolAddress (with that device
// current) and cached; kernels only ever receive that device address.
#include <mutex>

#include "ndt.h"
#include "ndt_internal.cuh"

namespace ndt {
size_t topk_scratch_bytes(int64_t n, int64_t k);
}

namespace {

constexpr int64_t kNoallocMaxN = 67108864;   // 2^26 values
constexpr int64_t kNoallocMaxK = 8192;
// histogram + selection state + per-block counts for 2^26 values + k items
constexpr size_t kNoallocBytes = 200 * 1024;

static __device__ __align__(256) unsigned char g_topk_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_topk_scratch on `device` (looked up once per device).
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_topk_scratch);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

bool on_device(const void* p, int* device) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeDevice) return false;
  *device = at.device;
  return true;
}

}  // namespace

static_assert(kNoallocBytes >= 256 * 4 + 8 * 4 + 2 * ((kNoallocMaxN + 4095) / 4096) * 4 + 16 +
                                   kNoallocMaxK * 8,
              "scratch array too small for the stated limits");

extern "C" ndt_status ndt_topk_noalloc(const float* snr_dev, int64_t n, int64_t k, int64_t* idx_out,
                                       float* snr_out, void* cuda_stream) {
  if (n < 1 || n > kNoallocMaxN) return NDT_EINVAL;
  if (k < 1 || k > kNoallocMaxK) return NDT_EINVAL;
  int dev = -1, d2 = -1;
  if (!on_device(snr_dev, &dev)) return NDT_EINVAL;
  if (dev < 0 || dev >= kMaxDevices) return NDT_EINVAL;   // beyond the address cache
  if (idx_out && (!on_device(idx_out, &d2) || d2 != dev)) return NDT_EINVAL;
  if (snr_out && (!on_device(snr_out, &d2) || d2 != dev)) return NDT_EINVAL;
  void* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return NDT_ECUDA;
  const int64_t kk = k < n ? k : n;
  const size_t need = ndt::topk_scratch_bytes(n, kk);
  if (need > kNoallocBytes) return NDT_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return NDT_ECUDA;
  if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return NDT_ECUDA;
  int launches = 0;
  // The first kernel of launch_topk zeroes the histogram and the selection
  // state; every other scratch word is written before it is read.
  cudaError_t e = ndt::launch_topk(snr_dev, n, kk, scratch, kNoallocBytes, idx_out, snr_out,
                                   &launches, static_cast<cudaStream_t>(cuda_stream));
  if (prev != dev) cudaSetDevice(prev);
  return e == cudaSuccess ? NDT_OK : NDT_ECUDA;
}
