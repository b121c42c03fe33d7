// k_peak.cu -- measured issue rate of the FP64 pipe, the denominator of the
// stacking kernel's roofline.
//
// The stacking kernel is bound by FP64 instructions (DFMA, DMUL, DADD), so
// its roofline is the rate at which this GPU retires them.  A rate derived
// from unit counts and the maximum clock assumes the clock holds and the pipe
// accepts one warp instruction every cycle on every sub-partition; this
// kernel measures what the pipe actually sustains: every thread runs eight
// independent dependency chains of one FP64 operation, at full occupancy,
// so neither latency nor issue slots other than the FP64 pipe's limit it.
#include <cuda_runtime.h>

#include <cstdint>

#include "ndt.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

// op 0: a = a * m + c (DFMA); op 1: a = a * m (DMUL); op 2: a = a + c, then
// a = a - c (DADD).  m = 1 - 2^-30 and c = 2^-40 keep every chain finite and
// non-constant over any number of iterations the host asks for.
template <int OP>
__global__ void __launch_bounds__(kThreads) k_fp64_rate(double* out, int iters, double m, double c) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1.0 + (threadIdx.x + i) * 1e-9;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if (OP == 0) a[i] = fma(a[i], m, c);
        else if (OP == 1) a[i] = a[i] * m;
        else a[i] = (u & 1) ? a[i] - c : a[i] + c;
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" ndt_status ndt_measure_fp64_rate(int device, int32_t op, double* inst_per_s,
                                            double* seconds) {
  if (op < 0 || op > 2 || !inst_per_s) return NDT_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return NDT_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return NDT_EINVAL;
  int n_sms = 0;
  cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = n_sms * (2048 / kThreads);
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ndt_status st = NDT_OK;
  const int iters = 1024;
  const double m = 1.0 - 1.0 / (1u << 30), c = 1.0 / (double)(1ull << 40);
  auto launch = [&]() {
    if (op == 0) k_fp64_rate<0><<<blocks, kThreads>>>(out, iters, m, c);
    else if (op == 1) k_fp64_rate<1><<<blocks, kThreads>>>(out, iters, m, c);
    else k_fp64_rate<2><<<blocks, kThreads>>>(out, iters, m, c);
  };
  float ms = 0.0f;
  if (cudaMalloc(&out, sizeof(double) * blocks * kThreads) != cudaSuccess) {
    st = NDT_ENOMEM;
  } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = NDT_ECUDA;
  } else {
    launch();                                   // warm-up (clocks ramp, code loaded)
    cudaEventRecord(e0);
    for (int r = 0; r < 4; ++r) launch();
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f))
      st = NDT_ECUDA;
  }
  if (st == NDT_OK) {
    const double inst = 4.0 * blocks * kThreads * (double)iters * kUnroll * kChains;
    *inst_per_s = inst / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaGetLastError();
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return st;
}
