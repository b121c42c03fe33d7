// k_cnn_tc.cu -- forward pass of the vetting CNN on the 5th-generation tensor
// core (tcgen05), for scoring candidates.
//
// The two 32 -> 32 channel 5x5 layers (97 % of the network's FLOPs) are
// implicit GEMMs: rows = the 441 output pixels of a stamp (four M = 128
// tiles, the last one padded), columns = 32 output channels, K = 800 ordered
// as k = (u * 5 + v) * 32 + c, so one K-step of 16 is one (u, v) tap and half
// of the input channels.  Per CTA (one stamp at a time):
//   * both layers' weights sit in shared memory as BF16 in the canonical
//     K-major no-swizzle layout (8-row x 16-byte core matrices), 50 KB each;
//   * activations are BF16, pixel-major over the zero-padded 25 x 25 plane
//     (64 bytes per pixel), so one im2col row chunk is one 16-byte copy;
//   * four producer warps build the A operand of a K-step (4 tiles x 4 KB)
//     into a two-stage ring; one thread of a fifth warp issues four
//     tcgen05.mma (M = 128, N = 32, K = 16, BF16 x BF16 -> FP32) into four
//     TMEM accumulators and commits each stage to an mbarrier that releases
//     the ring slot; every wait is bounded and records a timeout instead of
//     hanging;
//   * the producer warps read the accumulators back with tcgen05.ld, add the
//     bias, apply ReLU, round to BF16 for the next layer or pool for the head.
// The first layer (2 -> 32 channels, K = 50) runs on the FP32 cores.
// Precision: BF16 stamps, BF16 weights of layers 2-3, BF16 activations
// between layers, FP32 accumulation.
#include <cuda_bf16.h>

#include <cstdint>

#include "ndt_internal.cuh"
#include "tc_ptx.cuh"

namespace ndt {

namespace {

constexpr int S = 21, SP = 25, NPIX = S * S, PLANE = SP * SP, CH = 32, KK = 25;
constexpr int KSTEPS = CH * KK / 16;           // 50
constexpr int MTILES = 4;                      // 4 x 128 rows >= 441 pixels
constexpr int kThreadsTC = 160;                // 4 producer/epilogue warps + 1 MMA warp
constexpr int OW1 = 0, OB1 = 1600, OW2 = 1632, OB2 = 27232, OW3 = 27264, OB3 = 52864, OWL = 52896,
              OBL = 52928;

// shared-memory map (bytes from a 1024-aligned base)
constexpr int SZ_TILE = 128 * 16 * 2;          // one 128 x 16 BF16 A tile
constexpr int SZ_STAGE = MTILES * SZ_TILE;     // 16 KB
constexpr int SZ_WL = KSTEPS * 32 * 16 * 2;    // 51,200: one layer's weights
constexpr int SZ_ACT = PLANE * CH * 2;         // 40,000: one activation plane set
constexpr int O_RING = 0;
constexpr int O_W2 = O_RING + 2 * SZ_STAGE;
constexpr int O_W3 = O_W2 + SZ_WL;
constexpr int O_ACTA = O_W3 + SZ_WL;
constexpr int O_ACTB = O_ACTA + SZ_ACT;
constexpr int round16(int b) { return (b + 15) & ~15; }
constexpr int O_X = O_ACTB + SZ_ACT;                   // FP32 [2][625]
constexpr int O_W1T = O_X + round16(2 * PLANE * 4);    // FP32 [50][32], read as float4
constexpr int O_B = O_W1T + 50 * 32 * 4;               // FP32 b1, b2, b3, wl, gap: 5 x 32
constexpr int O_BAR = O_B + 5 * 32 * 4;                // 3 mbarriers
constexpr int O_MISC = O_BAR + 3 * 8;                  // tmem slot, abort flag
constexpr int SMEM_USED = O_MISC + 16;
constexpr size_t kSmemTC = SMEM_USED + 1024;           // + alignment slack
// every region at least as aligned as its widest access
static_assert(O_RING % 1024 == 0 && O_W2 % 1024 == 0 && O_W3 % 1024 == 0, "operand alignment");
static_assert(O_ACTA % 16 == 0 && O_ACTB % 16 == 0, "uint4 access to the activation planes");
static_assert(O_X % 16 == 0 && O_W1T % 16 == 0 && O_B % 16 == 0, "float4 access");
static_assert(O_BAR % 8 == 0 && O_MISC % 4 == 0, "mbarrier / slot alignment");
static_assert(kSmemTC <= 232448, "shared memory of one CTA");

constexpr uint32_t kIdesc = tc::idesc_bf16_f32(128, 32);
constexpr uint32_t kWaitLimit = 1u << 22;

// Byte offset of (row m, k) in a K-major no-swizzle tile: core matrices of
// 8 rows x 16 bytes, 8-row groups `sbo` apart, K halves `lbo` apart.
__device__ __forceinline__ int kmajor_off(int m, int k, int lbo, int sbo) {
  return (m & 7) * 16 + (k & 7) * 2 + (m >> 3) * sbo + (k >> 3) * lbo;
}

__device__ __forceinline__ int pad_pixel(int p) { return (p / S + 2) * SP + (p % S + 2); }

// Two floats rounded to BF16 (nearest-even) and packed low | high << 16.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return (uint32_t)__bfloat16_as_ushort(h.x) | ((uint32_t)__bfloat16_as_ushort(h.y) << 16);
}

__global__ void __launch_bounds__(kThreadsTC, 1)
    k_cnn_forward_tc(const float* __restrict__ th, const __nv_bfloat16* __restrict__ x, int64_t n,
                     float* __restrict__ logits, int* __restrict__ err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = sm + O_RING;
  uint8_t* wsm[2] = {sm + O_W2, sm + O_W3};
  uint8_t* act[2] = {sm + O_ACTA, sm + O_ACTB};
  float* X = reinterpret_cast<float*>(sm + O_X);
  float* W1T = reinterpret_cast<float*>(sm + O_W1T);
  float* bias = reinterpret_cast<float*>(sm + O_B);     // b1 | b2 | b3 | wl | gap
  float* gap = bias + 4 * 32;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + O_BAR);   // empty[0], empty[1], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + O_MISC);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + O_MISC + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- one-time set-up: zero planes, stage weights, barriers, TMEM --------
  for (int i = tid; i < (2 * SZ_ACT) / 16; i += kThreadsTC)
    reinterpret_cast<uint4*>(sm + O_ACTA)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < 2 * PLANE; i += kThreadsTC) X[i] = 0.0f;
  for (int i = tid; i < 2 * CH * CH * KK; i += kThreadsTC) {
    const int L = i / (CH * CH * KK), e = i % (CH * CH * KK);
    const int o = e / (CH * KK), c = (e / KK) % CH, uv = e % KK;   // w[o][c][u][v]
    const int k = uv * CH + c, s = k >> 4, kk = k & 15;
    const float w = th[(L ? OW3 : OW2) + e];
    *reinterpret_cast<__nv_bfloat16*>(wsm[L] + s * 1024 + kmajor_off(o, kk, 512, 128)) =
        __float2bfloat16_rn(w);
  }
  for (int i = tid; i < 50 * 32; i += kThreadsTC) {   // W1T[c*25 + uv][o] = w1[o][c][uv]
    const int kin = i / 32, o = i % 32;
    W1T[i] = th[OW1 + o * 50 + kin];
  }
  if (tid < 32) {
    bias[tid] = th[OB1 + tid];
    bias[32 + tid] = th[OB2 + tid];
    bias[64 + tid] = th[OB3 + tid];
    bias[96 + tid] = th[OWL + tid];
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_init(&bar[2], 1);
    tc::fence_mbar_init();
    *abort_flag = 0;
  }
  if (warp == 4) tc::tmem_alloc(tmem_slot, 128);
  tc::fence_proxy_async_smem();
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const float bl = th[OBL];
  uint32_t gstep = 0, nlayer = 0;

  for (int64_t b = blockIdx.x; b < n; b += gridDim.x) {
    // ---- stamp into the padded FP32 input planes ----------------------------
    for (int i = tid; i < 2 * NPIX; i += kThreadsTC)
      X[(i / NPIX) * PLANE + pad_pixel(i % NPIX)] = __bfloat162float(x[b * 2 * NPIX + i]);
    __syncthreads();
    // ---- layer 1 on the FP32 cores: a1 = relu(conv(x) + b1) -> BF16 plane A --
    if (warp < 4) {
      for (int p = tid; p < NPIX; p += 128) {
        const int py = p / S, px = p % S;
        float acc[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) acc[o] = bias[o];
        for (int kin = 0; kin < 50; ++kin) {
          const int c = kin / KK, uv = kin % KK;
          const float xv = X[c * PLANE + (py + uv / 5) * SP + px + uv % 5];
          const float4* w = reinterpret_cast<const float4*>(W1T + kin * 32);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 wq = w[q];
            acc[4 * q] = fmaf(wq.x, xv, acc[4 * q]);
            acc[4 * q + 1] = fmaf(wq.y, xv, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(wq.z, xv, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(wq.w, xv, acc[4 * q + 3]);
          }
        }
        uint4* dst = reinterpret_cast<uint4*>(act[0] + pad_pixel(p) * 64);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            w[j] = pack_bf16x2(fmaxf(acc[8 * q + 2 * j], 0.0f), fmaxf(acc[8 * q + 2 * j + 1], 0.0f));
          dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    }
    __syncthreads();
    // ---- layers 2 and 3 on the tensor core ----------------------------------
    for (int L = 0; L < 2; ++L) {
      const uint8_t* in = act[L];
      if (L == 1 && tid < 32) gap[tid] = 0.0f;
      for (int s = 0; s < KSTEPS; ++s) {
        const int st = gstep & 1;
        if (warp < 4) {
          if (gstep >= 2 && !*abort_flag &&
              !tc::mbar_wait_bounded(&bar[st], ((gstep >> 1) - 1) & 1, kWaitLimit))
            *abort_flag = 1;
          const int uv = s >> 1, g = s & 1, u = uv / 5, v = uv % 5;
          uint8_t* stage = ring + st * SZ_STAGE;
          for (int ch = tid; ch < MTILES * 256; ch += 128) {
            const int t = ch >> 8, r = (ch >> 1) & 127, half = ch & 1;
            const int p = t * 128 + r;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (p < NPIX) {
              const int q = (p / S + u) * SP + (p % S + v);
              val = *reinterpret_cast<const uint4*>(in + q * 64 + g * 32 + half * 16);
            }
            *reinterpret_cast<uint4*>(stage + t * SZ_TILE + (r & 7) * 16 + (r >> 3) * 128 + half * 2048) = val;
          }
          tc::fence_proxy_async_smem();
        }
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
        if (warp == 4 && lane == 0 && !*abort_flag) {
          const uint32_t a0 = tc::smem_addr(ring + st * SZ_STAGE);
          const uint64_t bdesc = tc::smem_desc(tc::smem_addr(wsm[L] + s * 1024), 512, 128);
#pragma unroll
          for (int t = 0; t < MTILES; ++t)
            tc::mma_bf16(tmem + 32 * t, tc::smem_desc(a0 + t * SZ_TILE, 2048, 128), bdesc, kIdesc, s > 0);
          tc::mma_commit(&bar[st]);
          if (s == KSTEPS - 1) tc::mma_commit(&bar[2]);
        }
        ++gstep;
      }
      // ---- epilogue: TMEM -> bias, ReLU -> next plane or pooled features ----
      if (warp < 4) {
        if (!*abort_flag && !tc::mbar_wait_bounded(&bar[2], nlayer & 1, kWaitLimit)) *abort_flag = 1;
        tc::tc_fence_after_sync();
        const float* bl_ = bias + 32 * (L + 1);
        float pool[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) pool[o] = 0.0f;
        for (int t = 0; t < MTILES; ++t) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32 * t, v);
          const int p = t * 128 + warp * 32 + lane;
          if (p >= NPIX) continue;
          if (L == 0) {
            uint4* dst = reinterpret_cast<uint4*>(act[1] + pad_pixel(p) * 64);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint32_t w[4];
#pragma unroll
              for (int j = 0; j < 4; ++j)
                w[j] = pack_bf16x2(fmaxf(v[8 * q + 2 * j] + bl_[8 * q + 2 * j], 0.0f),
                                   fmaxf(v[8 * q + 2 * j + 1] + bl_[8 * q + 2 * j + 1], 0.0f));
              dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
            }
          } else {
#pragma unroll
            for (int o = 0; o < 32; ++o) pool[o] += fmaxf(v[o] + bl_[o], 0.0f);
          }
        }
        if (L == 1) {
#pragma unroll
          for (int o = 0; o < 32; ++o) {
            float s2 = pool[o];
            for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
            if (lane == 0) atomicAdd(&gap[o], s2);
          }
        }
      }
      ++nlayer;
      tc::tc_fence_before_sync();
      __syncthreads();
      tc::tc_fence_after_sync();
    }
    // ---- head: logit = wl . mean(a3) + bl ----------------------------------
    if (tid < 32) {
      float z = gap[tid] * (1.0f / NPIX) * bias[96 + tid];
      for (int off = 16; off > 0; off >>= 1) z += __shfl_xor_sync(0xffffffffu, z, off);
      if (tid == 0) logits[b] = *abort_flag ? __int_as_float(0x7fc00000) : z + bl;
    }
    __syncthreads();
  }
  // ---- teardown: every MMA of this CTA has completed before TMEM is freed ----
  if (warp == 4) {
    if (lane == 0) {
      tc::mma_commit(&bar[2]);
      if (!tc::mbar_wait_bounded(&bar[2], nlayer & 1, kWaitLimit)) *abort_flag = 1;
    }
    __syncwarp();
    tc::tc_fence_after_sync();
    tc::tmem_dealloc(tmem, 128);
  }
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(err, 1);
}

}  // namespace

size_t cnn_tc_smem_bytes() { return kSmemTC; }

cudaError_t launch_cnn_forward_tc(const float* th, const __nv_bfloat16* x, int64_t n, float* logits,
                                  int* err, int n_sms, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_cnn_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmemTC);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(n < n_sms ? n : n_sms);
  k_cnn_forward_tc<<<blocks, kThreadsTC, kSmemTC, st>>>(th, x, n, logits, err);
  return cudaGetLastError();
}

}  // namespace ndt
