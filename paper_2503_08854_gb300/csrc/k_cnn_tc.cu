// k_cnn_tc.cu -- forward pass of the vetting CNN on the 5th-generation tensor
// core (tcgen05), for scoring candidates.
//
// All three 5x5 convolutions are implicit GEMMs whose A operand the tensor
// core reads straight out of the activation planes; no im2col copy is made.
//
//   * Outputs are computed on the padded 25-wide row grid: output m = py * 25
//     + px (py < 21; px < 25, of which px >= 21 are discarded), so the input
//     pixel under tap (u, v) is q = m + u * 25 + v, a pure shift.  Five M = 128
//     tiles cover m < 640 (525 rows carry the 441 outputs).
//   * Activations are BF16 and chunk-major: for each group of 8 channels a
//     plane of 768 pixels x 16 bytes (the zero-padded 25 x 25 stamp plus a
//     zero tail that only discarded rows read).  Eight consecutive pixels of
//     one chunk are then one 128-byte core matrix of the canonical K-major
//     no-swizzle layout, so the A descriptor of a K-step is the plane address
//     shifted by the tap's offset: SBO = 128 bytes (next 8 rows), LBO = the
//     distance to the K-step's second 8-wide K chunk.
//   * Layers 2 and 3: K = 800 ordered k = (u * 5 + v) * 32 + c, one K-step of
//     16 = one tap x 16 channels (two chunk planes, LBO = one plane).
//     Layer 1: the 2 input channels sit in an 8-channel chunk (6 zero
//     channels), K-step s pairs taps 2s and 2s+1 (LBO = their pixel distance
//     x 16 bytes), 13 steps with a zero-weight 26th tap.
//   * The weights of all three layers sit in shared memory as BF16 B
//     operands (N = 32 output channels x 16 K per step, 1 KB per step).
//   * Lane 0 of warp t issues the MMAs of tile t (13 or 50 K-steps, M = 128,
//     N = 32, K = 16, BF16 x BF16 -> FP32 in TMEM) back to back and commits
//     them to the layer's mbarrier (five issuers: a single thread's issue
//     rate, not the tensor core, would bound these small MMAs); four warps
//     then read the accumulators with
//     tcgen05.ld, add the bias, apply ReLU and write the next layer's BF16
//     chunk planes (or pool, after layer 3, by a warp transpose-reduce into
//     per-warp channel sums).  Every wait is bounded and records a timeout
//     instead of hanging.
// Precision: BF16 stamps, BF16 weights, BF16 activations between layers,
// FP32 accumulation; pooling, head and bias in FP32.
#include <cuda_bf16.h>

#include <cstdint>

#include "ndt_internal.cuh"
#include "tc_ptx.cuh"

namespace ndt {

namespace {

constexpr int S = 21, SP = 25, NPIX = S * S, CH = 32, KK = 25;
constexpr int OW1 = 0, OB1 = 1600, OW2 = 1632, OB2 = 27232, OW3 = 27264, OB3 = 52864, OWL = 52896,
              OBL = 52928;
constexpr int MTILES = 5;                      // 5 x 128 rows >= 525 = 21 x 25
constexpr int NPP = 768;                       // pixels per chunk plane
constexpr int KS1 = 13;                        // layer-1 K-steps (26 tap slots)
constexpr int KS2 = CH * KK / 16;              // 50 K-steps of layers 2 and 3
constexpr int kThreadsTC = 160;                // 5 warps: MMA issue per tile, 4 do the epilogue
constexpr uint32_t kTmemCols = 256;            // 5 x 32 accumulator columns, power of 2

// shared-memory map (bytes from a 128-aligned base)
constexpr int CHB = NPP * 16;                  // one chunk plane, 12,288 B
constexpr int O_IN = 0;                        // layer-1 input: one chunk plane
constexpr int O_ACT0 = O_IN + CHB;             // layer-1 output: 4 chunk planes
constexpr int O_ACT1 = O_ACT0 + 4 * CHB;       // layer-2 output: 4 chunk planes
constexpr int O_W1 = O_ACT1 + 4 * CHB;         // 13 K-steps x 1 KB
constexpr int O_W2 = O_W1 + KS1 * 1024;        // 50 K-steps x 1 KB
constexpr int O_W3 = O_W2 + KS2 * 1024;
constexpr int O_B = O_W3 + KS2 * 1024;         // FP32 b1 | b2 | b3 | wl: 4 x 32, pooled: 4 warps x 32
constexpr int O_BAR = O_B + 8 * 32 * 4;        // one mbarrier (layer done)
constexpr int O_MISC = O_BAR + 8;              // tmem slot, abort flag
constexpr int SMEM_USED = O_MISC + 16;
constexpr size_t kSmemTC = SMEM_USED + 128;    // + base alignment slack
static_assert(O_IN % 128 == 0 && O_ACT0 % 128 == 0 && O_ACT1 % 128 == 0, "operand alignment");
static_assert(O_W1 % 1024 == 0 && O_W2 % 1024 == 0 && O_W3 % 1024 == 0, "operand alignment");
static_assert(O_B % 16 == 0 && O_BAR % 8 == 0 && O_MISC % 4 == 0, "alignment");
static_assert(kSmemTC <= 232448, "shared memory of one CTA");
static_assert(CHB / 16 < (1 << 14), "LBO field");
static_assert(MTILES == kThreadsTC / 32, "warp t issues the MMAs of tile t");
// The farthest pixel a tile row reads: m <= 639 plus the largest tap shift,
// 125 pixels for the zero-weight 26th tap of layer 1 (104 for real taps).
static_assert(MTILES * 128 - 1 + 5 * SP < NPP, "chunk plane covers every shifted row");

constexpr uint32_t kIdesc = tc::idesc_bf16_f32(128, 32);
// Poll limit of every mbarrier wait: about a second with the back-off sleep
// (a layer's MMAs complete in ~20 us), after which the kernel records a
// timeout and winds down instead of hanging.
constexpr uint32_t kWaitLimit = 1u << 19;

__device__ __forceinline__ int tap_shift(int tap) { return (tap / 5) * SP + tap % 5; }

// Byte offset of (row n, k) in a 32 x 16 K-major no-swizzle B tile: core
// matrices of 8 rows x 16 bytes, 8-row groups 128 bytes apart, the two K
// halves 512 bytes apart.
__device__ __forceinline__ int b_off(int n, int k) {
  return (n & 7) * 16 + (n >> 3) * 128 + (k & 7) * 2 + (k >> 3) * 512;
}

// Two floats rounded to BF16 (nearest-even) and packed low | high << 16.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return (uint32_t)__bfloat16_as_ushort(h.x) | ((uint32_t)__bfloat16_as_ushort(h.y) << 16);
}

// Padded-plane pixel of stamp pixel (py, px).
__device__ __forceinline__ int pad_q(int py, int px) { return (py + 2) * SP + px + 2; }

__global__ void __launch_bounds__(kThreadsTC, 1)
    k_cnn_forward_tc(const float* __restrict__ th, const __nv_bfloat16* __restrict__ x, int64_t n,
                     float* __restrict__ logits, int* __restrict__ err, int withhold_first_layer) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
  uint8_t* in_plane = sm + O_IN;
  uint8_t* act[2] = {sm + O_ACT0, sm + O_ACT1};
  float* bias = reinterpret_cast<float*>(sm + O_B);        // b1 | b2 | b3 | wl
  float* pooled = bias + 4 * 32;                           // per-warp channel sums [4][32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + O_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + O_MISC);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + O_MISC + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- one-time set-up ------------------------------------------------------
  // zero the input and activation planes: borders and tails are never written
  for (int i = tid; i < (9 * CHB) / 16; i += kThreadsTC)
    reinterpret_cast<uint4*>(sm + O_IN)[i] = make_uint4(0u, 0u, 0u, 0u);
  // layer 1: step s, k = 8 * (tap - 2s) + c, weight w1[o][c][tap] for c < 2, tap < 25
  for (int i = tid; i < KS1 * 32 * 16; i += kThreadsTC) {
    const int s = i / 512, o = (i >> 4) & 31, kk = i & 15;
    const int tap = 2 * s + (kk >> 3), c = kk & 7;
    const float w = (c < 2 && tap < KK) ? th[OW1 + (o * 2 + c) * KK + tap] : 0.0f;
    *reinterpret_cast<__nv_bfloat16*>(sm + O_W1 + s * 1024 + b_off(o, kk)) = __float2bfloat16_rn(w);
  }
  // layers 2 and 3: k = (u * 5 + v) * 32 + c, weight w[o][c][u][v]
  for (int i = tid; i < 2 * CH * CH * KK; i += kThreadsTC) {
    const int L = i / (CH * CH * KK), e = i % (CH * CH * KK);
    const int o = e / (CH * KK), c = (e / KK) % CH, uv = e % KK;
    const int k = uv * CH + c;
    *reinterpret_cast<__nv_bfloat16*>(sm + (L ? O_W3 : O_W2) + (k >> 4) * 1024 + b_off(o, k & 15)) =
        __float2bfloat16_rn(th[(L ? OW3 : OW2) + e]);
  }
  if (tid < 32) {
    bias[tid] = th[OB1 + tid];
    bias[32 + tid] = th[OB2 + tid];
    bias[64 + tid] = th[OB3 + tid];
    bias[96 + tid] = th[OWL + tid];
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], MTILES);   // one commit per issuing thread and layer
    tc::fence_mbar_init();
    *abort_flag = 0;
  }
  if (warp == 4) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_proxy_async_smem();
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const float bl = th[OBL];
  uint32_t phase = 0;

  // stamp b -> channels 0 and 1 of the layer-1 input chunk (threads 0-127)
  auto load_input = [&](int64_t b) {
    const __nv_bfloat16* xs = x + b * 2 * NPIX;
    for (int p = tid; p < NPIX; p += 128) {
      const uint32_t v = (uint32_t)__bfloat16_as_ushort(xs[p]) |
                         ((uint32_t)__bfloat16_as_ushort(xs[NPIX + p]) << 16);
      *reinterpret_cast<uint32_t*>(in_plane + pad_q(p / S, p % S) * 16) = v;
    }
  };
  if (warp < 4 && blockIdx.x < n) load_input(blockIdx.x);
  tc::fence_proxy_async_smem();
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();

  for (int64_t b = blockIdx.x; b < n; b += gridDim.x) {
    for (int L = 0; L < 3; ++L) {
      // ---- MMA issue: lane 0 of warp t issues every K-step of tile t and -----
      // commits them (five issuers: one thread's issue rate would bound the
      // N = 32 MMAs well below the shared-memory operand rate)
      // (withhold_first_layer: self-test of the bounded waits; no MMA of layer
      // 1 is issued, so its wait must expire and the kernel wind down)
      if (lane == 0 && !*abort_flag && !(withhold_first_layer && L == 0)) {
        const int t = warp;
        if (L == 0) {
          const uint32_t a0 = tc::smem_addr(in_plane) + t * 128 * 16, w0 = tc::smem_addr(sm + O_W1);
#pragma unroll 1
          for (int s = 0; s < KS1; ++s) {
            const int sh0 = tap_shift(2 * s), sh1 = tap_shift(2 * s + 1);
            tc::mma_bf16(tmem + 32 * t, tc::smem_desc(a0 + sh0 * 16, (sh1 - sh0) * 16, 128),
                         tc::smem_desc(w0 + s * 1024, 512, 128), kIdesc, s > 0);
          }
        } else {
          const uint32_t a0 = tc::smem_addr(act[L - 1]) + t * 128 * 16;
          const uint32_t w0 = tc::smem_addr(sm + (L == 1 ? O_W2 : O_W3));
#pragma unroll 2
          for (int s = 0; s < KS2; ++s) {
            const int sh = tap_shift(s >> 1), g = s & 1;
            tc::mma_bf16(tmem + 32 * t, tc::smem_desc(a0 + 2 * g * CHB + sh * 16, CHB, 128),
                         tc::smem_desc(w0 + s * 1024, 512, 128), kIdesc, s > 0);
          }
        }
        tc::mma_commit(&bar[0]);
      }
      // ---- epilogue: TMEM -> bias, ReLU -> next chunk planes or the pool ----
      if (warp < 4) {
        // the input plane is read only by layer-1 MMAs: stage the next stamp
        // while layer 3 runs on the tensor core
        if (L == 2 && b + gridDim.x < n) load_input(b + gridDim.x);
        if (!*abort_flag && !tc::mbar_wait_bounded(&bar[0], phase & 1, kWaitLimit)) *abort_flag = 1;
        tc::tc_fence_after_sync();
        const float* bL = bias + 32 * L;
        float pool[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) pool[o] = 0.0f;
        for (int t = 0; t < MTILES; ++t) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32 * t, v);
          const int m = t * 128 + warp * 32 + lane;
          const int py = m / SP, px = m % SP;
          if (py >= S || px >= S) continue;
          if (L < 2) {
            uint8_t* dst = act[L] + pad_q(py, px) * 16;
#pragma unroll
            for (int c8 = 0; c8 < 4; ++c8) {
              uint32_t w[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int o = 8 * c8 + 2 * j;
                w[j] = pack_bf16x2(fmaxf(v[o] + bL[o], 0.0f), fmaxf(v[o + 1] + bL[o + 1], 0.0f));
              }
              *reinterpret_cast<uint4*>(dst + c8 * CHB) = make_uint4(w[0], w[1], w[2], w[3]);
            }
          } else {
#pragma unroll
            for (int o = 0; o < 32; ++o) pool[o] += fmaxf(v[o] + bL[o], 0.0f);
          }
        }
        if (L == 2) {
          // transpose-reduce over the warp: each round hands half of the
          // remaining channels to the partner lane, so after 16+8+4+2+1
          // shuffles lane o holds the warp's sum of channel o
#pragma unroll
          for (int h = 16; h >= 1; h >>= 1) {
            const bool upper = (lane & h) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
              const float give = upper ? pool[i] : pool[i + h];
              const float keep = upper ? pool[i + h] : pool[i];
              pool[i] = keep + __shfl_xor_sync(0xffffffffu, give, h);
            }
          }
          pooled[warp * 32 + lane] = pool[0];
        }
      }
      ++phase;
      tc::fence_proxy_async_smem();
      tc::tc_fence_before_sync();
      __syncthreads();
      tc::tc_fence_after_sync();
    }
    // ---- head: logit = wl . mean(a3) + bl -----------------------------------
    if (tid < 32) {
      const float g = (pooled[tid] + pooled[32 + tid]) + (pooled[64 + tid] + pooled[96 + tid]);
      float z = g * (1.0f / NPIX) * bias[96 + tid];
      for (int off = 16; off > 0; off >>= 1) z += __shfl_xor_sync(0xffffffffu, z, off);
      if (tid == 0) logits[b] = *abort_flag ? __int_as_float(0x7fc00000) : z + bl;
    }
  }
  // ---- teardown: every MMA of this CTA has completed before TMEM is freed ----
  // (each issuer commits once more; the phase completes when all of their
  // MMAs have, normally at once)
  if (lane == 0) tc::mma_commit(&bar[0]);
  if (tid == 0 && !tc::mbar_wait_bounded(&bar[0], phase & 1, kWaitLimit)) *abort_flag = 1;
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  if (warp == 4) tc::tmem_dealloc(tmem, kTmemCols);
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(err, 1);
}

}  // namespace

size_t cnn_tc_smem_bytes() { return kSmemTC; }

cudaError_t launch_cnn_forward_tc(const float* th, const __nv_bfloat16* x, int64_t n, float* logits,
                                  int* err, int n_sms, cudaStream_t st, int withhold_first_layer) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_cnn_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmemTC);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(n < n_sms ? n : n_sms);
  k_cnn_forward_tc<<<blocks, kThreadsTC, kSmemTC, st>>>(th, x, n, logits, err, withhold_first_layer);
  return cudaGetLastError();
}

}  // namespace ndt
