// k_mad.cu -- per-image noise estimate by the iterative median absolute
// deviation (paper sec. 3: each image's pixel noise variance comes from an
// iterated MAD of its pixels).
//
// Rule, per image of FP32 pixels x (S_0 = every pixel):
//   m_i = lower median of S_i (rank floor((n-1)/2)),
//   sigma_i = fl32(1.4826 * lower median of { fl32|x - m_i| : x in S_i }),
//   S_{i+1} = { x : fl32|x - m_i| <= fl32(3 sigma_i) } over every pixel,
//   stop when (m_i, sigma_i) repeats or after max_rounds; variance sigma^2.
// All membership tests and keys are FP32 operations as written, so the
// result is exact (bit for bit the same order statistics as any correct
// implementation of the rule).
//
// Selection is an exact radix select on order-preserving 32-bit keys, three
// digits of 11, 11 and 10 bits from the top.  A pass histograms, for every
// image at once, the digit of the keys that lie in S_i and match the digits
// chosen so far (a 2048-bin shared-memory histogram per CTA, merged with
// global atomics); a pick kernel (one CTA per image) scans the histogram,
// keeps the digit holding the wanted rank and clears the histogram.  A round
// is six passes (median, then MAD); S_i is never stored: it is re-derived
// from the previous round's (m, threshold) as the pixels stream by.
#include <climits>

#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int kMadBins = 2048;
constexpr int kMadThreads = 512;
constexpr int kMadChunk = 1 << 16;     // pixels per CTA and pass
constexpr float kMadToSigma = 1.4826f;
constexpr float kMadClip = 3.0f;

__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// digit d (0, 1, 2) of a key: bit offset and width
__device__ __forceinline__ int digit_shift(int d) { return d == 0 ? 21 : (d == 1 ? 10 : 0); }
__device__ __forceinline__ int digit_bits(int d) { return d == 2 ? 10 : 11; }

__global__ void __launch_bounds__(kMadThreads)
    k_mad_hist(const MadImage* __restrict__ imgs, MadState* __restrict__ st, uint32_t* __restrict__ hist,
               int digit, int what) {
  __shared__ uint32_t h[kMadBins];
  const int img = blockIdx.y;
  const MadState s = st[img];
  if (s.done) return;
  const MadImage im = imgs[img];
  const int64_t begin = (int64_t)blockIdx.x * kMadChunk;
  if (begin >= im.n) return;
  const int64_t end = begin + kMadChunk < im.n ? begin + kMadChunk : im.n;
  for (int i = threadIdx.x; i < kMadBins; i += kMadThreads) h[i] = 0;
  __syncthreads();
  const int sh = digit_shift(digit), bits = digit_bits(digit);
  const int hi_sh = sh + bits;   // bits above this digit must equal the prefix
  for (int64_t p = begin + threadIdx.x; p < end; p += kMadThreads) {
    const float x = __ldg(im.x + p);
    if (s.round > 0 && !(fabsf(__fsub_rn(x, s.m_prev)) <= s.thr_prev)) continue;
    const uint32_t key = what == 0 ? order_key(x) : order_key(fabsf(__fsub_rn(x, s.m_cur)));
    if (hi_sh < 32 && (key >> hi_sh) != s.prefix) continue;
    atomicAdd(&h[(key >> sh) & ((1u << bits) - 1u)], 1u);
  }
  __syncthreads();
  uint32_t* g = hist + (size_t)img * kMadBins;
  for (int i = threadIdx.x; i < kMadBins; i += kMadThreads)
    if (h[i]) atomicAdd(&g[i], h[i]);
}

// One CTA per image: choose the digit that holds rank krem, clear the
// histogram; after the last digit finish the median or the MAD.
__global__ void __launch_bounds__(kMadThreads)
    k_mad_pick(MadState* __restrict__ st, uint32_t* __restrict__ hist, int digit, int what, int max_rounds) {
  __shared__ unsigned long long part[kMadThreads];
  __shared__ int chosen;
  __shared__ unsigned long long before;
  const int img = blockIdx.x;
  MadState* s = st + img;
  if (s->done) return;
  uint32_t* g = hist + (size_t)img * kMadBins;
  constexpr int kPer = kMadBins / kMadThreads;     // 4 bins per thread
  unsigned long long c[kPer], tot = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    c[q] = g[threadIdx.x * kPer + q];
    tot += c[q];
  }
  part[threadIdx.x] = tot;
  __syncthreads();
  // inclusive scan of the per-thread totals (Hillis-Steele)
  for (int off = 1; off < kMadThreads; off <<= 1) {
    const unsigned long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  const unsigned long long total = part[kMadThreads - 1];
  if (digit == 0) {
    // the first digit's histogram counts all of S_i: set the wanted rank
    if (threadIdx.x == 0) {
      s->n_kept = (long long)total;
      s->krem = total ? (total - 1) / 2 : 0;
      s->prefix = 0;
    }
    __syncthreads();
  }
  const unsigned long long k = s->krem;
  if (threadIdx.x == 0) chosen = -1;
  __syncthreads();
  const unsigned long long excl = part[threadIdx.x] - tot;
  if (total > 0 && k >= excl && k < part[threadIdx.x]) {
    unsigned long long acc = excl;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (k < acc + c[q]) {
        chosen = threadIdx.x * kPer + q;
        before = acc;
        break;
      }
      acc += c[q];
    }
  }
  __syncthreads();
  for (int q = 0; q < kPer; ++q) g[threadIdx.x * kPer + q] = 0;   // ready for the next pass
  if (threadIdx.x != 0) return;
  if (total == 0 || chosen < 0) {   // empty set (non-finite image): stop with NaN
    s->m_cur = __int_as_float(0x7fc00000);
    s->sigma = __int_as_float(0x7fc00000);
    s->done = 1;
    return;
  }
  s->krem = k - before;
  s->prefix = (s->prefix << digit_bits(digit)) | (uint32_t)chosen;
  if (digit < 2) return;
  const float v = key_value(s->prefix);
  if (what == 0) {
    s->m_cur = v;
    return;
  }
  const float sigma = __fmul_rn(kMadToSigma, v);
  s->rounds = s->round + 1;
  if (s->round > 0 && s->m_cur == s->m_last && sigma == s->sigma) {
    s->done = 1;   // the rule repeats: fixed point
    return;
  }
  s->m_last = s->m_cur;
  s->sigma = sigma;
  s->m_prev = s->m_cur;
  s->thr_prev = __fmul_rn(kMadClip, sigma);
  s->round += 1;
  if (s->round >= max_rounds) s->done = 1;
}

}  // namespace

cudaError_t launch_mad_round(const MadImage* imgs, MadState* st, uint32_t* hist, int n_images,
                             int64_t max_pixels, int max_rounds, cudaStream_t stream) {
  const unsigned chunks = (unsigned)((max_pixels + kMadChunk - 1) / kMadChunk);
  if (chunks == 0 || n_images == 0) return cudaSuccess;
  const dim3 grid(chunks, (unsigned)n_images);
  for (int what = 0; what < 2; ++what)
    for (int d = 0; d < 3; ++d) {
      k_mad_hist<<<grid, kMadThreads, 0, stream>>>(imgs, st, hist, d, what);
      k_mad_pick<<<(unsigned)n_images, kMadThreads, 0, stream>>>(st, hist, d, what, max_rounds);
    }
  return cudaGetLastError();
}

size_t mad_hist_words(int n_images) { return (size_t)n_images * kMadBins; }

}  // namespace ndt
