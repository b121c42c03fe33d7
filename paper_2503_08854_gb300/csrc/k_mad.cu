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
// Selection.  Each order statistic (the median of S_i, then its MAD) is
// selected exactly on order-preserving 32-bit keys of the FP32 values, by
// passes that each stream the image once.  S_i is never stored: every pass
// re-derives it from the previous round's (m, threshold).
//  * A histogram pass counts the keys of S_i in 8192 bins of 2^shift keys
//    laid around a predicted key (the previous round's median or MAD; the
//    whole key range in round 0), plus one bin below and one above them.
//    The bin width comes from the key density the previous round found
//    near its result, so that a bin holds about cap/16 keys.
//  * The same pass copies, speculatively, every key of the few bins around
//    the prediction into a per-image buffer of `cap` keys.
//  * The pick kernel (one CTA per image) finds the bin holding the wanted
//    rank.  If it lies in the speculative bins the exact key is selected in
//    the buffer (radix select) and the selection took one pass; else a bin
//    of at most cap keys is copied out by a compaction pass and selected
//    there (two passes); a larger bin is histogrammed again at a finer width
//    (every level narrows the band 8192-fold, a single key ends it).
// Bins are monotone functions of the key and the buffer holds every key of
// the chosen bin, so the result is exact whatever the data; the prediction
// only decides how many passes it takes.  Once the estimate settles a round
// streams each image twice (median, MAD), against six times for a plain
// three-digit radix select.
#include <climits>

#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int kInner = 8192;           // inner bins of a histogram pass
constexpr int kBins = kInner + 2;      // + one below and one above the window
constexpr int kPassThreads = 512;
constexpr int kChunk4 = 1 << 15;       // float4 groups per CTA and pass (131,072 pixels)
constexpr int kUnroll = 4;
constexpr int kPickThreads = 1024;
constexpr int kDigitBins = 2048;       // radix select in the buffer: 11-bit digits
constexpr int kMaxShift = 19;          // widest bin: 2^19 keys (1/16 of a binade)
constexpr float kMadToSigma = 1.4826f;
constexpr float kMadClip = 3.0f;
constexpr int kPhaseHist = 1, kPhaseCompact = 2;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// bin of key k in a histogram pass: 0 below the window, kBins - 1 above it
__device__ __forceinline__ int bin_of(uint32_t k, uint32_t lo, int shift) {
  const uint32_t q = k < lo ? 0u : ((k - lo) >> shift) + 1u;
  return (int)min(q, (uint32_t)(kBins - 1));
}

constexpr int kStage = 256;                      // staged keys per warp
constexpr int kPassWarps = kPassThreads / 32;

// Keys a warp appends to its image's buffer, staged in shared memory so that
// one global atomic reserves room for up to kStage of them.  `n` (the same
// in every lane) counts the staged keys.
struct WarpStage {
  uint32_t* keys;   // kStage slots of this warp
  int n;
};

__device__ __forceinline__ void stage_flush(WarpStage& st, uint32_t* ib, uint32_t* ic, uint32_t cap) {
  const unsigned lane = threadIdx.x & 31u;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(ic, (uint32_t)st.n);
  base = __shfl_sync(kFull, base, 0);
  for (int i = (int)lane; i < st.n; i += 32)
    if (base + (uint32_t)i < cap) ib[base + i] = st.keys[i];
  __syncwarp();
  st.n = 0;
}

// Append the keys of `mask` (bit j: k[j]) of every lane; called by all 32
// lanes.  Positions at or beyond cap are counted but not written.
__device__ __forceinline__ void warp_append(const uint32_t (&k)[4], unsigned mask, WarpStage& st, uint32_t* ib,
                                            uint32_t* ic, uint32_t cap) {
  const unsigned lane = threadIdx.x & 31u;
  const int c = __popc(mask);
  int inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, inc, o);
    if ((int)lane >= o) inc += t;
  }
  const int total = __shfl_sync(kFull, inc, 31);
  if (st.n + total > kStage) stage_flush(st, ib, ic, cap);
  int pos = st.n + inc - c;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (mask >> j & 1u) st.keys[pos++] = k[j];
  __syncwarp();
  st.n += total;
}

// The per-pass constants of one image, in registers.
struct PassK {
  float m_prev, thr_prev, m_cur;
  uint32_t lo, blo, bspan, slo, scount;   // scount = 0: no speculative copies
  int shift;
};

// What one pass does with pixel value x: membership in S_i, the key of the
// selected quantity, a histogram count; returns whether the key goes to the
// buffer.  WHAT: 0 median, 1 MAD; HIST: histogram (else compaction); R0:
// round 0 (every pixel is in S_0); BAND: only keys in [blo, blo + bspan].
template <int WHAT, bool HIST, bool R0, bool BAND>
__device__ __forceinline__ bool classify(const PassK& p, float x, uint32_t* h, uint32_t& key) {
  if (!R0 && !(fabsf(__fsub_rn(x, p.m_prev)) <= p.thr_prev)) return false;
  key = order_key(WHAT == 0 ? x : fabsf(__fsub_rn(x, p.m_cur)));
  if (BAND && key - p.blo > p.bspan) return false;
  if (!HIST) return true;
  atomicAdd(&h[bin_of(key, p.lo, p.shift)], 1u);
  return !BAND && key - p.slo < p.scount;
}

template <int WHAT, bool HIST, bool R0, bool BAND>
__device__ __forceinline__ void pass_chunk(const PassK& p, const float* __restrict__ x, int64_t n,
                                           int64_t begin4, uint32_t* h, WarpStage& st, uint32_t* ib,
                                           uint32_t* ic, uint32_t cap) {
  // a scalar head up to the first 16-byte boundary, a float4 body, a scalar tail
  int64_t head = (int64_t)(((16u - (unsigned)(reinterpret_cast<uintptr_t>(x) & 15u)) & 15u) >> 2);
  if (head > n) head = n;
  const int64_t body4 = (n - head) >> 2;
  const int64_t tail0 = head + 4 * body4;
  const float4* __restrict__ x4 = reinterpret_cast<const float4*>(x + head);
  const int64_t end4 = begin4 + kChunk4 < body4 ? begin4 + kChunk4 : body4;
  // the trip count is the same for every thread (warp collectives inside)
  for (int64_t base = begin4; base < end4; base += (int64_t)kPassThreads * kUnroll) {
    float4 v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t q = base + (int64_t)u * kPassThreads + threadIdx.x;
      v[u] = q < end4 ? __ldcs(x4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t q = base + (int64_t)u * kPassThreads + threadIdx.x;
      uint32_t k[4] = {0u, 0u, 0u, 0u};
      unsigned mask = 0;
      if (q < end4) {
        mask |= classify<WHAT, HIST, R0, BAND>(p, v[u].x, h, k[0]) ? 1u : 0u;
        mask |= classify<WHAT, HIST, R0, BAND>(p, v[u].y, h, k[1]) ? 2u : 0u;
        mask |= classify<WHAT, HIST, R0, BAND>(p, v[u].z, h, k[2]) ? 4u : 0u;
        mask |= classify<WHAT, HIST, R0, BAND>(p, v[u].w, h, k[3]) ? 8u : 0u;
      }
      if (__any_sync(kFull, mask != 0u)) warp_append(k, mask, st, ib, ic, cap);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    // warp 0 of chunk 0 takes the scalar head and tail (at most 3 + 3 pixels)
    const int64_t n_head_tail = head + (n - tail0);
    const int64_t i = (int64_t)threadIdx.x < head ? (int64_t)threadIdx.x : tail0 + (int64_t)threadIdx.x - head;
    uint32_t k[4] = {0u, 0u, 0u, 0u};
    unsigned mask = 0;
    if ((int64_t)threadIdx.x < n_head_tail) mask = classify<WHAT, HIST, R0, BAND>(p, __ldg(x + i), h, k[0]) ? 1u : 0u;
    if (__any_sync(kFull, mask != 0u)) warp_append(k, mask, st, ib, ic, cap);
  }
}

template <int WHAT>
__device__ __forceinline__ void pass_dispatch(const MadState& s, const PassK& p, const float* x, int64_t n,
                                              int64_t begin4, uint32_t* h, WarpStage& st, uint32_t* ib,
                                              uint32_t* ic, uint32_t cap) {
  const bool r0 = s.round == 0;
  if (s.phase != kPhaseHist) {
    if (r0) pass_chunk<WHAT, false, true, true>(p, x, n, begin4, h, st, ib, ic, cap);
    else pass_chunk<WHAT, false, false, true>(p, x, n, begin4, h, st, ib, ic, cap);
  } else if (s.level == 0) {
    if (r0) pass_chunk<WHAT, true, true, false>(p, x, n, begin4, h, st, ib, ic, cap);
    else pass_chunk<WHAT, true, false, false>(p, x, n, begin4, h, st, ib, ic, cap);
  } else {
    if (r0) pass_chunk<WHAT, true, true, true>(p, x, n, begin4, h, st, ib, ic, cap);
    else pass_chunk<WHAT, true, false, true>(p, x, n, begin4, h, st, ib, ic, cap);
  }
}

// One pass over the chunk blockIdx.x of image blockIdx.y: a histogram (with
// speculative copies) or a compaction, as the image's state says.
__global__ void __launch_bounds__(kPassThreads, 3)
    k_mad_pass(const MadImage* __restrict__ imgs, const MadState* __restrict__ st, uint32_t* __restrict__ hist,
               uint32_t* __restrict__ cnt, uint32_t* __restrict__ buf, uint32_t cap) {
  __shared__ uint32_t h[kBins];
  __shared__ uint32_t stage[kPassWarps][kStage];
  const int img = blockIdx.y;
  const MadState s = st[img];
  if (s.done) return;
  const MadImage im = imgs[img];
  const int64_t begin4 = (int64_t)blockIdx.x * kChunk4;
  if (blockIdx.x != 0 && begin4 >= (im.n >> 2)) return;
  const bool hist_pass = s.phase == kPhaseHist;
  if (hist_pass) {
    for (int i = threadIdx.x; i < kBins; i += kPassThreads) h[i] = 0;
    __syncthreads();
  }
  PassK p;
  p.m_prev = s.m_prev;
  p.thr_prev = s.thr_prev;
  p.m_cur = s.m_cur;
  p.lo = s.lo;
  p.shift = s.shift;
  p.blo = s.blo;
  p.bspan = s.bhi - s.blo;
  p.slo = s.slo;
  p.scount = s.slo <= s.shi ? s.shi - s.slo + 1u : 0u;   // the range spans fewer than 2^32 keys
  WarpStage ws{stage[threadIdx.x >> 5], 0};
  uint32_t* const ib = buf + (size_t)img * cap;
  uint32_t* const ic = cnt + img;
  if (s.what == 0) pass_dispatch<0>(s, p, im.x, im.n, begin4, h, ws, ib, ic, cap);
  else pass_dispatch<1>(s, p, im.x, im.n, begin4, h, ws, ib, ic, cap);
  if (ws.n) stage_flush(ws, ib, ic, cap);   // ws.n is the same in every lane
  if (!hist_pass) return;
  __syncthreads();
  uint32_t* g = hist + (size_t)img * kBins;
  for (int i = threadIdx.x; i < kBins; i += kPassThreads)
    if (h[i]) atomicAdd(&g[i], h[i]);
}

// CTA-wide scan of counts[0..nb) (global or shared memory): the total, and
// for rank r < total the bin holding it and the number of items before it.
// When r_from_total is set the rank is floor((total - 1) / 2), the lower
// median.  Results in *out (shared), valid after the call on every thread.
struct Located {
  unsigned long long total, rank, before, count;
  int bin;
};
__device__ void locate(const uint32_t* counts, int nb, unsigned long long r, bool r_from_total, Located* out,
                       unsigned long long* warp_sums) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  const int per = (nb + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = t * per, b1 = min(b0 + per, nb);
  unsigned long long mine = 0;
  for (int b = b0; b < b1; ++b) mine += counts[b];
  unsigned long long inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < nw ? warp_sums[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += v;
    }
    if (lane < nw) warp_sums[lane] = w;   // inclusive prefix of the warp totals
  }
  __syncthreads();
  const unsigned long long excl = inc - mine + (warp > 0 ? warp_sums[warp - 1] : 0ull);
  const unsigned long long total = warp_sums[nw - 1];
  if (r_from_total) r = total ? (total - 1) / 2 : 0;
  if (t == 0) {
    out->total = total;
    out->rank = r;
    out->bin = -1;
  }
  __syncthreads();
  if (r < total && r >= excl && r < excl + mine) {
    unsigned long long acc = excl;
    for (int b = b0; b < b1; ++b) {
      const unsigned long long c = counts[b];
      if (r < acc + c) {
        out->bin = b;
        out->before = acc;
        out->count = c;
        break;
      }
      acc += c;
    }
  }
  __syncthreads();
}

// CTA-wide exact selection: the key of rank r among the keys of buf[0..n)
// that lie in [bl, bh] (11-bit digits of key - bl, from the top).
__device__ uint32_t select_in_buffer(const uint32_t* buf, uint32_t n, uint32_t bl, uint32_t bh,
                                     unsigned long long r, uint32_t* dh, Located* loc,
                                     unsigned long long* warp_sums) {
  const uint32_t span = bh - bl;
  if (span == 0) return bl;
  int pos = 32 - __clz(span);   // bits of key - bl still to decide
  uint32_t prefix = 0;
  while (pos > 0) {
    const int w = pos >= 11 ? 11 : pos, sft = pos - w;
    for (int i = threadIdx.x; i < kDigitBins; i += blockDim.x) dh[i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t k = buf[i];
      if (k < bl || k > bh) continue;
      const uint32_t d = k - bl;
      if ((uint32_t)((uint64_t)d >> pos) != prefix) continue;
      atomicAdd(&dh[(d >> sft) & ((1u << w) - 1u)], 1u);
    }
    __syncthreads();
    locate(dh, 1 << w, r, false, loc, warp_sums);
    if (loc->bin < 0) return bl;   // unreachable when the counts are consistent
    r -= loc->before;
    prefix = (prefix << w) | (uint32_t)loc->bin;
    pos = sft;
    __syncthreads();
  }
  return bl + prefix;
}

// Lay out the first histogram pass of selection `w` (0 median, 1 MAD).
__device__ void setup_selection(MadState& s, int w, uint32_t cap) {
  s.what = w;
  s.phase = kPhaseHist;
  s.level = 0;
  s.blo = 0u;
  s.bhi = 0xFFFFFFFFu;
  s.slo = 1u;
  s.shi = 0u;   // no speculative range
  const float rho = s.rho[w];
  if (s.round == 0 || !(rho > 0.0f) || !isfinite(rho)) {
    s.lo = w ? 0x80000000u : 0u;   // deviations are >= +0
    s.shift = w ? kMaxShift - 1 : kMaxShift;
    return;
  }
  const double bw = (double)cap / 16.0 / (double)rho;   // keys per bin for ~cap/16 per bin
  int sft = 0;
  while (sft < kMaxShift && (double)(1u << sft) < bw) ++sft;
  const uint64_t kp = s.kpred[w];
  const uint64_t half = (uint64_t)(kInner / 2) << sft;
  const uint64_t lo = kp > half ? kp - half : 0u;
  s.lo = (uint32_t)lo;
  s.shift = sft;
  const int bc = 1 + (int)((kp - lo) >> sft);
  double hbf = (double)cap / 8.0 / ((double)rho * (double)(1ull << sft));
  const int hb = hbf < 1.0 ? 1 : (hbf > 64.0 ? 64 : (int)hbf);
  const int b0 = max(1, bc - hb), b1 = min(kInner, bc + hb);
  const uint64_t slo = lo + ((uint64_t)(b0 - 1) << sft);
  const uint64_t shi = lo + ((uint64_t)b1 << sft) - 1u;
  if (slo > 0xFFFFFFFFull) return;
  s.slo = (uint32_t)slo;
  s.shi = shi > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)shi;
}

// A selection ended with key `key`, found in the band [bl, bh] of cb keys.
__device__ void finish_selection(MadState& s, uint32_t key, uint32_t bl, uint32_t bh, unsigned long long cb,
                                 uint32_t cap, int max_rounds) {
  const int w = s.what;
  s.rho[w] = (float)((double)cb / ((double)bh - (double)bl + 1.0));
  s.kpred[w] = key;
  const float v = key_value(key);
  if (w == 0) {
    s.m_cur = v;
    setup_selection(s, 1, cap);
    return;
  }
  const float sigma = __fmul_rn(kMadToSigma, v);
  s.rounds = s.round + 1;
  if (s.round > 0 && s.m_cur == s.m_last && sigma == s.sigma) {
    s.done = 1;   // the rule repeats: fixed point
    return;
  }
  s.m_last = s.m_cur;
  s.sigma = sigma;
  s.m_prev = s.m_cur;
  s.thr_prev = __fmul_rn(kMadClip, sigma);
  s.round += 1;
  if (s.round >= max_rounds) {
    s.done = 1;
    return;
  }
  setup_selection(s, 0, cap);
}

// One CTA per image: consume the pass that just ran and plan the next one.
__global__ void __launch_bounds__(kPickThreads)
    k_mad_pick(MadState* __restrict__ st, uint32_t* __restrict__ hist, uint32_t* __restrict__ cnt,
               const uint32_t* __restrict__ buf, uint32_t cap, int max_rounds) {
  __shared__ MadState s;
  __shared__ uint32_t dh[kDigitBins];
  __shared__ unsigned long long warp_sums[32];
  __shared__ Located loc;
  __shared__ int action;          // 0 plan only, 1 select in the buffer, 2 single key
  __shared__ uint32_t band_lo, band_hi;
  __shared__ unsigned long long band_count, band_rank;
  const int img = blockIdx.x;
  if (threadIdx.x == 0) s = st[img];
  __syncthreads();
  if (s.done) return;
  uint32_t* g = hist + (size_t)img * kBins;
  const uint32_t nc = cnt[img];
  const uint32_t* ib = buf + (size_t)img * cap;
  if (s.phase == kPhaseHist) {
    locate(g, kBins, s.krem, s.level == 0, &loc, warp_sums);
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) g[i] = 0;   // ready for the next pass
    if (threadIdx.x == 0) {
      s.passes += 1;
      action = 0;
      if (s.level == 0) s.n_kept = (long long)loc.total;
      if (loc.total == 0 || loc.bin < 0) {   // empty set (non-finite image): stop with NaN
        s.m_cur = s.m_last = s.sigma = __int_as_float(0x7fc00000);
        s.done = 1;
      } else {
        const unsigned long long r = loc.rank - loc.before;
        const int b = loc.bin;
        uint64_t bl64, bh64;
        if (b == 0) {
          bl64 = 0;
          bh64 = (uint64_t)s.lo - 1u;
        } else if (b == kBins - 1) {
          bl64 = (uint64_t)s.lo + ((uint64_t)kInner << s.shift);
          bh64 = 0xFFFFFFFFull;
        } else {
          bl64 = (uint64_t)s.lo + ((uint64_t)(b - 1) << s.shift);
          bh64 = bl64 + (1ull << s.shift) - 1u;
        }
        if (bl64 < s.blo) bl64 = s.blo;
        if (bh64 > s.bhi) bh64 = s.bhi;
        const uint32_t bl = (uint32_t)bl64, bh = (uint32_t)bh64;
        band_lo = bl;
        band_hi = bh;
        band_count = loc.count;
        band_rank = r;
        const bool spec = s.slo <= s.shi && bl >= s.slo && bh <= s.shi && nc <= cap;
        if (bl == bh) {
          action = 2;
        } else if (spec) {
          action = 1;
        } else if (loc.count <= cap) {
          s.phase = kPhaseCompact;
          s.level += 1;
          s.blo = bl;
          s.bhi = bh;
          s.krem = r;
          s.slo = 1u;
          s.shi = 0u;
        } else {
          s.phase = kPhaseHist;
          s.level += 1;
          s.blo = bl;
          s.bhi = bh;
          s.krem = r;
          s.slo = 1u;
          s.shi = 0u;
          s.lo = bl;
          int sft = 0;
          while (((bh - bl) >> sft) >= (uint32_t)kInner) ++sft;
          s.shift = sft;
        }
      }
    }
    __syncthreads();
  } else {
    if (threadIdx.x == 0) {
      s.passes += 1;
      band_lo = s.blo;
      band_hi = s.bhi;
      band_count = nc;
      band_rank = s.krem;
      action = 1;
    }
    __syncthreads();
  }
  if (action == 1) {
    const uint32_t key = select_in_buffer(ib, nc < cap ? nc : cap, band_lo, band_hi, band_rank, dh, &loc,
                                          warp_sums);
    if (threadIdx.x == 0) finish_selection(s, key, band_lo, band_hi, band_count, cap, max_rounds);
  } else if (action == 2 && threadIdx.x == 0) {
    finish_selection(s, band_lo, band_lo, band_hi, band_count, cap, max_rounds);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cnt[img] = 0u;
    st[img] = s;
  }
}

}  // namespace

MadState mad_initial_state() {
  MadState s{};
  s.phase = kPhaseHist;
  s.lo = 0u;
  s.shift = kMaxShift;
  s.blo = 0u;
  s.bhi = 0xFFFFFFFFu;
  s.slo = 1u;
  s.shi = 0u;
  return s;
}

cudaError_t launch_mad_passes(const MadImage* imgs, MadState* st, uint32_t* hist, uint32_t* cnt, uint32_t* buf,
                              uint32_t cap, int n_images, int64_t max_pixels, int max_rounds, int n_pairs,
                              cudaStream_t stream) {
  if (n_images == 0) return cudaSuccess;
  const int64_t body4 = max_pixels / 4 + 1;
  const unsigned chunks = (unsigned)((body4 + kChunk4 - 1) / kChunk4);
  const dim3 grid(chunks ? chunks : 1u, (unsigned)n_images);
  for (int i = 0; i < n_pairs; ++i) {
    k_mad_pass<<<grid, kPassThreads, 0, stream>>>(imgs, st, hist, cnt, buf, cap);
    k_mad_pick<<<(unsigned)n_images, kPickThreads, 0, stream>>>(st, hist, cnt, buf, cap, max_rounds);
  }
  return cudaGetLastError();
}

size_t mad_hist_words(int n_images) { return (size_t)n_images * kBins; }

}  // namespace ndt
