// k_topk.cu -- ranking of the stacked statistic (paper Algorithm 1,
// FindSignificantResults): the k orbits with the largest nu, ordered by nu
// descending and then by orbit index ascending.
//
// nu is mapped to a 32-bit key whose ascending order is nu's descending
// order.  A four-pass most-significant-digit radix select (8-bit digits)
// finds the k-th key T, the number of keys below it and how many keys equal
// to T are needed.  An order-preserving compaction then writes the keys
// below T in index order followed by the lowest-index keys equal to T, and a
// final sort of the k (key, index) pairs gives the ranking: a single-CTA
// bitonic sort for k <= 8192, a stable multi-block LSD radix sort above.
// Every kernel is a bounded pass; nothing waits on another block.
#include <algorithm>

#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 4096;            // items per compaction block
constexpr int kSortMax = 8192;          // single-CTA sort capacity

// Ascending key <=> descending nu; NaN ranks with -inf.
__device__ __forceinline__ unsigned int nu_key(float nu) {
  if (nu != nu) nu = -INFINITY;
  unsigned int u = __float_as_uint(nu);
  unsigned int ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ~ord;
}

__device__ __forceinline__ float key_nu(unsigned int key) {
  unsigned int ord = ~key;
  unsigned int u = (ord & 0x80000000u) ? (ord & 0x7fffffffu) : ~ord;
  return __uint_as_float(u);
}

// sel = {prefix, mask, k_remaining, n_less}
__global__ void k_select_init(unsigned int* hist, unsigned int* sel, unsigned int k) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
  if (threadIdx.x == 0) {
    sel[0] = 0u;
    sel[1] = 0u;
    sel[2] = k;
    sel[3] = 0u;
  }
}

__global__ void __launch_bounds__(kThreads) k_select_hist(const float* __restrict__ nu, int64_t n,
                                                          const unsigned int* __restrict__ sel,
                                                          int shift, unsigned int* hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += kThreads) h[i] = 0u;
  __syncthreads();
  const unsigned int prefix = sel[0], mask = sel[1];
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const unsigned int key = nu_key(__ldg(nu + i));
    if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += kThreads)
    if (h[i]) atomicAdd(hist + i, h[i]);
}

// One block of 256 threads: choose the digit holding the k_remaining-th key.
__global__ void k_select_digit(unsigned int* hist, unsigned int* sel, int shift) {
  __shared__ unsigned int scan[256];
  const int t = threadIdx.x;
  const unsigned int c = hist[t];
  scan[t] = c;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    unsigned int v = t >= off ? scan[t - off] : 0u;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  const unsigned int incl = scan[t], excl = incl - c;
  const unsigned int krem = sel[2];
  __syncthreads();
  if (c > 0 && excl < krem && krem <= incl) {
    sel[0] |= (unsigned int)t << shift;
    sel[1] |= 255u << shift;
    sel[2] = krem - excl;
    sel[3] += excl;
  }
  hist[t] = 0u;   // ready for the next pass
}

// Counts per compaction block of keys below T and equal to T.
__global__ void __launch_bounds__(kThreads) k_compact_count(const float* __restrict__ nu, int64_t n,
                                                            const unsigned int* __restrict__ sel,
                                                            unsigned int* __restrict__ counts) {
  const unsigned int T = sel[0];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  unsigned int less = 0, eq = 0;
  for (int i = threadIdx.x; i < kChunk; i += kThreads) {
    const int64_t g = base + i;
    if (g < n) {
      const unsigned int key = nu_key(__ldg(nu + g));
      less += key < T;
      eq += key == T;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    less += __shfl_xor_sync(0xffffffffu, less, off);
    eq += __shfl_xor_sync(0xffffffffu, eq, off);
  }
  __shared__ unsigned int sl[kThreads / 32], se[kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    sl[threadIdx.x >> 5] = less;
    se[threadIdx.x >> 5] = eq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int a = 0, b = 0;
    for (int w = 0; w < kThreads / 32; ++w) { a += sl[w]; b += se[w]; }
    counts[2 * blockIdx.x] = a;
    counts[2 * blockIdx.x + 1] = b;
  }
}

// Exclusive scan of the per-block counts (one block, sequential chunks).
__global__ void k_compact_scan(unsigned int* counts, int nblocks) {
  __shared__ unsigned int carry_l, carry_e;
  __shared__ unsigned int sl[1024], se[1024];
  if (threadIdx.x == 0) { carry_l = 0; carry_e = 0; }
  __syncthreads();
  for (int base = 0; base < nblocks; base += 1024) {
    const int i = base + threadIdx.x;
    const unsigned int l = i < nblocks ? counts[2 * i] : 0u;
    const unsigned int e = i < nblocks ? counts[2 * i + 1] : 0u;
    sl[threadIdx.x] = l;
    se[threadIdx.x] = e;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      unsigned int vl = threadIdx.x >= off ? sl[threadIdx.x - off] : 0u;
      unsigned int ve = threadIdx.x >= off ? se[threadIdx.x - off] : 0u;
      __syncthreads();
      sl[threadIdx.x] += vl;
      se[threadIdx.x] += ve;
      __syncthreads();
    }
    if (i < nblocks) {
      counts[2 * i] = carry_l + sl[threadIdx.x] - l;
      counts[2 * i + 1] = carry_e + se[threadIdx.x] - e;
    }
    __syncthreads();
    if (threadIdx.x == 1023) {
      carry_l += sl[1023];
      carry_e += se[1023];
    }
    __syncthreads();
  }
}

// Order-preserving scatter of the selected items as (key << 32 | index).
__global__ void __launch_bounds__(kThreads) k_compact_scatter(const float* __restrict__ nu,
                                                              int64_t n,
                                                              const unsigned int* __restrict__ sel,
                                                              const unsigned int* __restrict__ offs,
                                                              unsigned long long* __restrict__ items) {
  const unsigned int T = sel[0];
  const unsigned int need_eq = sel[2], n_less = sel[3];
  __shared__ unsigned int wl[kThreads / 32], we[kThreads / 32];
  unsigned int run_l = offs[2 * blockIdx.x], run_e = offs[2 * blockIdx.x + 1];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int lt_mask = (1u << lane) - 1u;
  for (int sub = 0; sub < kChunk; sub += kThreads) {
    const int64_t g = base + sub + threadIdx.x;
    unsigned int key = 0xffffffffu;
    bool is_l = false, is_e = false;
    if (g < n) {
      key = nu_key(__ldg(nu + g));
      is_l = key < T;
      is_e = key == T;
    }
    const unsigned int bl = __ballot_sync(0xffffffffu, is_l);
    const unsigned int be = __ballot_sync(0xffffffffu, is_e);
    if (lane == 0) { wl[warp] = __popc(bl); we[warp] = __popc(be); }
    __syncthreads();
    unsigned int pl = 0, pe = 0, tl = 0, te = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      if (w < warp) { pl += wl[w]; pe += we[w]; }
      tl += wl[w];
      te += we[w];
    }
    if (is_l) {
      const unsigned int pos = run_l + pl + __popc(bl & lt_mask);
      items[pos] = ((unsigned long long)key << 32) | (unsigned long long)(uint32_t)g;
    } else if (is_e) {
      const unsigned int r = run_e + pe + __popc(be & lt_mask);
      if (r < need_eq)
        items[n_less + r] = ((unsigned long long)key << 32) | (unsigned long long)(uint32_t)g;
    }
    run_l += tl;
    run_e += te;
    __syncthreads();
  }
}

// Bitonic sort of k <= kSortMax composite keys in shared memory, then write
// index (int64) and nu (FP32) outputs.
__global__ void __launch_bounds__(1024) k_sort_small(const unsigned long long* __restrict__ items,
                                                     int k, int64_t* idx_out, float* snr_out) {
  extern __shared__ unsigned long long s[];
  int npow = 1;
  while (npow < k) npow <<= 1;
  for (int i = threadIdx.x; i < npow; i += blockDim.x) s[i] = i < k ? items[i] : ~0ull;
  __syncthreads();
  for (int size = 2; size <= npow; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < npow; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const unsigned long long a = s[i], b = s[j];
          if ((a > b) == up) { s[i] = b; s[j] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const unsigned long long v = s[i];
    if (idx_out) idx_out[i] = (int64_t)(v & 0xffffffffull);
    if (snr_out) snr_out[i] = key_nu((unsigned int)(v >> 32));
  }
}

// ---------------------------------------------------------------------------
// Large k: stable least-significant-digit radix sort of the k compacted items
// on their 32-bit key (bits 32..63 of the composite), 8 bits per pass.  The
// compaction left equal keys in index order, so stability gives the index
// tie-break.  Per pass: block histograms (bin-major), one exclusive scan, and
// a stable scatter that ranks equal digits by position inside each block.
// ---------------------------------------------------------------------------
constexpr int kRsItems = 8192;               // items per block (32 rounds of 256)

__global__ void __launch_bounds__(kThreads) k_rs_hist(const unsigned long long* __restrict__ in,
                                                      int64_t k, int shift, int nb,
                                                      unsigned int* __restrict__ hist) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsItems;
  for (int i = threadIdx.x; i < kRsItems; i += kThreads) {
    const int64_t g = base + i;
    if (g < k) atomicAdd(&h[(unsigned)(in[g] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];   // bin-major
}

// Exclusive scan of the bin-major block histograms by one block of 1024
// threads: each warp owns one contiguous segment, read 32 consecutive counts
// at a time (coalesced); the warp totals are scanned once, then each warp
// rewrites its segment with running offsets, loading eight rounds ahead.
__global__ void __launch_bounds__(1024) k_rs_scan(unsigned int* hist, int64_t total) {
  constexpr unsigned kFull = 0xffffffffu;
  constexpr int kAhead = 8;
  __shared__ unsigned int warp_sum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = (total + 1023) / 1024 * 32;        // a multiple of 32 per warp
  const int64_t s0 = (int64_t)warp * seg, s1 = s0 + seg < total ? s0 + seg : total;
  unsigned int mine = 0u;
  for (int64_t i = s0 + lane; i < s1; i += 32) mine += hist[i];
  mine = __reduce_add_sync(kFull, mine);
  if (lane == 0) warp_sum[warp] = mine;
  __syncthreads();
  if (warp == 0) {
    const unsigned int w0 = warp_sum[lane];
    unsigned int w = w0;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    warp_sum[lane] = w - w0;                            // exclusive
  }
  __syncthreads();
  unsigned int carry = warp_sum[warp];
  for (int64_t base = s0; base < s1; base += 32 * kAhead) {
    unsigned int v[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      const int64_t i = base + u * 32 + lane;
      v[u] = i < s1 ? hist[i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      unsigned int x = v[u];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      const int64_t i = base + u * 32 + lane;
      if (i < s1) hist[i] = carry + x - v[u];
      carry += __shfl_sync(kFull, x, 31);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_rs_scatter(const unsigned long long* __restrict__ in,
                                                         unsigned long long* __restrict__ out,
                                                         int64_t k, int shift, int nb,
                                                         const unsigned int* __restrict__ offs) {
  __shared__ unsigned int run[256];          // items of each digit already placed by this block
  __shared__ unsigned int wc[kThreads / 32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  run[threadIdx.x] = offs[(int64_t)threadIdx.x * nb + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kRsItems;
  for (int r = 0; r < kRsItems; r += kThreads) {
    for (int i = threadIdx.x; i < (kThreads / 32) * 256; i += kThreads) (&wc[0][0])[i] = 0u;
    __syncthreads();
    const int64_t g = base + r + threadIdx.x;
    const bool valid = g < k;
    const unsigned long long v = valid ? in[g] : 0ull;
    const unsigned int d = valid ? (unsigned)(v >> shift) & 255u : 256u + lane;   // no peers when invalid
    const unsigned int peers = __match_any_sync(0xffffffffu, d);
    const unsigned int lower = __popc(peers & ((1u << lane) - 1u));
    if (valid && lower == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned int before = run[d] + lower;
      for (int w = 0; w < warp; ++w) before += wc[w][d];
      out[before] = v;
    }
    __syncthreads();
    {   // advance the running offsets by this round's counts
      unsigned int add = 0u;
      for (int w = 0; w < kThreads / 32; ++w) add += wc[w][threadIdx.x];
      run[threadIdx.x] += add;
    }
    __syncthreads();
  }
}

__global__ void k_unpack(const unsigned long long* __restrict__ items, int64_t k, int64_t* idx_out,
                         float* snr_out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long v = items[i];
    if (idx_out) idx_out[i] = (int64_t)(v & 0xffffffffull);
    if (snr_out) snr_out[i] = key_nu((unsigned int)(v >> 32));
  }
}

}  // namespace

// Number of orbits whose nu is at least thr (NaN never counts).
__global__ void __launch_bounds__(kThreads) k_count_ge(const float* __restrict__ nu, int64_t n, float thr,
                                                       unsigned long long* __restrict__ out) {
  unsigned int c = 0u;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    c += nu[i] >= thr ? 1u : 0u;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}

cudaError_t launch_count_ge(const float* nu, int64_t n, float thr, unsigned long long* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess || n <= 0) return e;
  const int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
  k_count_ge<<<blocks, kThreads, 0, st>>>(nu, n, thr, out);
  return cudaGetLastError();
}

cudaError_t sort_items_hi32(unsigned long long* a, unsigned long long* b, unsigned int* hist, int64_t k,
                            int passes, unsigned long long** sorted, cudaStream_t st) {
  const int nb = (int)((k + kRsItems - 1) / kRsItems);
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 32 + 8 * pass;
    k_rs_hist<<<nb, kThreads, 0, st>>>(a, k, shift, nb, hist);
    k_rs_scan<<<1, 1024, 0, st>>>(hist, (int64_t)256 * nb);
    k_rs_scatter<<<nb, kThreads, 0, st>>>(a, b, k, shift, nb, hist);
    unsigned long long* t = a;
    a = b;
    b = t;
  }
  *sorted = a;
  return cudaGetLastError();
}

size_t sort_hist_bytes(int64_t k) { return (size_t)256 * ((k + kRsItems - 1) / kRsItems) * 4; }

size_t topk_scratch_bytes(int64_t n, int64_t k) {
  const int64_t nblocks = (n + kChunk - 1) / kChunk;
  size_t b = 256 * 4 + 8 * 4;
  b += (size_t)(2 * nblocks) * 4;
  b = (b + 15) & ~(size_t)15;
  b += (size_t)(k > 0 ? k : 1) * 8;
  if (k > kSortMax) {   // radix sort: a second item buffer and the block histograms
    const int64_t nb = (k + kRsItems - 1) / kRsItems;
    b += (size_t)k * 8 + (size_t)256 * nb * 4 + 16;
  }
  return b;
}

int64_t topk_max_k() { return kSortMax; }

cudaError_t launch_topk(const float* snr, int64_t n, int64_t k, void* scratch, size_t scratch_bytes,
                        int64_t* idx_out, float* snr_out, int* launches, cudaStream_t st) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  if (k > n) k = n;
  if (n > 0xffffffffll) return cudaErrorInvalidValue;
  if (scratch_bytes < topk_scratch_bytes(n, k)) return cudaErrorInvalidValue;
  const int64_t nblocks = (n + kChunk - 1) / kChunk;
  char* p = static_cast<char*>(scratch);
  unsigned int* hist = reinterpret_cast<unsigned int*>(p);
  unsigned int* sel = hist + 256;
  unsigned int* counts = sel + 8;
  size_t off = 256 * 4 + 8 * 4 + (size_t)(2 * nblocks) * 4;
  off = (off + 15) & ~(size_t)15;
  unsigned long long* items = reinterpret_cast<unsigned long long*>(p + off);
  int L = 0;
  k_select_init<<<1, 256, 0, st>>>(hist, sel, (unsigned int)k); ++L;
  const int hblocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    k_select_hist<<<hblocks, kThreads, 0, st>>>(snr, n, sel, shift, hist); ++L;
    k_select_digit<<<1, 256, 0, st>>>(hist, sel, shift); ++L;
  }
  k_compact_count<<<(unsigned)nblocks, kThreads, 0, st>>>(snr, n, sel, counts); ++L;
  k_compact_scan<<<1, 1024, 0, st>>>(counts, (int)nblocks); ++L;
  k_compact_scatter<<<(unsigned)nblocks, kThreads, 0, st>>>(snr, n, sel, counts, items); ++L;
  if (k > kSortMax) {
    const int nb = (int)((k + kRsItems - 1) / kRsItems);
    unsigned long long* tmp = items + k;
    unsigned int* hist = reinterpret_cast<unsigned int*>(tmp + k);
    unsigned long long* a = items;
    unsigned long long* b = tmp;
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 32 + 8 * pass;
      k_rs_hist<<<nb, kThreads, 0, st>>>(a, k, shift, nb, hist); ++L;
      k_rs_scan<<<1, 1024, 0, st>>>(hist, (int64_t)256 * nb); ++L;
      k_rs_scatter<<<nb, kThreads, 0, st>>>(a, b, k, shift, nb, hist); ++L;
      unsigned long long* t = a; a = b; b = t;
    }
    // four passes: the sorted items are back in `items`
    k_unpack<<<(unsigned)std::min<int64_t>((k + 255) / 256, 4096), 256, 0, st>>>(a, k, idx_out, snr_out); ++L;
    if (launches) *launches += L;
    return cudaGetLastError();
  }
  int npow = 1;
  while (npow < k) npow <<= 1;
  const size_t smem = (size_t)npow * 8;
  cudaError_t e = cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kSortMax * 8));
  if (e != cudaSuccess) return e;
  k_sort_small<<<1, 1024, smem, st>>>(items, (int)k, idx_out, snr_out); ++L;
  if (launches) *launches += L;
  return cudaGetLastError();
}

}  // namespace ndt
