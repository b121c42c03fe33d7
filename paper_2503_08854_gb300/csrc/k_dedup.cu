// k_dedup.cu -- duplicate suppression of ranked candidates by predicted track.
//
// A stacked search tests orbits far more densely than objects exist: every
// real detection (and every strong noise peak) is found by a whole cloud of
// neighbouring hypotheses whose tracks cross the same pixels.  A candidate is
// a duplicate when a higher-ranked candidate's predicted pixel positions lie
// within the radius r of its own at every one of a few reference exposures
// (spread over the epoch range); duplicates are dropped and the rest keep
// their rank order (a local-maximum rule in track space).
//
// Positions come from the same propagation, light time and double-float TAN
// projection as the stack (chained two-body steps through the reference
// epochs, in the stack's state arithmetic).  Neighbours are found through a hash grid over the
// positions at the first and last reference exposures (four coordinates;
// the middle one alone when n_ref = 1) with cells of size 2r: a track within
// r of candidate i lies, in each coordinate, in i's cell or in the adjacent
// cell on the side of the half that i occupies, so 2^4 buckets hold every
// possible duplicate.  The candidates are sorted by (bucket, rank) with the
// stable radix sort of the ranking, so each bucket is a run in rank order; a
// candidate scans the runs of its 16 buckets only up to its own rank and
// stops at the first better-ranked candidate within r at every reference (a
// bucket also holds the candidates of other cells that hash to it: the
// distance test sorts them out).  A candidate with an undefined position at
// some reference exposure is within r of nothing: it is kept and never
// inserted.
#include <climits>
#include <cstdint>

#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int kDedupThreads = 256;
constexpr int kScanBlock = 1024;               // compaction: flags per block

// Pixel coordinates (x, y) of a topocentric double-float vector through the
// exposure's TAN rows, as pixel_of but without the floor; false when
// cos c <= 0.
__device__ __forceinline__ bool pixel_xy_df(const ExpDev& e, const dfloat R[3], float& x, float& y) {
  const dfloat P[3] = {{e.p0_f[0], e.p0_l[0]}, {e.p0_f[1], e.p0_l[1]}, {e.p0_f[2], e.p0_l[2]}};
  const dfloat den = df_dot3(R, P);
  if (!(den.h > 1e-30f)) return false;
  const dfloat AX[3] = {{e.axc_f[0], e.axc_l[0]}, {e.axc_f[1], e.axc_l[1]}, {e.axc_f[2], e.axc_l[2]}};
  const dfloat AY[3] = {{e.ayc_f[0], e.ayc_l[0]}, {e.ayc_f[1], e.ayc_l[1]}, {e.ayc_f[2], e.ayc_l[2]}};
  const dfloat xh = df_div(df_dot3(R, AX), den);
  const dfloat yh = df_div(df_dot3(R, AY), den);
  // the rows give x + 1/2 and y + 1/2
  x = (xh.h - 0.5f) + xh.l;
  y = (yh.h - 0.5f) + yh.l;
  return true;
}

// Positions of every candidate at the reference exposures (sorted positions
// ref[0] < ref[1] < ... in epoch order): P[i * n_ref + k], NaN where the
// tangent point is 90 degrees or more away or the candidate index is out of
// range.  DFS: the double-float state (as the stack's default), else FP64.
template <bool DFS>
__global__ void __launch_bounds__(kDedupThreads)
    k_track_ref(const double* __restrict__ states, int64_t n, double t0, double t_ref,
                const int64_t* __restrict__ cand, int64_t n_cand, const ExpDev* __restrict__ ex,
                const int32_t* __restrict__ ref, int n_ref, Phys ph, float2* __restrict__ P,
                unsigned long long* counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cand) return;
  float2* out = P + i * n_ref;
  const float nan = __int_as_float(0x7fc00000);
  const int64_t o = cand[i];
  if (o < 0 || o >= n) {
    for (int k = 0; k < n_ref; ++k) out[k] = make_float2(nan, nan);
    return;
  }
  Track<DFS> w;
  w.init(ph, states, n, o, t0, t_ref);
  bool failed = false;
  for (int k = 0; k < n_ref; ++k) {
    const ExpDev& e = ex[ref[k]];
    float2 p = make_float2(nan, nan);
    if (!failed) {
      dfloat rho[3];
      if (!w.step(ph, e, rho)) {
        failed = true;
        atomicAdd(counters + 1, 1ull);
      } else {
        float x, y;
        if (pixel_xy_df(e, rho, x, y)) p = make_float2(x, y);
      }
    }
    out[k] = p;
  }
}

// Hash-grid coordinates of a candidate: the cells (size 2r) of its
// positions at the key references, and per coordinate the side (-1 or +1) of
// the neighbouring cell that a track within r can fall into.  False when a
// position at any reference is undefined (or absurdly far off the chip).
struct GridKey {
  int c[4];
  int side[4];
};

__device__ __forceinline__ bool grid_key(const float2* p, int n_ref, float inv_cell2, GridKey& g) {
  for (int k = 0; k < n_ref; ++k)
    if (!(fabsf(p[k].x) < 1e9f && fabsf(p[k].y) < 1e9f)) return false;
  // first and last references; with one reference its position, the other
  // two coordinates zero (one cell)
  const float2 a = p[0], b = n_ref == 1 ? make_float2(0.0f, 0.0f) : p[n_ref - 1];
  const float v[4] = {a.x, a.y, b.x, b.y};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const float q = v[d] * inv_cell2;
    const float f = floorf(q);
    g.c[d] = (int)f;
    g.side[d] = q - f < 0.5f ? -1 : 1;
  }
  return true;
}

__device__ __forceinline__ uint32_t key_hash(const int c[4], uint32_t mask) {
  uint32_t h = (uint32_t)c[0] * 73856093u;
  h ^= (uint32_t)c[1] * 19349663u;
  h ^= (uint32_t)c[2] * 83492791u;
  h ^= (uint32_t)c[3] * 2654435761u;
  return (h ^ (h >> 15)) & mask;
}

// items[i] = (bucket of i's own cell) << 32 | i; candidates with an
// undefined position get the bucket past the table (sorted last, never
// scanned).
__global__ void __launch_bounds__(kDedupThreads)
    k_dedup_items(const float2* __restrict__ P, int n_cand, int n_ref, float inv_cell2, uint32_t mask,
                  unsigned long long* __restrict__ items) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cand) return;
  GridKey g;
  const uint32_t b = grid_key(P + (int64_t)i * n_ref, n_ref, inv_cell2, g) ? key_hash(g.c, mask) : mask + 1;
  items[i] = ((unsigned long long)b << 32) | (unsigned)i;
}

// Runs of the sorted items: first[b] .. last[b] (exclusive) hold bucket b.
__global__ void __launch_bounds__(kDedupThreads)
    k_dedup_runs(const unsigned long long* __restrict__ items, int n_cand, uint32_t mask,
                 int* __restrict__ first, int* __restrict__ last) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cand) return;
  const uint32_t b = (uint32_t)(items[i] >> 32);
  if (b > mask) return;
  if (i == 0 || (uint32_t)(items[i - 1] >> 32) != b) first[b] = i;
  if (i == n_cand - 1 || (uint32_t)(items[i + 1] >> 32) != b) last[b] = i + 1;
}

// keep[i] = 0 when a candidate of smaller rank (index) lies within r of i at
// every reference exposure (both positions defined), else 1.  Thread q takes
// the candidate at position q of the sorted items, so that the threads of a
// bucket's run read the same bucket bounds, run entries and leading
// neighbours (most candidates are duplicates of their bucket's first entry).
__global__ void __launch_bounds__(kDedupThreads)
    k_dedup_mark(const float2* __restrict__ P, int n_cand, int n_ref, float inv_cell2, float r2,
                 const unsigned long long* __restrict__ items, const int* __restrict__ first,
                 const int* __restrict__ last, uint32_t mask, uint8_t* __restrict__ keep) {
  const int q0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (q0 >= n_cand) return;
  const int i = (int)(unsigned)items[q0];
  const float2* pi = P + (int64_t)i * n_ref;
  GridKey g;
  bool dup = false;
  if (grid_key(pi, n_ref, inv_cell2, g)) {
    const int dims = n_ref == 1 ? 2 : 4;       // one reference: its two coordinates only
    for (int combo = 0; combo < (1 << dims) && !dup; ++combo) {
      int c[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) c[d] = g.c[d] + (((combo >> d) & 1) ? g.side[d] : 0);
      const uint32_t b = key_hash(c, mask);
      const int e = last[b];
      for (int q = first[b]; q < e && !dup; ++q) {
        const int j = (int)(unsigned)items[q];
        if (j >= i) break;                     // the run is in rank order
        const float2* pj = P + (int64_t)j * n_ref;
        bool close = true;
        for (int k = 0; k < n_ref && close; ++k) {
          const float ex = pi[k].x - pj[k].x, ey = pi[k].y - pj[k].y;
          close = ex * ex + ey * ey < r2;      // false for NaN
        }
        dup = close;
      }
    }
  }
  keep[i] = dup ? 0 : 1;
}

// Order-preserving compaction: per-block counts, one block's exclusive scan
// of the counts, then each block writes its kept indices.
__global__ void __launch_bounds__(kScanBlock) k_keep_count(const uint8_t* __restrict__ keep, int n,
                                                           int* __restrict__ counts) {
  __shared__ int warp_sum[kScanBlock / 32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int f = i < n ? keep[i] : 0;
  const int s = __reduce_add_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int t = __reduce_add_sync(0xffffffffu, warp_sum[threadIdx.x]);
    if (threadIdx.x == 0) counts[blockIdx.x] = t;
  }
}

// Exclusive scan of n_blocks counts by one block (loops in chunks of
// kScanBlock); offsets[n_blocks] = the total.
__global__ void __launch_bounds__(kScanBlock) k_keep_scan(const int* __restrict__ counts, int n_blocks,
                                                          int* __restrict__ offsets) {
  __shared__ int warp_sum[kScanBlock / 32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < n_blocks; c0 += kScanBlock) {
    const int i = c0 + threadIdx.x;
    const int v = i < n_blocks ? counts[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = warp_sum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_sum[lane] = w;
    }
    __syncthreads();
    const int incl = x + (warp > 0 ? warp_sum[warp - 1] : 0) + carry;
    if (i < n_blocks) offsets[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[n_blocks] = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_keep_write(const uint8_t* __restrict__ keep, int n,
                                                           const int* __restrict__ offsets,
                                                           const int64_t* __restrict__ cand,
                                                           int64_t* __restrict__ out) {
  __shared__ int warp_sum[kScanBlock / 32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int f = i < n ? keep[i] : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned ballot = __ballot_sync(0xffffffffu, f);
  const int before = __popc(ballot & ((1u << lane) - 1u));
  if (lane == 0) warp_sum[warp] = __popc(ballot);
  __syncthreads();
  if (warp == 0) {
    const int w = warp_sum[lane];
    int x = w;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    warp_sum[lane] = x - w;                    // exclusive
  }
  __syncthreads();
  if (f) out[offsets[blockIdx.x] + warp_sum[warp] + before] = cand[i];
}

}  // namespace

size_t dedup_scratch_bytes(int64_t n_cand, int n_ref, uint32_t table) {
  const int64_t nb = (n_cand + kScanBlock - 1) / kScanBlock;
  // eight sub-buffers, each rounded up to 256 bytes by launch_dedup
  return sizeof(float2) * n_cand * n_ref + 2 * sizeof(unsigned long long) * n_cand +
         sort_hist_bytes(n_cand) + 2 * sizeof(int) * (size_t)table + n_cand + sizeof(int) * (2 * nb + 1) +
         8 * 256;
}

uint32_t dedup_table_size(int64_t n_cand) {
  uint32_t t = 1024;
  while ((int64_t)t < 2 * n_cand && t < (1u << 26)) t <<= 1;
  return t;
}

cudaError_t launch_dedup(const double* states, int64_t n, double t0, double t_ref, bool state_df,
                         const int64_t* cand, int64_t n_cand, const ExpDev* ex, const int32_t* ref_dev,
                         int n_ref, Phys ph, float radius, void* scratch, unsigned long long* counters,
                         int64_t* out, int* n_keep_dev, cudaStream_t st) {
  if (n_cand == 0) return cudaMemsetAsync(n_keep_dev, 0, sizeof(int), st);
  const uint32_t table = dedup_table_size(n_cand);
  const int64_t nb = (n_cand + kScanBlock - 1) / kScanBlock;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  auto take = [&](size_t bytes) {
    unsigned char* q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  float2* P = reinterpret_cast<float2*>(take(sizeof(float2) * n_cand * n_ref));
  auto* items_a = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * n_cand));
  auto* items_b = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * n_cand));
  unsigned int* hist = reinterpret_cast<unsigned int*>(take(sort_hist_bytes(n_cand)));
  int* first = reinterpret_cast<int*>(take(sizeof(int) * table));
  int* last = reinterpret_cast<int*>(take(sizeof(int) * table));
  uint8_t* keep = reinterpret_cast<uint8_t*>(take(n_cand));
  int* counts = reinterpret_cast<int*>(take(sizeof(int) * nb));
  int* offsets = reinterpret_cast<int*>(take(sizeof(int) * (nb + 1)));
  const unsigned grid = (unsigned)((n_cand + kDedupThreads - 1) / kDedupThreads);
  // empty buckets: first = last = 0
  cudaError_t e = cudaMemsetAsync(first, 0, sizeof(int) * table, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(last, 0, sizeof(int) * table, st);
  if (e != cudaSuccess) return e;
  if (state_df)
    k_track_ref<true><<<grid, kDedupThreads, 0, st>>>(states, n, t0, t_ref, cand, n_cand, ex, ref_dev, n_ref,
                                                      ph, P, counters);
  else
    k_track_ref<false><<<grid, kDedupThreads, 0, st>>>(states, n, t0, t_ref, cand, n_cand, ex, ref_dev, n_ref,
                                                       ph, P, counters);
  const float inv_cell2 = 0.5f / radius;       // cells of size 2r
  const uint32_t mask = table - 1;
  k_dedup_items<<<grid, kDedupThreads, 0, st>>>(P, (int)n_cand, n_ref, inv_cell2, mask, items_a);
  int bits = 0;                                // bucket values up to mask + 1 = table
  while ((1u << bits) <= table) ++bits;
  unsigned long long* sorted = nullptr;
  if ((e = sort_items_hi32(items_a, items_b, hist, n_cand, (bits + 7) / 8, &sorted, st)) != cudaSuccess)
    return e;
  k_dedup_runs<<<grid, kDedupThreads, 0, st>>>(sorted, (int)n_cand, mask, first, last);
  k_dedup_mark<<<grid, kDedupThreads, 0, st>>>(P, (int)n_cand, n_ref, inv_cell2, radius * radius, sorted,
                                               first, last, mask, keep);
  k_keep_count<<<(unsigned)nb, kScanBlock, 0, st>>>(keep, (int)n_cand, counts);
  k_keep_scan<<<1, kScanBlock, 0, st>>>(counts, (int)nb, offsets);
  k_keep_write<<<(unsigned)nb, kScanBlock, 0, st>>>(keep, (int)n_cand, offsets, cand, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(n_keep_dev, offsets + nb, sizeof(int), cudaMemcpyDeviceToDevice, st);
}

}  // namespace ndt
