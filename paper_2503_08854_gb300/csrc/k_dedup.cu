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
// projection as the stack (chained universal-variable steps through the
// reference epochs).  Neighbours are found through a hash grid of cell size
// r on the middle reference exposure: two tracks within r there lie in the
// same or adjacent cells, so every candidate scans the lists of 9 cells; a
// list holds the candidates of every cell that hashes to its bucket, and the
// distance test sorts them out.
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
  const dfloat AX[3] = {{e.ax_f[0], e.ax_l[0]}, {e.ax_f[1], e.ax_l[1]}, {e.ax_f[2], e.ax_l[2]}};
  const dfloat AY[3] = {{e.ay_f[0], e.ay_l[0]}, {e.ay_f[1], e.ay_l[1]}, {e.ay_f[2], e.ay_l[2]}};
  const dfloat xh = df_add({e.crh_h[0], e.crh_l[0]}, df_div(df_dot3(R, AX), den));
  const dfloat yh = df_add({e.crh_h[1], e.crh_l[1]}, df_div(df_dot3(R, AY), den));
  // the rows give x + 1/2 and y + 1/2
  x = (xh.h - 0.5f) + xh.l;
  y = (yh.h - 0.5f) + yh.l;
  return true;
}

// Positions of every candidate at the reference exposures (sorted positions
// ref[0] < ref[1] < ... in epoch order): P[i * n_ref + k], NaN where the
// tangent point is 90 degrees or more away or the candidate index is out of
// range.
__global__ void __launch_bounds__(kDedupThreads)
    k_track_ref(const double* __restrict__ states, int64_t n, double t0, const int64_t* __restrict__ cand,
                int64_t n_cand, const ExpDev* __restrict__ ex, const int32_t* __restrict__ ref, int n_ref,
                Phys ph, float2* __restrict__ P, unsigned long long* counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cand) return;
  float2* out = P + i * n_ref;
  const float nan = __int_as_float(0x7fc00000);
  const int64_t o = cand[i];
  if (o < 0 || o >= n) {
    for (int k = 0; k < n_ref; ++k) out[k] = make_float2(nan, nan);
    return;
  }
  double r[3], v[3];
  for (int c = 0; c < 3; ++c) {
    r[c] = states[c * n + o];
    v[c] = states[(c + 3) * n + o];
  }
  double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  double inv_r = 1.0 / rn;
  const OrbitConst oc = orbit_const(ph, r, v, inv_r);
  double t_prev = t0;
  bool failed = false;
  for (int k = 0; k < n_ref; ++k) {
    const ExpDev& e = ex[ref[k]];
    float2 p = make_float2(nan, nan);
    if (!failed) {
      if (kepler_step(ph, oc, e.t - t_prev, r, v, rn, inv_r) < 0) {
        failed = true;
        atomicAdd(counters + 1, 1ull);
      } else {
        t_prev = e.t;
        dfloat rho[3];
        apparent_rho_df(ph, r, v, inv_r, e, rho);
        float x, y;
        if (pixel_xy_df(e, rho, x, y)) p = make_float2(x, y);
      }
    }
    out[k] = p;
  }
}

__device__ __forceinline__ bool cell_of(float2 p, float inv_cell, int& cx, int& cy) {
  if (!(fabsf(p.x) < 1e9f && fabsf(p.y) < 1e9f)) return false;   // NaN or far beyond any chip
  cx = (int)floorf(p.x * inv_cell);
  cy = (int)floorf(p.y * inv_cell);
  return true;
}

__device__ __forceinline__ uint32_t cell_hash(int cx, int cy, uint32_t mask) {
  return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u) & mask;
}

// Lists of candidates per hash bucket of their middle-reference cell.
__global__ void __launch_bounds__(kDedupThreads)
    k_dedup_insert(const float2* __restrict__ P, int n_cand, int n_ref, int kmid, float inv_cell,
                   int* __restrict__ head, uint32_t mask, int* __restrict__ next) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cand) return;
  int cx, cy;
  if (!cell_of(P[(int64_t)i * n_ref + kmid], inv_cell, cx, cy)) return;
  next[i] = atomicExch(head + cell_hash(cx, cy, mask), i);
}

// keep[i] = 0 when a candidate of smaller rank (index) lies within r of i at
// every reference exposure (both positions defined), else 1.
__global__ void __launch_bounds__(kDedupThreads)
    k_dedup_mark(const float2* __restrict__ P, int n_cand, int n_ref, int kmid, float inv_cell, float r2,
                 const int* __restrict__ head, uint32_t mask, const int* __restrict__ next,
                 uint8_t* __restrict__ keep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cand) return;
  const float2* pi = P + (int64_t)i * n_ref;
  int cx, cy;
  bool dup = false;
  if (cell_of(pi[kmid], inv_cell, cx, cy)) {
    for (int dy = -1; dy <= 1 && !dup; ++dy) {
      for (int dx = -1; dx <= 1 && !dup; ++dx) {
        for (int j = head[cell_hash(cx + dx, cy + dy, mask)]; j >= 0 && !dup; j = next[j]) {
          if (j >= i) continue;
          const float2* pj = P + (int64_t)j * n_ref;
          bool close = true;
          for (int k = 0; k < n_ref && close; ++k) {
            const float ex = pi[k].x - pj[k].x, ey = pi[k].y - pj[k].y;
            close = ex * ex + ey * ey < r2;    // false for NaN
          }
          dup = close;
        }
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
  // six sub-buffers, each rounded up to 256 bytes by launch_dedup
  return sizeof(float2) * n_cand * n_ref + sizeof(int) * (table + n_cand) + n_cand +
         sizeof(int) * (2 * nb + 1) + 6 * 256;
}

uint32_t dedup_table_size(int64_t n_cand) {
  uint32_t t = 1024;
  while ((int64_t)t < 2 * n_cand && t < (1u << 30)) t <<= 1;
  return t;
}

cudaError_t launch_dedup(const double* states, int64_t n, double t0, const int64_t* cand, int64_t n_cand,
                         const ExpDev* ex, const int32_t* ref_dev, int n_ref, Phys ph, float radius,
                         void* scratch, unsigned long long* counters, int64_t* out, int* n_keep_dev,
                         cudaStream_t st) {
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
  int* head = reinterpret_cast<int*>(take(sizeof(int) * table));
  int* next = reinterpret_cast<int*>(take(sizeof(int) * n_cand));
  uint8_t* keep = reinterpret_cast<uint8_t*>(take(n_cand));
  int* counts = reinterpret_cast<int*>(take(sizeof(int) * nb));
  int* offsets = reinterpret_cast<int*>(take(sizeof(int) * (nb + 1)));
  const unsigned grid = (unsigned)((n_cand + kDedupThreads - 1) / kDedupThreads);
  cudaError_t e = cudaMemsetAsync(head, 0xff, sizeof(int) * table, st);   // -1: empty
  if (e != cudaSuccess) return e;
  k_track_ref<<<grid, kDedupThreads, 0, st>>>(states, n, t0, cand, n_cand, ex, ref_dev, n_ref, ph, P,
                                              counters);
  const int kmid = n_ref / 2;
  const float inv_cell = 1.0f / radius;
  k_dedup_insert<<<grid, kDedupThreads, 0, st>>>(P, (int)n_cand, n_ref, kmid, inv_cell, head, table - 1,
                                                 next);
  k_dedup_mark<<<grid, kDedupThreads, 0, st>>>(P, (int)n_cand, n_ref, kmid, inv_cell, radius * radius,
                                               head, table - 1, next, keep);
  k_keep_count<<<(unsigned)nb, kScanBlock, 0, st>>>(keep, (int)n_cand, counts);
  k_keep_scan<<<1, kScanBlock, 0, st>>>(counts, (int)nb, offsets);
  k_keep_write<<<(unsigned)nb, kScanBlock, 0, st>>>(keep, (int)n_cand, offsets, cand, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(n_keep_dev, offsets + nb, sizeof(int), cudaMemcpyDeviceToDevice, st);
}

}  // namespace ndt
