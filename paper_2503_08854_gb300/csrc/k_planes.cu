// k_planes.cu -- matched-filter planes (paper sec. 3: a matched filter for
// a Gaussian PSF, its width read from each image's header):
//   psi(p) = sum_k P(k) I(p+k) / V(p+k),   phi(p) = sum_k P(k)^2 / V(p+k),
// P the Gaussian of sigma truncated at R = ceil(4 sigma), unit sum over the
// (2R+1)^2 window, terms outside the image dropped.  The truncated Gaussian
// factorises, P = g (x) g with g the unit-sum 1-D window, so both planes are
// separable correlations (zero padding factorises too).  One CTA computes a
// strip of kTY vertically stacked 32 x 32 output tiles from a
// (32+2R) x (32 kTY+2R) input block in shared memory (taller strips share
// more of the halo) and writes each as one contiguous tile of the tile-major
// (psi, phi) plane.  The window
// weights come precomputed with the job.  FP32 planes: one pass, 4 bytes read
// (8 with a variance plane) and 8 written per pixel.  BF16 planes: one pass
// writing 4 bytes per pixel, values divided by a-priori per-exposure scales
// that are powers of two (BF16 has the FP32 exponent range, so no
// data-dependent range is needed, and the division is an exact product).
// FP16 planes: two passes, one reducing the largest |psi| and phi of each
// plane, one writing 16-bit pairs scaled so those maxima map to 2^14.
//
// Two forms of the kernel.  The TMA form (k_planes_tma) serves every
// exposure with a constant variance whose rows are 16-byte multiples: one
// CTA per strip of four 32 x 32 tiles side by side, several per SM; a
// strip's (128 + 2R) x (32 + 2R) input block arrives by one TMA tiled load
// (zero fill outside the image, no per-element address or bounds work); the
// vertical pass runs first over column pairs and the horizontal pass over
// row pairs, both with packed FP32x2 FMAs; 1/V and the BF16 scales ride on
// the weights; the strip is staged in shared memory and stored as whole
// 128-byte tile rows.  The general form (k_planes) serves per-pixel variance
// planes and rows that TMA cannot address.
#include <cudaTypedefs.h>

#include <mutex>

#include "ndt_internal.cuh"
#include "tc_ptx.cuh"

namespace ndt {

namespace {

constexpr int kThreads = 256;
// 32 x 32 tiles per CTA, stacked vertically: the BF16 planes of 200 x 4096^2
// take 15.1 ms with one tile per CTA, 11.8 ms with 2 and 11.0 ms with 4
#ifndef NDT_PLANES_TY
#define NDT_PLANES_TY 4
#endif
constexpr int kTY = NDT_PLANES_TY;

// Tile geometry for a compile-time window radius RM >= the jobs' R: the
// weights are zero-padded to 2 RM + 1 taps, which adds exact zeros in the same
// accumulation order (the planes are bit-identical to an R-tap loop) and lets
// every tap loop unroll.
template <int RM>
struct PlaneGeom {
  static constexpr int EW = kTile + 2 * RM;        // input block width
  static constexpr int EH = kTY * kTile + 2 * RM;  // input block height
  static constexpr int ES = EW + 1;                // odd row stride: conflict-free horizontal pass
  static constexpr int HS = kTile + 1;             // row stride of the horizontal results (odd)
  static constexpr int NT = 2 * RM + 1;            // taps
  static constexpr int HW = 8;                     // horizontal outputs per thread (sliding window)
  static constexpr int VH = kTY * kTile / (kThreads / kTile);   // vertical outputs per thread
  static constexpr int HDR = 112 + kTY * kTile;    // weights (2 x 40), ex (32), ey (32 kTY)
  static constexpr int SMEM_FLOATS = HDR + 2 * (EH * ES + EH * HS);
  static_assert(kTile % VH == 0, "a thread's vertical outputs lie in one tile");
};

// CTAs per job: tiles_x x (strips of kTY tile rows)
int planes_ctas_per_job_impl(int tiles_x, int tiles_y) { return tiles_x * ((tiles_y + kTY - 1) / kTY); }

// VP: the jobs carry variance planes (the API gives either one per exposure
// or none), compiled separately so that the constant-variance form issues no
// variance-plane instruction at all.
template <int MODE, int RM, bool VP>
__global__ void __launch_bounds__(kThreads) k_planes(const PlaneJob* __restrict__ jobs,
                                                     void* __restrict__ out,
                                                     unsigned int* __restrict__ absmax2) {
  using G = PlaneGeom<RM>;
  constexpr int EW = G::EW, EH = G::EH, ES = G::ES, HS = G::HS, NT = G::NT, HW = G::HW, VH = G::VH;
  static_assert((kThreads / kTile) * VH == kTY * kTile, "vertical pass: one thread per (column, strip)");
  const PlaneJob& J = jobs[blockIdx.y];
  if (J.tma) return;                           // served by the TMA form
  const int tiles_x = J.tiles_x, tiles_y = J.tiles_y, W = J.W, H = J.H;
  const int blk = blockIdx.x;
  if (blk >= tiles_x * ((tiles_y + kTY - 1) / kTY)) return;
  const int tx = blk % tiles_x, ty0 = (blk / tiles_x) * kTY;   // first tile row of the strip
  const int R = J.R;
  extern __shared__ float sm[];
  float* gw = sm;                              // NT (<= 33) zero-padded weights
  float* gw2 = sm + 40;
  float* ex = sm + 80;                         // 32: sum of g^2 inside the image along x
  float* ey = sm + 112;                        // 32 kTY: same along y
  float* in = sm + G::HDR;                     // EH rows of stride ES : I / V
  float* hor = in + EH * ES;                   // EH rows of stride HS : horizontal pass of psi
  float* inw = hor + EH * HS;                  // EH rows of stride ES : 1 / V (variance plane only)
  float* horw = inw + EH * ES;                 // EH rows of stride HS
  constexpr bool vplane = VP;
  if (threadIdx.x < NT) {
    const int k = (int)threadIdx.x - RM;
    const bool inside = k >= -R && k <= R;
    gw[threadIdx.x] = inside ? J.g[k + R] : 0.0f;
    gw2[threadIdx.x] = inside ? J.g2[k + R] : 0.0f;
  }
  const int x0 = tx * kTile - RM, y0 = ty0 * kTile - RM;
  const float inv_vc = 1.0f / J.var_c;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // input tile: rows by warps, columns by lanes, with compile-time trip
  // counts so that every load of a thread is issued before the first is used
  // (a CTA lives a few microseconds: its loads must overlap, not queue)
  constexpr int kWarps = kThreads / 32;
  constexpr int RPW = (EH + kWarps - 1) / kWarps, CPL = (EW + 31) / 32;
  float a[RPW][CPL], wv[RPW][CPL];
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = warp + kWarps * i, yy = y0 + r;
    const bool row_in = r < EH && yy >= 0 && yy < H;
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j, xx = x0 + c;
      const bool ok = row_in && c < EW && xx >= 0 && xx < W;
      const int64_t p = (int64_t)yy * W + xx;
      a[i][j] = ok ? __ldg(J.image + p) : 0.0f;
      if constexpr (VP) wv[i][j] = ok ? __ldg(J.var + p) : 0.0f;
    }
  }
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = warp + kWarps * i, yy = y0 + r;
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j, xx = x0 + c;
      if (r < EH && c < EW) {
        if constexpr (VP) {
          // outside the image a = w = 0 (zero padding of both planes)
          const bool ok = yy >= 0 && yy < H && xx >= 0 && xx < W;
          const float w = ok ? 1.0f / wv[i][j] : 0.0f;
          in[r * ES + c] = a[i][j] * w;
          inw[r * ES + c] = w;
        } else {
          in[r * ES + c] = a[i][j] * inv_vc;
        }
      }
    }
  }
  __syncthreads();
  if (!vplane && threadIdx.x < (1 + kTY) * kTile) {
    // constant variance: phi = (1/V) * (sum of g^2 inside the image along x)
    //                                * (sum of g^2 inside the image along y)
    const bool along_x = threadIdx.x < kTile;
    const int idx = along_x ? (int)threadIdx.x : (int)threadIdx.x - kTile;
    const int c = (along_x ? tx : ty0) * kTile + idx;
    const int lim = along_x ? W : H;
    float s = 0.0f;
    for (int k = 0; k < NT; ++k) {
      const int q = c + k - RM;
      if (q >= 0 && q < lim) s += gw2[k];
    }
    (along_x ? ex : ey)[idx] = s;
  }
  // the window weights, once per thread, in registers
  float gr[NT], gr2[VP ? NT : 1];
#pragma unroll
  for (int k = 0; k < NT; ++k) gr[k] = gw[k];
  if constexpr (VP) {
#pragma unroll
    for (int k = 0; k < NT; ++k) gr2[k] = gw2[k];
  }
  // horizontal pass: a thread slides a register window along HW outputs
  for (int item = threadIdx.x; item < EH * (kTile / HW); item += kThreads) {
    const int r = item / (kTile / HW), c0 = (item % (kTile / HW)) * HW;
    {
      float w[HW + 2 * RM];
      const float* row = in + r * ES + c0;
#pragma unroll
      for (int t = 0; t < HW + 2 * RM; ++t) w[t] = row[t];
      float acc[HW];
#pragma unroll
      for (int j = 0; j < HW; ++j) acc[j] = 0.0f;
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        const float g = gr[k];
#pragma unroll
        for (int j = 0; j < HW; ++j) acc[j] = fmaf(g, w[j + k], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < HW; ++j) hor[r * HS + c0 + j] = acc[j];
    }
    if constexpr (VP) {
      float w[HW + 2 * RM];
      const float* row = inw + r * ES + c0;
#pragma unroll
      for (int t = 0; t < HW + 2 * RM; ++t) w[t] = row[t];
      float acc[HW];
#pragma unroll
      for (int j = 0; j < HW; ++j) acc[j] = 0.0f;
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        const float g = gr2[k];
#pragma unroll
        for (int j = 0; j < HW; ++j) acc[j] = fmaf(g, w[j + k], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < HW; ++j) horw[r * HS + c0 + j] = acc[j];
    }
  }
  __syncthreads();
  float s0 = 1.0f, s1 = 1.0f, m0 = 0.0f, m1 = 0.0f;
  if (MODE == kPlaneStoreBF16) {
    s0 = J.s_psi;
    s1 = J.s_phi;
  } else if (MODE == kPlaneStoreF16) {
    const float a0 = __uint_as_float(absmax2[2 * blockIdx.y]);
    const float a1 = __uint_as_float(absmax2[2 * blockIdx.y + 1]);
    s0 = a0 > 0.0f ? a0 / 16384.0f : 1.0f;
    s1 = a1 > 0.0f ? a1 / 16384.0f : 1.0f;
  }
  const float is0 = 1.0f / s0, is1 = 1.0f / s1;
  // vertical pass: thread (column x, strip of VH rows)
  const int x = threadIdx.x & (kTile - 1), ys = (threadIdx.x / kTile) * VH;
  float psi[VH], phi[VH];
  {
    float v[VH + 2 * RM];
#pragma unroll
    for (int t = 0; t < VH + 2 * RM; ++t) v[t] = hor[(ys + t) * HS + x];
#pragma unroll
    for (int j = 0; j < VH; ++j) psi[j] = 0.0f;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const float g = gr[k];
#pragma unroll
      for (int j = 0; j < VH; ++j) psi[j] = fmaf(g, v[j + k], psi[j]);
    }
  }
  if constexpr (VP) {
    float v[VH + 2 * RM];
#pragma unroll
    for (int t = 0; t < VH + 2 * RM; ++t) v[t] = horw[(ys + t) * HS + x];
#pragma unroll
    for (int j = 0; j < VH; ++j) phi[j] = 0.0f;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const float g = gr2[k];
#pragma unroll
      for (int j = 0; j < VH; ++j) phi[j] = fmaf(g, v[j + k], phi[j]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < VH; ++j) phi[j] = ex[x] * ey[ys + j] * inv_vc;
  }
  // the thread's rows lie in one tile of the strip; a strip may run past the
  // last tile row of the image, whose tiles are not stored
  const int ty = ty0 + ys / kTile, y_in = ys % kTile;
  const bool tile_ok = ty < tiles_y;
  const int64_t base = J.plane_off + ((int64_t)(ty * tiles_x + tx) << (2 * kTileShift));
#pragma unroll
  for (int j = 0; j < VH; ++j) {
    const int y = y_in + j, i = (y << kTileShift) + x;
    if (!tile_ok) break;
    if (MODE == kPlaneStoreF32) {
      reinterpret_cast<float2*>(out)[base + i] = make_float2(psi[j], phi[j]);
    } else if (MODE == kPlaneAbsMax) {
      if (tx * kTile + x < W && ty * kTile + y < H) {
        m0 = fmaxf(m0, fabsf(psi[j]));
        m1 = fmaxf(m1, fabsf(phi[j]));
      }
    } else {
      // round-to-nearest-even of value / scale
      // BF16: the scales are powers of two, so value * (1/scale) is the
      // exact quotient; FP16: an IEEE division by the data-dependent scale
      const float q0 = MODE == kPlaneStoreBF16 ? psi[j] * is0 : __fdiv_rn(psi[j], s0);
      const float q1 = MODE == kPlaneStoreBF16 ? phi[j] * is1 : __fdiv_rn(phi[j], s1);
      if (MODE == kPlaneStoreBF16)
        reinterpret_cast<__nv_bfloat162*>(out)[base + i] =
            __halves2bfloat162(__float2bfloat16_rn(q0), __float2bfloat16_rn(q1));
      else
        reinterpret_cast<__half2*>(out)[base + i] = __halves2half2(__float2half_rn(q0), __float2half_rn(q1));
    }
  }
  if (MODE == kPlaneAbsMax) {
    // reduce over the CTA first: one atomic per CTA and plane
    __shared__ float red[2][kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
      m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = m0;
      red[1][threadIdx.x >> 5] = m1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kThreads / 32; ++w) {
        m0 = fmaxf(m0, red[0][w]);
        m1 = fmaxf(m1, red[1][w]);
      }
      atomicMax(absmax2 + 2 * blockIdx.y, __float_as_uint(m0));
      atomicMax(absmax2 + 2 * blockIdx.y + 1, __float_as_uint(m1));
    }
  }
}

// ---- TMA form --------------------------------------------------------------

constexpr int kStripTiles = 4;                 // 32 x 32 tiles per strip, side by side
constexpr int kSW = kStripTiles * kTile;       // strip width, px
constexpr int kVR = 8;                         // vertical pass: output rows per thread
constexpr int kHW = 8;                         // horizontal pass: outputs per thread and row
constexpr int kMS = kTile / 2 + 1;             // vertical results: column stride in float2 (odd)
constexpr int kHThreads = (kTile / 2) * (kSW / kHW);   // horizontal pass: 16 row pairs x 16
constexpr uint32_t kTmaWaitLimit = 1u << 21;   // polls of a load barrier (under a second)

template <int MODE, int RM>
struct TmaGeom {
  static constexpr int EW = kSW + 2 * RM;            // input block width (TMA box), px
  static constexpr int EH = kTile + 2 * RM;          // input block height
  static constexpr int NCP = EW / 2;                 // column pairs of the vertical pass
  static constexpr int THREADS = NCP * (kTile / kVR);
  static constexpr int MINB = RM == 8 ? 4 : 3;       // CTAs per SM (shared memory admits these)
  static constexpr uint32_t BOX_BYTES = EW * EH * 4;
  static constexpr int PXW = MODE == kPlaneStoreF32 ? 2 : 1;   // 32-bit words per stored pixel
  // staging of the finished strip: 32 rows of PXW-word pixels, row stride in
  // words a multiple of 4 (16-byte aligned rows); it reuses the input block,
  // dead after the vertical pass
  static constexpr int OS = PXW * kSW + 4;
  static constexpr int O_MID = ((BOX_BYTES > 32 * OS * 4 ? BOX_BYTES : 32 * OS * 4) + 127) / 128 * 128;
  static constexpr int O_EXS = O_MID + EW * kMS * 8; // kSW phi factors along x
  static constexpr int O_EYS = O_EXS + kSW * 4;      // kTile along y
  static constexpr int O_W = O_EYS + kTile * 4;      // weight pairs: 2 x (RM + 1) float2
  static constexpr int O_BAR = O_W + 2 * (RM + 1) * 8;
  static constexpr int SMEM = O_BAR + 8 + 128;       // barrier + base alignment slack
  static_assert(EW % 2 == 0 && EW <= 256 && EH <= 256, "TMA box");
  static_assert((RM * 4) % 16 == 0, "box x coordinate: a multiple of 16 bytes");
  static_assert(THREADS >= kHThreads + 32, "thread roles: horizontal pass + one warp for phi");
  static_assert(O_BAR % 8 == 0, "barrier alignment");
};

// Vertical results: column c, row pair rp, stored at c kMS + rp.  The
// horizontal pass's lanes 0-15 (16-31) are the 16 row pairs of one segment,
// so a half-warp reads 16 consecutive float2.

// phi factors of one strip (constant variance: phi = (1/V) (sum of g^2 over
// the taps inside the image along x) (the same along y)), from the job's
// prefix sums of g^2; lane i of one warp covers columns i, i + 32, ... and
// row i.
__device__ __forceinline__ void phi_factors(const PlaneJob& J, int tx0, int ty, float is1, float* exs,
                                            float* eys, int lane) {
  const int R = J.R;
  const float f = (1.0f / J.var_c) * is1;
#pragma unroll
  for (int q = 0; q < kSW / 32 + 1; ++q) {
    const bool along_x = q < kSW / 32;
    const int idx = along_x ? q * 32 + lane : lane;
    const int c = (along_x ? tx0 : ty) * kTile + idx;
    const int lim = along_x ? J.W : J.H;
    const int lo = max(-R, -c), hi = min(R, lim - 1 - c);
    const float e = hi >= lo ? J.pre[hi + R + 1] - J.pre[lo + R] : 0.0f;
    if (along_x) exs[idx] = e * f;
    else eys[idx] = e;
  }
}

// Vertical pass: thread (column pair cp, row block rb) slides down kVR rows
// with 2 RM + 1 taps (weights beyond the job's R are zero).
template <int RM>
__device__ __forceinline__ void vertical_pass(const unsigned char* box, const float2* wp, float2* mid,
                                              int tid) {
  constexpr int NCP = (kSW + 2 * RM) / 2;
  const int cp = tid % NCP, rb = tid / NCP;
  float2 acc[kVR];
#pragma unroll
  for (int j = 0; j < kVR; ++j) acc[j] = make_float2(0.0f, 0.0f);
  const float2* col = reinterpret_cast<const float2*>(box) + rb * kVR * NCP + cp;
#pragma unroll
  for (int t = 0; t < kVR + 2 * RM; ++t) {
    const float2 v = col[t * NCP];
#pragma unroll
    for (int j = 0; j < kVR; ++j) {
      const int k = t - j;                     // tap k - RM, taps in ascending order
      if (k >= 0 && k <= 2 * RM) acc[j] = __ffma2_rn(wp[k < RM ? RM - k : k - RM], v, acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kVR; j += 2) {
    const int rp = (rb * kVR + j) >> 1;
    mid[(2 * cp) * kMS + rp] = make_float2(acc[j].x, acc[j + 1].x);
    mid[(2 * cp + 1) * kMS + rp] = make_float2(acc[j].y, acc[j + 1].y);
  }
}

// Horizontal pass: thread (segment seg, row pair rp) slides along kHW
// outputs of rows 2 rp (h.x) and 2 rp + 1 (h.y).
template <int RM>
__device__ __forceinline__ void horizontal_pass(const float2* mid, const float2* wp, int seg, int rp,
                                                float2 (&h)[kHW]) {
  const float2* row = mid + seg * kHW * kMS + rp;
#pragma unroll
  for (int i = 0; i < kHW; ++i) h[i] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < kHW + 2 * RM; ++t) {
    const float2 v = row[t * kMS];
#pragma unroll
    for (int i = 0; i < kHW; ++i) {
      const int k = t - i;
      if (k >= 0 && k <= 2 * RM) h[i] = __ffma2_rn(wp[k < RM ? RM - k : k - RM], v, h[i]);
    }
  }
}

// One CTA per strip (grid: strips x jobs); several CTAs per SM overlap one
// another's TMA loads with their passes.
template <int MODE, int RM>
__global__ void __launch_bounds__(TmaGeom<MODE, RM>::THREADS, TmaGeom<MODE, RM>::MINB)
    k_planes_tma(const PlaneJob* __restrict__ jobs, void* __restrict__ out,
                 unsigned int* __restrict__ absmax2, unsigned int* __restrict__ err) {
  using G = TmaGeom<MODE, RM>;
  constexpr int PXW = G::PXW;
  const PlaneJob& J = jobs[blockIdx.y];
  if (J.tma != RM) {                           // general form, or a map for another box
    if (J.tma != 0 && threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(err, 1u);
    return;
  }
  if ((int)blockIdx.x >= J.n_strips) return;
  const int tiles_x = J.tiles_x, W = J.W, H = J.H;
  const int strips_x = (tiles_x + kStripTiles - 1) / kStripTiles;
  const int tx0 = ((int)blockIdx.x % strips_x) * kStripTiles, ty = (int)blockIdx.x / strips_x;
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smraw) + 127) & ~static_cast<uintptr_t>(127));
  float2* mid = reinterpret_cast<float2*>(sm + G::O_MID);    // EW columns x kMS row pairs
  float* exs = reinterpret_cast<float*>(sm + G::O_EXS);
  float* eys = reinterpret_cast<float*>(sm + G::O_EYS);
  float2* wsm = reinterpret_cast<float2*>(sm + G::O_W);      // pairs, |tap| 0..RM: vertical, horizontal
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + G::O_BAR);
  const int tid = threadIdx.x;
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();                             // the barrier is initialised before anyone waits
  if (tid == 0) {
    tc::tmap_acquire(&J.tmap);
    tc::mbar_arrive_expect_tx(bar, G::BOX_BYTES);
    tc::tma_load_2d(sm, &J.tmap, tx0 * kTile - RM, ty * kTile - RM, bar);
  }
  // while the block arrives: weight pairs and phi factors.  1/V rides on the
  // horizontal weights and on phi's x factor, and so do the BF16 scales
  // (powers of two: exact products).
  const float is1 = MODE == kPlaneStoreBF16 ? 1.0f / J.s_phi : 1.0f;
  if (tid < 2 * (RM + 1)) {
    const int d = tid % (RM + 1), R = J.R;
    const float gg = d <= R ? J.g[R + d] : 0.0f;
    const float w = tid < RM + 1 ? gg
                                 : gg * (1.0f / J.var_c) * (MODE == kPlaneStoreBF16 ? 1.0f / J.s_psi : 1.0f);
    wsm[tid] = make_float2(w, w);
  } else if (tid >= kHThreads && tid < kHThreads + 32) {
    phi_factors(J, tx0, ty, is1, exs, eys, tid & 31);
  }
  const bool arrived = tc::mbar_wait_bounded(bar, 0, kTmaWaitLimit);
  if (!__syncthreads_and(arrived)) {           // also publishes the weights and phi factors
    if (tid == 0) atomicAdd(err, 1u);
    return;
  }
  vertical_pass<RM>(sm, wsm, mid, tid);
  __syncthreads();
  float m0 = 0.0f, m1 = 0.0f;
  uint32_t* stage = reinterpret_cast<uint32_t*>(sm);         // the input block is dead now
  if (tid < kHThreads) {
    // horizontal pass: lanes 0-15 (16-31) are the row pairs of one segment
    const int rp = tid & (kTile / 2 - 1), seg = tid / (kTile / 2);
    float2 h[kHW];
    horizontal_pass<RM>(mid, wsm + RM + 1, seg, rp, h);
    float s0 = 1.0f, s1 = 1.0f;
    if (MODE == kPlaneStoreF16) {
      const float a0 = __uint_as_float(absmax2[2 * blockIdx.y]);
      const float a1 = __uint_as_float(absmax2[2 * blockIdx.y + 1]);
      s0 = a0 > 0.0f ? a0 / 16384.0f : 1.0f;
      s1 = a1 > 0.0f ? a1 / 16384.0f : 1.0f;
    }
    float ex[kHW];
#pragma unroll
    for (int i = 0; i < kHW; ++i) ex[i] = exs[seg * kHW + i];
    // epilogue: rows 2 rp (h.x) and 2 rp + 1 (h.y), columns seg kHW + i,
    // into the staging rows
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int r = 2 * rp + half;
      const float ey = eys[r];
      uint4* dst = reinterpret_cast<uint4*>(stage + r * G::OS + seg * kHW * PXW);
      constexpr int PPC = 4 / PXW;             // pixels per 16-byte chunk
#pragma unroll
      for (int q = 0; q < kHW / PPC; ++q) {
        uint32_t wds[4];
#pragma unroll
        for (int u = 0; u < PPC; ++u) {
          const int i = q * PPC + u;
          const float psi = half ? h[i].y : h[i].x;
          const float phi = ex[i] * ey;
          if (MODE == kPlaneStoreF32) {
            wds[2 * u] = __float_as_uint(psi);
            wds[2 * u + 1] = __float_as_uint(phi);
          } else if (MODE == kPlaneStoreBF16) {
            const __nv_bfloat162 bb = __floats2bfloat162_rn(psi, phi);
            wds[u] = *reinterpret_cast<const uint32_t*>(&bb);
          } else if (MODE == kPlaneStoreF16) {
            const __half2 bb = __floats2half2_rn(__fdiv_rn(psi, s0), __fdiv_rn(phi, s1));
            wds[u] = *reinterpret_cast<const uint32_t*>(&bb);
          } else if (tx0 * kTile + seg * kHW + i < W && ty * kTile + r < H) {
            m0 = fmaxf(m0, fabsf(psi));
            m1 = fmaxf(m1, phi);
          }
        }
        if (MODE != kPlaneAbsMax) dst[q] = make_uint4(wds[0], wds[1], wds[2], wds[3]);
      }
    }
  }
  if (MODE != kPlaneAbsMax) {
    __syncthreads();
    // store the staged tiles as whole rows: 16-byte chunks, a warp covering
    // 512 contiguous bytes of the tile-major plane
    constexpr int CPR = kTile * PXW / 4;       // chunks per tile row
    const int nt = min(kStripTiles, tiles_x - tx0);
    uint4* gout = reinterpret_cast<uint4*>(static_cast<uint32_t*>(out) +
                                           (J.plane_off + ((int64_t)(ty * tiles_x + tx0) << (2 * kTileShift))) * PXW);
    for (int c = tid; c < nt * kTile * CPR; c += G::THREADS) {
      const int tile = c / (kTile * CPR), r = (c / CPR) % kTile, q = c % CPR;
      gout[c] = *reinterpret_cast<const uint4*>(stage + r * G::OS + tile * kTile * PXW + 4 * q);
    }
  }
  if (MODE == kPlaneAbsMax) {
    // reduce over the CTA first: one atomic per CTA and plane
    __shared__ float red[2][(G::THREADS + 31) / 32];
    for (int o = 16; o > 0; o >>= 1) {
      m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = m0;
      red[1][tid >> 5] = m1;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < (G::THREADS + 31) / 32; ++w) {
        m0 = fmaxf(m0, red[0][w]);
        m1 = fmaxf(m1, red[1][w]);
      }
      atomicMax(absmax2 + 2 * blockIdx.y, __float_as_uint(m0));
      atomicMax(absmax2 + 2 * blockIdx.y + 1, __float_as_uint(m1));
    }
  }
}

template <int PT>
__global__ void __launch_bounds__(kThreads) k_plane_decode(const void* __restrict__ planes,
                                                           ExpDev e, float* __restrict__ psi,
                                                           float* __restrict__ phi) {
  const int64_t n = (int64_t)e.W * e.H;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const int y = (int)(i / e.W), x = (int)(i % e.W);
    const float2 v = gather_plane<PT>(planes, e, x, y);
    if (psi) psi[i] = v.x;
    if (phi) phi[i] = v.y;
  }
}

template <int MODE, int RM, bool VP>
cudaError_t launch_rm(const PlaneJob* jobs_dev, int n_jobs, int max_ctas, void* out,
                      unsigned int* absmax2, cudaStream_t st) {
  using G = PlaneGeom<RM>;
  // the variance-plane half of the buffers is only needed with variance planes
  const size_t smem = sizeof(float) * (VP ? G::SMEM_FLOATS : G::HDR + G::EH * G::ES + G::EH * G::HS);
  cudaError_t e = cudaFuncSetAttribute(k_planes<MODE, RM, VP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * G::SMEM_FLOATS));
  if (e != cudaSuccess) return e;
  dim3 grid(max_ctas, n_jobs);
  k_planes<MODE, RM, VP><<<grid, kThreads, smem, st>>>(jobs_dev, out, absmax2);
  return cudaGetLastError();
}

template <int MODE, int RM>
cudaError_t launch_tma_rm(const PlaneJob* jobs_dev, int n_jobs, int max_strips, void* out,
                          unsigned int* absmax2, unsigned int* err, cudaStream_t st) {
  using G = TmaGeom<MODE, RM>;
  cudaError_t e = cudaFuncSetAttribute(k_planes_tma<MODE, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       G::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(max_strips, n_jobs);
  k_planes_tma<MODE, RM><<<grid, G::THREADS, G::SMEM, st>>>(jobs_dev, out, absmax2, err);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(const PlaneJob* jobs_dev, const PlaneJob* jobs_host, int n_jobs, int max_R,
                        bool any_var, void* out, unsigned int* absmax2, unsigned int* err,
                        cudaStream_t st) {
  // the window radius of a launch covers the largest one among the jobs;
  // variance planes come for every exposure or for none
  int ctas_gen = 0, strips = 0;
  for (int s = 0; s < n_jobs; ++s) {
    const PlaneJob& J = jobs_host[s];
    if (J.tma) strips = std::max(strips, J.n_strips);
    else ctas_gen = std::max(ctas_gen, planes_ctas_per_job_impl(J.tiles_x, J.tiles_y));
  }
  cudaError_t e = cudaSuccess;
  const bool small = max_R <= 8;
  if (strips > 0)
    e = small ? launch_tma_rm<MODE, 8>(jobs_dev, n_jobs, strips, out, absmax2, err, st)
              : launch_tma_rm<MODE, kMaxPsfRadius>(jobs_dev, n_jobs, strips, out, absmax2, err, st);
  if (e != cudaSuccess || ctas_gen == 0) return e;
  if (small)
    return any_var ? launch_rm<MODE, 8, true>(jobs_dev, n_jobs, ctas_gen, out, absmax2, st)
                   : launch_rm<MODE, 8, false>(jobs_dev, n_jobs, ctas_gen, out, absmax2, st);
  return any_var ? launch_rm<MODE, kMaxPsfRadius, true>(jobs_dev, n_jobs, ctas_gen, out, absmax2, st)
                 : launch_rm<MODE, kMaxPsfRadius, false>(jobs_dev, n_jobs, ctas_gen, out, absmax2, st);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

}  // namespace

void plane_jobs_prepare(PlaneJob* jobs, int n_jobs, int max_R) {
  for (int s = 0; s < n_jobs; ++s) {
    PlaneJob& J = jobs[s];
    plane_job_try_tma(J, max_R);
    // prefix sums of g^2 (FP32, in tap order) for phi's edge factors
    float acc = 0.0f;
    J.pre[0] = 0.0f;
    for (int k = 0; k <= 2 * J.R; ++k) J.pre[k + 1] = (acc += J.g2[k]);
    J.n_strips = J.tma ? ((J.tiles_x + kStripTiles - 1) / kStripTiles) * J.tiles_y : 0;
  }
}

void plane_job_try_tma(PlaneJob& J, int max_R) {
  J.tma = 0;
  if (J.var || !J.image || J.W % 4 != 0 || (reinterpret_cast<uintptr_t>(J.image) & 15) != 0) return;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return;
  // the box of the launch's compile-time radius, which the largest R of all
  // jobs decides (launch_mode); J.tma records it and the kernel checks it
  const int rm = max_R <= 8 ? 8 : kMaxPsfRadius;
  const cuuint64_t dims[2] = {(cuuint64_t)J.W, (cuuint64_t)J.H};
  const cuuint64_t strides[1] = {(cuuint64_t)J.W * 4};
  const cuuint32_t box[2] = {(cuuint32_t)(kSW + 2 * rm), (cuuint32_t)(kTile + 2 * rm)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&J.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(J.image), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  J.tma = r == CUDA_SUCCESS ? rm : 0;
}

cudaError_t launch_planes(const PlaneJob* jobs_dev, const PlaneJob* jobs_host, int n_jobs, int max_R,
                          bool any_var, int mode, void* out, unsigned int* absmax2, unsigned int* err,
                          cudaStream_t st) {
  switch (mode) {
    case kPlaneStoreF32:
      return launch_mode<kPlaneStoreF32>(jobs_dev, jobs_host, n_jobs, max_R, any_var, out, absmax2, err, st);
    case kPlaneAbsMax:
      return launch_mode<kPlaneAbsMax>(jobs_dev, jobs_host, n_jobs, max_R, any_var, out, absmax2, err, st);
    case kPlaneStoreBF16:
      return launch_mode<kPlaneStoreBF16>(jobs_dev, jobs_host, n_jobs, max_R, any_var, out, absmax2, err, st);
    case kPlaneStoreF16:
      return launch_mode<kPlaneStoreF16>(jobs_dev, jobs_host, n_jobs, max_R, any_var, out, absmax2, err, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_plane_decode(const void* planes, int plane_type, const ExpDev* e_host_copy,
                                float* psi, float* phi, cudaStream_t st) {
  const ExpDev e = *e_host_copy;
  const int blocks = 1024;
  if (plane_type == kF32)
    k_plane_decode<kF32><<<blocks, kThreads, 0, st>>>(planes, e, psi, phi);
  else if (plane_type == kBF16)
    k_plane_decode<kBF16><<<blocks, kThreads, 0, st>>>(planes, e, psi, phi);
  else
    k_plane_decode<kF16><<<blocks, kThreads, 0, st>>>(planes, e, psi, phi);
  return cudaGetLastError();
}

}  // namespace ndt
