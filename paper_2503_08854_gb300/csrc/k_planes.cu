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
#include "ndt_internal.cuh"

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

template <int MODE>
cudaError_t launch_mode(const PlaneJob* jobs_dev, int n_jobs, int max_ctas, int max_R, bool any_var,
                        void* out, unsigned int* absmax2, cudaStream_t st) {
  // the window radius of the launch covers the largest one among the jobs;
  // variance planes come for every exposure or for none
  if (max_R <= 8) {
    return any_var ? launch_rm<MODE, 8, true>(jobs_dev, n_jobs, max_ctas, out, absmax2, st)
                   : launch_rm<MODE, 8, false>(jobs_dev, n_jobs, max_ctas, out, absmax2, st);
  }
  return any_var ? launch_rm<MODE, kMaxPsfRadius, true>(jobs_dev, n_jobs, max_ctas, out, absmax2, st)
                 : launch_rm<MODE, kMaxPsfRadius, false>(jobs_dev, n_jobs, max_ctas, out, absmax2, st);
}

}  // namespace

int planes_ctas_per_job(int tiles_x, int tiles_y) { return planes_ctas_per_job_impl(tiles_x, tiles_y); }

cudaError_t launch_planes(const PlaneJob* jobs_dev, int n_jobs, int max_ctas, int max_R, bool any_var,
                          int mode, void* out, unsigned int* absmax2, cudaStream_t st) {
  switch (mode) {
    case kPlaneStoreF32:
      return launch_mode<kPlaneStoreF32>(jobs_dev, n_jobs, max_ctas, max_R, any_var, out, absmax2, st);
    case kPlaneAbsMax:
      return launch_mode<kPlaneAbsMax>(jobs_dev, n_jobs, max_ctas, max_R, any_var, out, absmax2, st);
    case kPlaneStoreBF16:
      return launch_mode<kPlaneStoreBF16>(jobs_dev, n_jobs, max_ctas, max_R, any_var, out, absmax2, st);
    case kPlaneStoreF16:
      return launch_mode<kPlaneStoreF16>(jobs_dev, n_jobs, max_ctas, max_R, any_var, out, absmax2, st);
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
