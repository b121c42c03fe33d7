// k_planes.cu -- matched-filter planes (paper sec. 3: matched filter with a
// Gaussian PSF whose width is given in the image header):
//   psi(p) = sum_k P(k) I(p+k) / V(p+k),   phi(p) = sum_k P(k)^2 / V(p+k),
// P the Gaussian of sigma truncated at R = ceil(4 sigma), unit sum over the
// (2R+1)^2 window, terms outside the image dropped.  The truncated Gaussian
// factorises, P = g (x) g with g the unit-sum 1-D window, so both planes are
// separable correlations (zero padding factorises too).  One CTA computes one
// 32 x 32 output tile from a (32+2R)^2 input tile in shared memory and writes
// it as one contiguous tile of the tile-major (psi, phi) plane.  The window
// weights come precomputed with the job.  FP32 planes: one pass, 4 bytes read
// (8 with a variance plane) and 8 written per pixel.  BF16 planes: one pass
// writing 4 bytes per pixel, values divided by a-priori per-exposure scales
// (BF16 has the FP32 exponent range, so no data-dependent range is needed).
// FP16 planes: two passes, one reducing the largest |psi| and phi of each
// plane, one writing 16-bit pairs scaled so those maxima map to 2^14.
#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int kThreads = 256;

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_planes(const PlaneJob* __restrict__ jobs,
                                                     void* __restrict__ out,
                                                     unsigned int* __restrict__ absmax2) {
  const PlaneJob& J = jobs[blockIdx.y];
  const int tile = blockIdx.x;
  const int tiles_x = J.tiles_x, W = J.W, H = J.H;
  if (tile >= tiles_x * J.tiles_y) return;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int R = J.R;
  const int E = kTile + 2 * R;                 // input tile edge
  extern __shared__ float sm[];
  float* gw = sm;                              // 2R+1 (<= 33)
  float* gw2 = sm + 40;
  float* ex = sm + 80;                         // 32: sum of g^2 inside the image along x
  float* ey = sm + 112;                        // 32: same along y
  float* in = sm + 144;                        // E x E  : I / V
  float* hor = in + E * E;                     // E x 32 : horizontal pass of psi
  float* inw = hor + E * kTile;                // E x E  : 1 / V   (variance plane only)
  float* horw = inw + E * E;                   // E x 32
  const bool vplane = J.var != nullptr;
  const int n2 = 2 * R + 1;
  if (threadIdx.x < n2) {
    gw[threadIdx.x] = J.g[threadIdx.x];
    gw2[threadIdx.x] = J.g2[threadIdx.x];
  }
  const int x0 = tx * kTile - R, y0 = ty * kTile - R;
  const float inv_vc = 1.0f / J.var_c;
  for (int i = threadIdx.x; i < E * E; i += kThreads) {
    const int yy = y0 + i / E, xx = x0 + i % E;
    float a = 0.0f, w = 0.0f;
    if (xx >= 0 && xx < W && yy >= 0 && yy < H) {
      const int64_t p = (int64_t)yy * W + xx;
      const float I = __ldg(J.image + p);
      if (vplane) {
        w = 1.0f / __ldg(J.var + p);
        a = I * w;
      } else {
        a = I * inv_vc;
      }
    }
    in[i] = a;
    if (vplane) inw[i] = w;
  }
  __syncthreads();
  if (!vplane && threadIdx.x < 2 * kTile) {
    // constant variance: phi = (1/V) * (sum of g^2 inside the image along x)
    //                                * (sum of g^2 inside the image along y)
    const bool along_x = threadIdx.x < kTile;
    const int c = (along_x ? tx : ty) * kTile + (threadIdx.x % kTile);
    const int lim = along_x ? W : H;
    float s = 0.0f;
    for (int k = 0; k < n2; ++k) {
      const int q = c + k - R;
      if (q >= 0 && q < lim) s += gw2[k];
    }
    (along_x ? ex : ey)[threadIdx.x % kTile] = s;
  }
  for (int i = threadIdx.x; i < E * kTile; i += kThreads) {
    const int r = i / kTile, c = i % kTile;
    const float* row = in + r * E + c;
    float acc = 0.0f;
    for (int k = 0; k < n2; ++k) acc = fmaf(gw[k], row[k], acc);
    hor[i] = acc;
    if (vplane) {
      const float* roww = inw + r * E + c;
      float accw = 0.0f;
      for (int k = 0; k < n2; ++k) accw = fmaf(gw2[k], roww[k], accw);
      horw[i] = accw;
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
  const int64_t base = J.plane_off + ((int64_t)tile << (2 * kTileShift));
  for (int i = threadIdx.x; i < kTile * kTile; i += kThreads) {
    const int y = i >> kTileShift, x = i & (kTile - 1);
    float psi = 0.0f, phi = 0.0f;
    for (int k = 0; k < n2; ++k) psi = fmaf(gw[k], hor[(y + k) * kTile + x], psi);
    if (vplane) {
      for (int k = 0; k < n2; ++k) phi = fmaf(gw2[k], horw[(y + k) * kTile + x], phi);
    } else {
      phi = ex[x] * ey[y] * inv_vc;
    }
    if (MODE == kPlaneStoreF32) {
      reinterpret_cast<float2*>(out)[base + i] = make_float2(psi, phi);
    } else if (MODE == kPlaneAbsMax) {
      if (tx * kTile + x < W && ty * kTile + y < H) {
        m0 = fmaxf(m0, fabsf(psi));
        m1 = fmaxf(m1, fabsf(phi));
      }
    } else {
      // round-to-nearest-even of value / scale; the scale maps the plane's
      // largest magnitude to 2^14
      const float q0 = __fdiv_rn(psi, s0), q1 = __fdiv_rn(phi, s1);
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

size_t planes_smem_bytes(int R, bool vplane) {
  const int E = kTile + 2 * R;
  size_t f = 144 + (size_t)E * E + (size_t)E * kTile;
  if (vplane) f += (size_t)E * E + (size_t)E * kTile;
  return f * sizeof(float);
}

template <int MODE>
cudaError_t launch_mode(const PlaneJob* jobs_dev, int n_jobs, int max_tiles, int max_R, bool any_var,
                        void* out, unsigned int* absmax2, cudaStream_t st) {
  // sized for the largest window radius among the jobs
  const size_t smem = planes_smem_bytes(max_R, any_var);
  cudaError_t e = cudaFuncSetAttribute(k_planes<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)planes_smem_bytes(kMaxPsfRadius, true));
  if (e != cudaSuccess) return e;
  dim3 grid(max_tiles, n_jobs);
  k_planes<MODE><<<grid, kThreads, smem, st>>>(jobs_dev, out, absmax2);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_planes(const PlaneJob* jobs_dev, int n_jobs, int max_tiles, int max_R, bool any_var,
                          int mode, void* out, unsigned int* absmax2, cudaStream_t st) {
  switch (mode) {
    case kPlaneStoreF32:
      return launch_mode<kPlaneStoreF32>(jobs_dev, n_jobs, max_tiles, max_R, any_var, out, absmax2, st);
    case kPlaneAbsMax:
      return launch_mode<kPlaneAbsMax>(jobs_dev, n_jobs, max_tiles, max_R, any_var, out, absmax2, st);
    case kPlaneStoreBF16:
      return launch_mode<kPlaneStoreBF16>(jobs_dev, n_jobs, max_tiles, max_R, any_var, out, absmax2, st);
    case kPlaneStoreF16:
      return launch_mode<kPlaneStoreF16>(jobs_dev, n_jobs, max_tiles, max_R, any_var, out, absmax2, st);
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
