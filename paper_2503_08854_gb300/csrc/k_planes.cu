// k_planes.cu -- matched-filter planes (paper sec. 3: matched filter with a
// Gaussian PSF whose width is given in the image header):
//   psi(p) = sum_k P(k) I(p+k) / V(p+k),   phi(p) = sum_k P(k)^2 / V(p+k),
// P the Gaussian of sigma truncated at R = ceil(4 sigma), unit sum over the
// (2R+1)^2 window, terms outside the image dropped.  The truncated Gaussian
// factorises, P = g (x) g with g the unit-sum 1-D window, so both planes are
// separable correlations (zero padding factorises too).  One CTA computes one
// 32 x 32 output tile from a (32+2R)^2 input tile in shared memory and writes
// it as one contiguous tile of the tile-major (psi, phi) plane.  The path is
// HBM-bound: 4 bytes read (8 with a variance plane) and 8 written per pixel.
#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int kThreads = 256;

// 1-D unit-sum Gaussian window (FP64 exp, rounded to FP32) and its square.
__device__ void psf_window(float sigma, int R, float* gw, float* gw2) {
  const int lane = threadIdx.x;
  if (lane < 32) {
    double w0 = 0.0, w1 = 0.0;
    const double s2 = 2.0 * (double)sigma * (double)sigma;
    int k0 = lane - R, k1 = lane + 32 - R;
    if (lane <= 2 * R) w0 = exp(-(double)(k0 * k0) / s2);
    if (lane + 32 <= 2 * R) w1 = exp(-(double)(k1 * k1) / s2);
    double sum = w0 + w1;
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane <= 2 * R) {
      double g = w0 / sum;
      gw[lane] = (float)g;
      gw2[lane] = (float)(g * g);
    }
    if (lane + 32 <= 2 * R) {
      double g = w1 / sum;
      gw[lane + 32] = (float)g;
      gw2[lane + 32] = (float)(g * g);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_planes_f32(const PlaneJob* __restrict__ jobs,
                                                         float2* __restrict__ out) {
  const PlaneJob J = jobs[blockIdx.y];
  const int tile = blockIdx.x;
  if (tile >= J.tiles_x * J.tiles_y) return;
  const int tx = tile % J.tiles_x, ty = tile / J.tiles_x;
  const int R = (int)ceil(4.0 * (double)J.sigma);
  const int E = kTile + 2 * R;                 // input tile edge
  extern __shared__ float sm[];
  float* gw = sm;                              // 2R+1 (<= 33)
  float* gw2 = sm + 40;
  float* in = sm + 80;                         // E x E  : I / V
  float* hor = in + E * E;                     // E x 32 : horizontal pass of psi
  float* inw = hor + E * kTile;                // E x E  : 1 / V   (variance plane only)
  float* horw = inw + E * E;                   // E x 32
  const bool vplane = J.var != nullptr;

  psf_window(J.sigma, R, gw, gw2);
  const int x0 = tx * kTile - R, y0 = ty * kTile - R;
  const float inv_vc = 1.0f / J.var_c;
  for (int i = threadIdx.x; i < E * E; i += kThreads) {
    const int yy = y0 + i / E, xx = x0 + i % E;
    float a = 0.0f, w = 0.0f;
    if (xx >= 0 && xx < J.W && yy >= 0 && yy < J.H) {
      const int64_t p = (int64_t)yy * J.W + xx;
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
  const int n2 = 2 * R + 1;
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
  float2* dst = out + J.plane_off + ((int64_t)tile << (2 * kTileShift));
  for (int i = threadIdx.x; i < kTile * kTile; i += kThreads) {
    const int y = i >> kTileShift, x = i & (kTile - 1);
    float psi = 0.0f, phi = 0.0f;
    for (int k = 0; k < n2; ++k) psi = fmaf(gw[k], hor[(y + k) * kTile + x], psi);
    if (vplane) {
      for (int k = 0; k < n2; ++k) phi = fmaf(gw2[k], horw[(y + k) * kTile + x], phi);
    } else {
      // constant variance: phi = (1/V) * (sum of g^2 inside the image along x)
      //                                * (sum of g^2 inside the image along y)
      const int gx = tx * kTile + x, gy = ty * kTile + y;
      float sx = 0.0f, sy = 0.0f;
      for (int k = 0; k < n2; ++k) {
        const int xx = gx + k - R, yy = gy + k - R;
        if (xx >= 0 && xx < J.W) sx += gw2[k];
        if (yy >= 0 && yy < J.H) sy += gw2[k];
      }
      phi = sx * sy * inv_vc;
    }
    dst[i] = make_float2(psi, phi);
  }
}

// Largest |psi| and phi over the pixels inside each image (as ordered bits).
__global__ void __launch_bounds__(kThreads) k_plane_absmax(const PlaneJob* __restrict__ jobs,
                                                           const float2* __restrict__ planes,
                                                           unsigned int* __restrict__ absmax2) {
  const PlaneJob J = jobs[blockIdx.y];
  const int64_t n = (int64_t)J.tiles_x * J.tiles_y * kTile * kTile;
  float m0 = 0.0f, m1 = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const int tile = (int)(i >> (2 * kTileShift));
    const int w = (int)(i & (kTile * kTile - 1));
    const int x = (tile % J.tiles_x) * kTile + (w & (kTile - 1));
    const int y = (tile / J.tiles_x) * kTile + (w >> kTileShift);
    if (x < J.W && y < J.H) {
      const float2 v = planes[J.plane_off + i];
      m0 = fmaxf(m0, fabsf(v.x));
      m1 = fmaxf(m1, fabsf(v.y));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(absmax2 + 2 * blockIdx.y, __float_as_uint(m0));
    atomicMax(absmax2 + 2 * blockIdx.y + 1, __float_as_uint(m1));
  }
}

// Round-to-nearest-even of value / scale into BF16 or FP16 pairs; the scale
// of each plane maps its largest magnitude to 2^14.
template <int PT>
__global__ void __launch_bounds__(kThreads) k_plane_quantize(const PlaneJob* __restrict__ jobs,
                                                             const float2* __restrict__ planes,
                                                             const unsigned int* __restrict__ absmax2,
                                                             void* __restrict__ out,
                                                             float* __restrict__ scales2) {
  const PlaneJob J = jobs[blockIdx.y];
  const float a0 = __uint_as_float(absmax2[2 * blockIdx.y]);
  const float a1 = __uint_as_float(absmax2[2 * blockIdx.y + 1]);
  const float s0 = a0 > 0.0f ? a0 / 16384.0f : 1.0f;
  const float s1 = a1 > 0.0f ? a1 / 16384.0f : 1.0f;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scales2[2 * blockIdx.y] = s0;
    scales2[2 * blockIdx.y + 1] = s1;
  }
  const int64_t n = (int64_t)J.tiles_x * J.tiles_y * kTile * kTile;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const float2 v = planes[J.plane_off + i];
    const float q0 = __fdiv_rn(v.x, s0), q1 = __fdiv_rn(v.y, s1);
    if (PT == kBF16) {
      reinterpret_cast<__nv_bfloat162*>(out)[J.plane_off + i] =
          __halves2bfloat162(__float2bfloat16_rn(q0), __float2bfloat16_rn(q1));
    } else {
      reinterpret_cast<__half2*>(out)[J.plane_off + i] =
          __halves2half2(__float2half_rn(q0), __float2half_rn(q1));
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
  size_t f = 80 + (size_t)E * E + (size_t)E * kTile;
  if (vplane) f += (size_t)E * E + (size_t)E * kTile;
  return f * sizeof(float);
}

}  // namespace

cudaError_t launch_planes_f32(const PlaneJob* jobs_dev, int n_jobs, int max_tiles, float2* out,
                              cudaStream_t st) {
  // worst case: R = 16 and a variance plane -> 2 * (64*64 + 64*32) + 80 floats = 49.5 KB
  const size_t smem = planes_smem_bytes(kMaxPsfRadius, true);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_planes_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid(max_tiles, n_jobs);
  k_planes_f32<<<grid, kThreads, smem, st>>>(jobs_dev, out);
  return cudaGetLastError();
}

cudaError_t launch_plane_absmax(const PlaneJob* jobs_dev, int n_jobs, const float2* planes,
                                unsigned int* absmax2, cudaStream_t st) {
  dim3 grid(64, n_jobs);
  k_plane_absmax<<<grid, kThreads, 0, st>>>(jobs_dev, planes, absmax2);
  return cudaGetLastError();
}

cudaError_t launch_plane_quantize(const PlaneJob* jobs_dev, int n_jobs, const float2* planes,
                                  const unsigned int* absmax2, int plane_type, void* out,
                                  float* scales2, cudaStream_t st) {
  dim3 grid(256, n_jobs);
  if (plane_type == kBF16)
    k_plane_quantize<kBF16><<<grid, kThreads, 0, st>>>(jobs_dev, planes, absmax2, out, scales2);
  else
    k_plane_quantize<kF16><<<grid, kThreads, 0, st>>>(jobs_dev, planes, absmax2, out, scales2);
  return cudaGetLastError();
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
