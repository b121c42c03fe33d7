// k_vet.cu -- learned vetting of candidates (paper sec. 5.2.3: a network
// that learns to tell stacked images of real detections from stacks of false
// ones; the paper leaves it as future work and fixes no architecture).
//
// Stamps.  For each candidate the positions along its track are computed by
// the same device code as the stacking path; one CTA then accumulates, for
// every offset q of a 21 x 21 window centred on the predicted pixel, the
// matched-filter sums over the exposures where the centre lies inside the
// image: SPsi(q), SPhi(q), Q(q) = sum psi^2/phi and the count n(q).
//   channel 0 = SPsi / sqrt(SPhi)                     (stacked SNR)
//   channel 1 = (Q - SPsi^2/SPhi - (n-1)) / sqrt(2(n-1))  (constant-flux
//               chi-square excess: large when one exposure dominates)
// Stamps are written in FP32 and rounded to BF16 for the network.
//
// Network.  x (2,21,21) BF16 -> conv5x5 2->32 -> ReLU -> conv5x5 32->32 ->
// ReLU -> conv5x5 32->32 -> ReLU -> global average pool -> linear 32->1.
// This file holds the training pass (loss and gradients, FP32 throughout);
// scoring runs on the tensor core (k_cnn_tc.cu).
// One CTA owns one stamp at a time; activations live in shared memory as
// zero-padded 25 x 25 planes, weights of 8 output channels at a time are
// staged in shared memory, and each thread accumulates 8 channels x 2 pixels
// in FP32 registers.  The backward pass recomputes the forward pass in the
// same CTA, keeps the first activation in a global per-stamp scratch, and adds
// its weight gradients to the batch gradient with FP32 atomics.
#include <algorithm>
#include <climits>

#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int S = 21, SP = 25, NPIX = S * S, PLANE = SP * SP, CH = 32, KS = 5, KK = KS * KS;
constexpr int kVetThreads = 256;
// parameter offsets in the flat vector
constexpr int OW1 = 0, OB1 = OW1 + CH * 2 * KK, OW2 = OB1 + CH, OB2 = OW2 + CH * CH * KK,
              OW3 = OB2 + CH, OB3 = OW3 + CH * CH * KK, OWL = OB3 + CH, OBL = OWL + CH,
              NPARAM = OBL + 1;
static_assert(NPARAM == 52929, "parameter layout");

// ------------------------------------------------------------------ stamps --

// Positions along each candidate's track, compacted: entry k < cnt[i] of
// candidate i is (ix << 16 | j, iy) for its k-th exposure j
// (in epoch order) whose nearest pixel lies inside the image.  Before each
// step, the FP32 off-chip test of the persistent stack
// (certainly_off_chip, from the last computed state) removes the exposures
// the track certainly misses: the state stays at its last epoch, and the
// next computed step is longer (still exact).  In a sparse survey this
// removes almost every step.
template <bool DFS>
__global__ void __launch_bounds__(128) k_stamp_pos(const double* __restrict__ states, int64_t n,
                                                   double t0, double t_ref, const int64_t* __restrict__ cand,
                                                   int64_t n_cand, const ExpDev* __restrict__ ex,
                                                   int32_t n_exp, Phys ph, int2* __restrict__ pos,
                                                   int* __restrict__ cnt, unsigned long long* counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cand) return;
  const int64_t o = cand[i];
  int2* out = pos + i * n_exp;
  if (o < 0 || o >= n) {
    cnt[i] = 0;
    return;
  }
  Track<DFS> w;
  w.init(ph, states, n, o, t0, t_ref);
  float rf[3], vf[3], tf;
  w.fp32(rf, vf, tf);
  int k = 0;
  for (int j = 0; j < n_exp; ++j) {
    const ExpDev& e = ex[j];
    if (certainly_off_chip(ph, w.oc, rf, vf, tf, e)) continue;
    dfloat rho[3];
    if (!w.step(ph, e, rho)) {
      atomicAdd(counters + 1, 1ull);
      break;
    }
    w.fp32(rf, vf, tf);
    int ix, iy;
    if (pixel_of(e, rho, ix, iy)) out[k++] = make_int2((ix << 16) | j, iy);   // j < 2^16, ix < 2^15
  }
  cnt[i] = k;
}

// One thread per stamp pixel (448 threads, 441 active); exposures are taken
// kStampUnroll at a time: every thread issues the gathers of all of them
// before accumulating (in exposure order), so several independent loads are
// in flight per thread.  The sums are blocked: each group's kStampUnroll
// terms are added first, then the group sum joins the running sum, so the
// rounding error grows with n/kStampUnroll + kStampUnroll - 1 terms
// (<= 53 u sum|terms| for 200 exposures, u = 2^-24) instead of n, at one add
// per term (a compensated sum takes seven).  The stamps feed a BF16 CNN.
constexpr int kStampUnroll = 4;
constexpr int kStampThreads = 448;

template <int PT>
__global__ void __launch_bounds__(kStampThreads) k_stamps(const int2* __restrict__ pos,
                                                          const int* __restrict__ pos_cnt, int64_t n_cand,
                                                          const ExpDev* __restrict__ ex, int32_t n_exp,
                                                          const void* __restrict__ planes,
                                                          float* __restrict__ out_f32,
                                                          __nv_bfloat16* __restrict__ out_bf16) {
  const int p = threadIdx.x;
  const int dx = p % S - S / 2, dy = p / S - S / 2;
  for (int64_t c = blockIdx.x; c < n_cand; c += gridDim.x) {
    float sp = 0.0f, sf = 0.0f, sq = 0.0f;
    int cnt = 0;
    const int2* cpos = pos + c * n_exp;
    const int m = pos_cnt[c];
    for (int k0 = 0; k0 < m; k0 += kStampUnroll) {
      float2 v[kStampUnroll];
      bool ok[kStampUnroll];
#pragma unroll
      for (int u = 0; u < kStampUnroll; ++u) {
        const int k = k0 + u;
        ok[u] = false;
        v[u] = make_float2(0.0f, 0.0f);
        if (k >= m || p >= NPIX) continue;
        const int2 ctr = cpos[k];
        const ExpDev& e = ex[ctr.x & 0xffff];
        const int px = (ctr.x >> 16) + dx, py = ctr.y + dy;
        if ((unsigned)px >= (unsigned)e.W || (unsigned)py >= (unsigned)e.H) continue;
        v[u] = gather_plane<PT>(planes, e, px, py);
        ok[u] = true;
      }
      float gp = 0.0f, gf = 0.0f, gq = 0.0f;
#pragma unroll
      for (int u = 0; u < kStampUnroll; ++u) {
        if (!ok[u] || !(v[u].y > 0.0f)) continue;
        gp += v[u].x;
        gf += v[u].y;
        gq += __fdividef(v[u].x * v[u].x, v[u].y);   // ~2 ulp
        cnt += 1;
      }
      sp += gp;
      sf += gf;
      sq += gq;
    }
    if (p < NPIX) {
      const float P = sp, F = sf, Q = sq;
      const float ch0 = F > 0.0f ? __fdiv_rn(P, __fsqrt_rn(F)) : 0.0f;
      float ch1 = 0.0f;
      if (cnt >= 2) {
        const float m = (float)(cnt - 1);
        ch1 = __fdiv_rn(Q - __fdiv_rn(P * P, F) - m, __fsqrt_rn(2.0f * m));
      }
      const int64_t base = c * 2 * NPIX;
      if (out_f32) {
        out_f32[base + p] = ch0;
        out_f32[base + NPIX + p] = ch1;
      }
      if (out_bf16) {
        out_bf16[base + p] = __float2bfloat16_rn(ch0);
        out_bf16[base + NPIX + p] = __float2bfloat16_rn(ch1);
      }
    }
  }
}

// --------------------------------------------------------------------- CNN --

// Shared-memory layout of one CNN CTA (floats).
constexpr int SM_X = 0;                       // 2 padded planes (input stamp)
constexpr int SM_A = SM_X + 2 * PLANE + 2;    // 32 padded planes (16-byte aligned start)
constexpr int SM_B = SM_A + CH * PLANE;       // 32 padded planes
constexpr int SM_W = SM_B + CH * PLANE;       // staged weights: [cin][25][8]
constexpr int SM_G = SM_W + CH * KK * 8;      // 32 pooled features
constexpr int SM_M = SM_G + CH;               // 32 x 441 mask bits (y3 > 0), as words
constexpr int SM_MW = (CH * NPIX + 31) / 32;
constexpr int SM_FLOATS = SM_M + SM_MW + 8;
constexpr size_t kCnnSmem = SM_FLOATS * sizeof(float);
static_assert(SM_W % 4 == 0, "staged weights are read as float4");
static_assert(kCnnSmem <= 227 * 1024, "shared memory of one CNN CTA");

__device__ __forceinline__ int pad_idx(int p) { return (p / S + 2) * SP + (p % S + 2); }

// Zero the padded buffers (borders stay zero: only interiors are written).
__device__ void clear_smem(float* sm) {
  for (int i = threadIdx.x; i < SM_W; i += kVetThreads) sm[i] = 0.0f;
}

// Load stamp b (BF16, [2][441]) into the padded input planes.
__device__ void load_stamp(float* sm, const __nv_bfloat16* __restrict__ x, int64_t b) {
  for (int i = threadIdx.x; i < 2 * NPIX; i += kVetThreads) {
    const int c = i / NPIX, p = i % NPIX;
    sm[SM_X + c * PLANE + pad_idx(p)] = __bfloat162float(x[b * 2 * NPIX + i]);
  }
}

// Output modes of conv_layer.
enum ConvOut { kReluStore = 0, kHeadPool = 1, kMaskByPrev = 2 };

// One 5x5 "same" convolution layer from padded `in` (CIN planes) to 32
// output channels.  FLIP = false: weights w[o][c][u][v] (forward);
// FLIP = true: the input-gradient convolution, weights w[c][o][4-u][4-v] of
// the forward layer with c the forward output channel (no bias).
//   kReluStore : out[o] = relu(conv + b) into the padded plane `out`
//   kHeadPool  : pooled g[o] += relu(conv + b) / 441 and mask bits y > 0
//   kMaskByPrev: out[o] = conv * (out[o] > 0), in place (gradient through ReLU)
template <int CIN, bool FLIP, int MODE>
__device__ void conv_layer(float* sm, const float* in, const float* __restrict__ w,
                           const float* __restrict__ bias, float* out) {
  float* ws = sm + SM_W;
  const int t = threadIdx.x;
  const int pa = 2 * t, pb = 2 * t + 1;        // two pixels per thread
  const bool va = pa < NPIX, vb = pb < NPIX;
  const int ia = va ? (pa / S) * SP + pa % S : 0;   // top-left of the 5x5 window in padded coords
  const int ib = vb ? (pb / S) * SP + pb % S : 0;
  for (int og = 0; og < CH / 8; ++og) {
    __syncthreads();
    for (int i = t; i < CIN * KK * 8; i += kVetThreads) {
      const int ol = i % 8, k = (i / 8) % KK, c = i / (8 * KK);
      const int o = og * 8 + ol;
      float wv;
      if (!FLIP) wv = w[(o * CIN + c) * KK + k];
      else wv = w[(c * CH + o) * KK + (KK - 1 - k)];   // w_fwd[c][o][4-u][4-v]
      ws[i] = wv;
    }
    __syncthreads();
    float acc[8][2];
#pragma unroll
    for (int ol = 0; ol < 8; ++ol) {
      const float b0 = bias ? bias[og * 8 + ol] : 0.0f;
      acc[ol][0] = b0;
      acc[ol][1] = b0;
    }
    if (va || vb) {
      for (int c = 0; c < CIN; ++c) {
        const float* ip = in + c * PLANE;
        const float* wc = ws + c * KK * 8;
#pragma unroll
        for (int u = 0; u < KS; ++u) {
#pragma unroll
          for (int v = 0; v < KS; ++v) {
            const float xa = ip[ia + u * SP + v], xb = ip[ib + u * SP + v];
            const float4 w0 = *reinterpret_cast<const float4*>(wc + (u * KS + v) * 8);
            const float4 w1 = *reinterpret_cast<const float4*>(wc + (u * KS + v) * 8 + 4);
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int ol = 0; ol < 8; ++ol) {
              acc[ol][0] = fmaf(wv[ol], xa, acc[ol][0]);
              acc[ol][1] = fmaf(wv[ol], xb, acc[ol][1]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int ol = 0; ol < 8; ++ol) {
      const int o = og * 8 + ol;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int p = q ? pb : pa;
        if (p >= NPIX) continue;
        const float y = acc[ol][q];
        if (MODE == kReluStore) {
          out[o * PLANE + pad_idx(p)] = fmaxf(y, 0.0f);
        } else if (MODE == kHeadPool) {
          if (y > 0.0f) {
            atomicAdd(sm + SM_G + o, y * (1.0f / NPIX));
            atomicOr(reinterpret_cast<unsigned*>(sm + SM_M) + ((o * NPIX + p) >> 5), 1u << ((o * NPIX + p) & 31));
          }
        } else {
          float* dst = out + o * PLANE + pad_idx(p);
          *dst = (*dst > 0.0f) ? y : 0.0f;
        }
      }
    }
  }
  __syncthreads();
}

// Forward pass of the stamp in sm[SM_X]; leaves a1 in A, a2 in B, pooled
// features in G and the y3 > 0 mask in M.  Returns the logit (all threads).
__device__ float cnn_forward_cta(float* sm, const float* __restrict__ th) {
  float* A = sm + SM_A;
  float* B = sm + SM_B;
  for (int i = threadIdx.x; i < CH + SM_MW; i += kVetThreads) sm[SM_G + i] = 0.0f;
  conv_layer<2, false, kReluStore>(sm, sm + SM_X, th + OW1, th + OB1, A);
  conv_layer<CH, false, kReluStore>(sm, A, th + OW2, th + OB2, B);
  conv_layer<CH, false, kHeadPool>(sm, B, th + OW3, th + OB3, nullptr);
  __shared__ float z_sh;
  if (threadIdx.x < 32) {
    float v = sm[SM_G + threadIdx.x] * th[OWL + threadIdx.x];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) z_sh = v + th[OBL];
  }
  __syncthreads();
  return z_sh;
}

// dW[o][c][u][v] += sum_p dy(o, p) * in[c][p + (u, v)] for one layer; dy(o,p)
// is read from the padded plane `dy` (interior) or, with FROM_MASK, built from
// the y3 mask bits and dg[o] / 441.  Also db[o] += sum_p dy(o, p).
template <int CIN, bool FROM_MASK>
__device__ void weight_grad(float* sm, const float* in, const float* dy, const float* dg,
                            float* __restrict__ gw, float* __restrict__ gb) {
  const unsigned* mask = reinterpret_cast<const unsigned*>(sm + SM_M);
  // items: (o quad, c, u): 8 * CIN * 5, each 4 x 5 accumulators
  for (int it = threadIdx.x; it < 8 * CIN * KS; it += kVetThreads) {
    const int u = it % KS, c = (it / KS) % CIN, oq = it / (KS * CIN);
    float acc[4][KS];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int v = 0; v < KS; ++v) acc[a][v] = 0.0f;
    const float* ip = in + c * PLANE + u * SP;
    for (int p = 0; p < NPIX; ++p) {
      float d[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int o = oq * 4 + a;
        if (FROM_MASK) {
          const int bit = o * NPIX + p;
          d[a] = ((mask[bit >> 5] >> (bit & 31)) & 1u) ? dg[o] * (1.0f / NPIX) : 0.0f;
        } else {
          d[a] = dy[o * PLANE + pad_idx(p)];
        }
      }
      const float* row = ip + (p / S) * SP + (p % S);
#pragma unroll
      for (int v = 0; v < KS; ++v) {
        const float x = row[v];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][v] = fmaf(d[a], x, acc[a][v]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int v = 0; v < KS; ++v)
        atomicAdd(gw + ((oq * 4 + a) * CIN + c) * KK + u * KS + v, acc[a][v]);
  }
  // bias gradients: one warp per output channel group
  for (int o = threadIdx.x >> 5; o < CH; o += kVetThreads / 32) {
    float s = 0.0f;
    for (int p = threadIdx.x & 31; p < NPIX; p += 32) {
      if (FROM_MASK) {
        const int bit = o * NPIX + p;
        s += ((mask[bit >> 5] >> (bit & 31)) & 1u) ? dg[o] * (1.0f / NPIX) : 0.0f;
      } else {
        s += dy[o * PLANE + pad_idx(p)];
      }
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(gb + o, s);
  }
  __syncthreads();
}

// Loss and gradient of the mean BCE over the batch: grad must be zeroed and
// loss_sum set to 0 before the launch; a1_scratch holds CH x 441 floats per CTA.
__global__ void __launch_bounds__(kVetThreads) k_cnn_backward(const float* __restrict__ th,
                                                              const __nv_bfloat16* __restrict__ x,
                                                              const float* __restrict__ labels,
                                                              int64_t n, float* __restrict__ grad,
                                                              float* __restrict__ loss_sum,
                                                              float* __restrict__ a1_scratch,
                                                              float* __restrict__ logits) {
  extern __shared__ float sm[];
  float* A = sm + SM_A;
  float* B = sm + SM_B;
  float* gsave = a1_scratch + (int64_t)blockIdx.x * CH * NPIX;
  __shared__ float dg[CH];
  clear_smem(sm);
  const float inv_n = 1.0f / (float)n;
  for (int64_t b = blockIdx.x; b < n; b += gridDim.x) {
    __syncthreads();
    load_stamp(sm, x, b);
    __syncthreads();
    const float z = cnn_forward_cta(sm, th);
    // head: dL/dz for the mean BCE with logits
    const float y = labels[b];
    const float s = 1.0f / (1.0f + __expf(-z));
    const float dz = (s - y) * inv_n;
    if (threadIdx.x == 0) {
      if (logits) logits[b] = z;
      atomicAdd(loss_sum, (fmaxf(z, 0.0f) - z * y + log1pf(__expf(-fabsf(z)))) * inv_n);
      atomicAdd(grad + OBL, dz);
    }
    if (threadIdx.x < CH) {
      atomicAdd(grad + OWL + threadIdx.x, dz * sm[SM_G + threadIdx.x]);
      dg[threadIdx.x] = dz * th[OWL + threadIdx.x];
    }
    // keep a1 for the conv2 weight gradient
    for (int i = threadIdx.x; i < CH * NPIX; i += kVetThreads)
      gsave[i] = A[(i / NPIX) * PLANE + pad_idx(i % NPIX)];
    __syncthreads();
    // layer 3: weight gradient from the mask, then dy3 as a padded plane in A
    weight_grad<CH, true>(sm, B, nullptr, dg, grad + OW3, grad + OB3);
    {
      const unsigned* mask = reinterpret_cast<const unsigned*>(sm + SM_M);
      for (int i = threadIdx.x; i < CH * NPIX; i += kVetThreads) {
        const int o = i / NPIX, p = i % NPIX;
        A[o * PLANE + pad_idx(p)] = ((mask[i >> 5] >> (i & 31)) & 1u) ? dg[o] * (1.0f / NPIX) : 0.0f;
      }
    }
    __syncthreads();
    // dy2 = (W3^T * dy3) masked by a2 > 0, in place in B
    conv_layer<CH, true, kMaskByPrev>(sm, A, th + OW3, nullptr, B);
    // reload a1 into A, then the conv2 weight gradient
    for (int i = threadIdx.x; i < CH * NPIX; i += kVetThreads)
      A[(i / NPIX) * PLANE + pad_idx(i % NPIX)] = gsave[i];
    __syncthreads();
    weight_grad<CH, false>(sm, A, B, nullptr, grad + OW2, grad + OB2);
    // dy1 = (W2^T * dy2) masked by a1 > 0, in place in A
    conv_layer<CH, true, kMaskByPrev>(sm, B, th + OW2, nullptr, A);
    weight_grad<2, false>(sm, sm + SM_X, A, nullptr, grad + OW1, grad + OB1);
  }
}

// Adam (Kingma & Ba 2015) with bias correction; step t starts at 1.
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

__global__ void k_sigmoid(float* __restrict__ z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] = 1.0f / (1.0f + __expf(-z[i]));
}

}  // namespace

cudaError_t launch_sigmoid(float* z, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_sigmoid<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(z, n);
  return cudaGetLastError();
}

int cnn_param_count() { return NPARAM; }
size_t cnn_smem_bytes() { return kCnnSmem; }

cudaError_t launch_stamp_positions(const double* states, int64_t n, double t0, double t_ref, bool state_df,
                                   const int64_t* cand, int64_t n_cand, const ExpDev* ex, int32_t n_exp,
                                   Phys ph, int2* pos, int* cnt, unsigned long long* counters,
                                   cudaStream_t st) {
  // one warp per block while the candidates do not fill every SM with four
  // 128-thread blocks, so that they spread over all SMs (latency-bound threads)
  const int threads = n_cand < 128 * 4 * 152 ? 32 : 128;
  const int64_t blocks = (n_cand + threads - 1) / threads;
  if (blocks == 0) return cudaSuccess;
  if (state_df)
    k_stamp_pos<true><<<(unsigned)blocks, threads, 0, st>>>(states, n, t0, t_ref, cand, n_cand, ex, n_exp, ph,
                                                            pos, cnt, counters);
  else
    k_stamp_pos<false><<<(unsigned)blocks, threads, 0, st>>>(states, n, t0, t_ref, cand, n_cand, ex, n_exp, ph,
                                                             pos, cnt, counters);
  return cudaGetLastError();
}

cudaError_t launch_stamps(const int2* pos, const int* pos_cnt, int64_t n_cand, const ExpDev* ex, int32_t n_exp,
                          const void* planes, int plane_type, float* out_f32,
                          __nv_bfloat16* out_bf16, int n_sms, cudaStream_t st) {
  if (n_cand == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<int64_t>(n_cand, (int64_t)n_sms * 16);
  if (plane_type == kF32)
    k_stamps<kF32><<<blocks, kStampThreads, 0, st>>>(pos, pos_cnt, n_cand, ex, n_exp, planes, out_f32, out_bf16);
  else if (plane_type == kBF16)
    k_stamps<kBF16><<<blocks, kStampThreads, 0, st>>>(pos, pos_cnt, n_cand, ex, n_exp, planes, out_f32, out_bf16);
  else
    k_stamps<kF16><<<blocks, kStampThreads, 0, st>>>(pos, pos_cnt, n_cand, ex, n_exp, planes, out_f32, out_bf16);
  return cudaGetLastError();
}

int cnn_backward_blocks(int64_t n, int n_sms) { return (int)std::min<int64_t>(n, n_sms); }

cudaError_t launch_cnn_backward(const float* th, const __nv_bfloat16* x, const float* labels,
                                int64_t n, float* grad, float* loss_sum, float* a1_scratch,
                                float* logits, int n_sms, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_cnn_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kCnnSmem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)cnn_backward_blocks(n, n_sms);
  k_cnn_backward<<<blocks, kVetThreads, kCnnSmem, st>>>(th, x, labels, n, grad, loss_sum, a1_scratch,
                                                        logits);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* th, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, int step, cudaStream_t st) {
  const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
  k_adam<<<64, 256, 0, st>>>(th, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace ndt
