// k_trim.cu -- outlier trimming of candidates' intersections (paper
// sec. 5.2.3: an intersection whose own SNR lies far above what the
// constant-flux combination of the others predicts is dropped by sigma
// clipping, and the stacked SNR is recomputed).
//
// Rule (the paper fixes neither statistic nor threshold).  For a candidate's
// valid intersections j (nearest pixel inside the image, phi_j > 0), with
// s_j = psi_j / sqrt(phi_j) the intersection's own SNR and K the kept set
// (initially every valid intersection), one round computes
//   a_hat = sum_K psi / sum_K phi,   r_j = s_j - a_hat sqrt(phi_j),
//   K' = { j valid : r_j <= kappa }                 (one-sided clip)
// and stops when K' == K or after max_iter rounds (else K = K').  The result
// is nu' = sum_K psi / sqrt(sum_K phi) over the final K (-inf when the sum
// of phi is 0 or |K| < min_obs) and |K|.
//
// One warp per candidate.  The intersections' pixels come from the stamp
// position kernel (one walk per candidate, the stacking path's device code);
// every round re-gathers psi and phi (L2-resident: a candidate touches a few
// hundred pixels) instead of holding them, so any number of exposures fits.
// Lane l owns exposures l, l + 32, ...; the kept set is a bitmask in global
// scratch, word w holding exposures 32w .. 32w + 31, built by warp ballots.
// Sums are compensated FP32 per lane, combined across the warp in FP64.
#include <algorithm>
#include <climits>

#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int kTrimWarps = 4;   // warps (candidates) per block

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Entry k of a candidate's compacted positions: (ix << 16 | exposure, iy).
template <int PT>
__device__ __forceinline__ bool intersection(const int2* __restrict__ cpos, const ExpDev* __restrict__ ex,
                                             const void* __restrict__ planes, int k, float2& v) {
  const int2 p = cpos[k];
  v = gather_plane<PT>(planes, ex[p.x & 0xffff], p.x >> 16, p.y);
  return v.y > 0.0f;
}

template <int PT>
__global__ void __launch_bounds__(kTrimWarps * 32)
    k_trim(const int2* __restrict__ pos, const int* __restrict__ pos_cnt, int64_t n_cand,
           const ExpDev* __restrict__ ex, int32_t n_exp,
           const void* __restrict__ planes, float kappa, int32_t max_iter, int32_t min_obs,
           uint32_t* __restrict__ keep_bits, float* __restrict__ nu_out, int32_t* __restrict__ n_out,
           float* __restrict__ psi_out, float* __restrict__ phi_out) {
  const int lane = threadIdx.x & 31;
  for (int64_t c = (int64_t)blockIdx.x * kTrimWarps + (threadIdx.x >> 5); c < n_cand;
       c += (int64_t)gridDim.x * kTrimWarps) {
    const int2* cpos = pos + c * n_exp;
    const int m = pos_cnt[c];                     // the candidate's in-image intersections
    const int64_t n_words = (m + 31) / 32;
    uint32_t* bits = keep_bits + c * ((n_exp + 31) / 32);
    // round 0 keeps every valid intersection
    for (int64_t w = 0; w < n_words; ++w) {
      const int j = (int)(w * 32) + lane;
      float2 v;
      const bool ok = j < m && intersection<PT>(cpos, ex, planes, j, v);
      const uint32_t word = __ballot_sync(0xffffffffu, ok);
      if (lane == 0) bits[w] = word;
    }
    __syncwarp();
    for (int round = 0; round < max_iter; ++round) {
      // sums over the kept set
      CSum sp{0.0f, 0.0f}, sf{0.0f, 0.0f};
      for (int64_t w = 0; w < n_words; ++w) {
        const int j = (int)(w * 32) + lane;
        const bool kept = (bits[w] >> lane) & 1u;
        float2 v;
        if (kept && intersection<PT>(cpos, ex, planes, j, v)) {
          sp.add(v.x);
          sf.add(v.y);
        }
      }
      const double P = warp_sum_d((double)sp.s + (double)sp.c);
      const double F = warp_sum_d((double)sf.s + (double)sf.c);
      const float a_hat = F > 0.0 ? (float)(P / F) : 0.0f;
      // re-test every valid intersection against the new flux
      bool changed = false;
      for (int64_t w = 0; w < n_words; ++w) {
        const int j = (int)(w * 32) + lane;
        float2 v;
        bool keep = false;
        if (j < m && intersection<PT>(cpos, ex, planes, j, v)) {
          const float rs = __fsqrt_rn(v.y);
          keep = __fdiv_rn(v.x, rs) - a_hat * rs <= kappa;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, keep);
        changed |= word != bits[w];
        __syncwarp();
        if (lane == 0) bits[w] = word;
        __syncwarp();
      }
      if (!changed) break;
    }
    // final sums over the kept set
    CSum sp{0.0f, 0.0f}, sf{0.0f, 0.0f};
    int cnt = 0;
    for (int64_t w = 0; w < n_words; ++w) {
      const int j = (int)(w * 32) + lane;
      float2 v;
      if (((bits[w] >> lane) & 1u) && intersection<PT>(cpos, ex, planes, j, v)) {
        sp.add(v.x);
        sf.add(v.y);
        cnt += 1;
      }
    }
    const double P = warp_sum_d((double)sp.s + (double)sp.c);
    const double F = warp_sum_d((double)sf.s + (double)sf.c);
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (lane == 0) {
      const float Pf = (float)P, Ff = (float)F;
      float nu = -INFINITY;
      if (Ff > 0.0f && cnt >= min_obs) nu = __fdiv_rn(Pf, __fsqrt_rn(Ff));
      nu_out[c] = nu;
      if (n_out) n_out[c] = cnt;
      if (psi_out) psi_out[c] = Pf;
      if (phi_out) phi_out[c] = Ff;
    }
  }
}

}  // namespace

size_t trim_scratch_words(int64_t n_cand, int32_t n_exp) { return (size_t)n_cand * ((n_exp + 31) / 32); }

cudaError_t launch_trim(const int2* pos, const int* pos_cnt, int64_t n_cand, const ExpDev* ex, int32_t n_exp,
                        const void* planes,
                        int plane_type, float kappa, int32_t max_iter, int32_t min_obs, uint32_t* keep_bits,
                        float* nu_out, int32_t* n_out, float* psi_out, float* phi_out, int n_sms,
                        cudaStream_t st) {
  if (n_cand == 0) return cudaSuccess;
  const int64_t want = (n_cand + kTrimWarps - 1) / kTrimWarps;
  const unsigned blocks = (unsigned)std::min<int64_t>(want, (int64_t)n_sms * 16);
  const unsigned threads = kTrimWarps * 32;
  if (plane_type == kF32)
    k_trim<kF32><<<blocks, threads, 0, st>>>(pos, pos_cnt, n_cand, ex, n_exp, planes, kappa, max_iter, min_obs,
                                              keep_bits, nu_out, n_out, psi_out, phi_out);
  else if (plane_type == kBF16)
    k_trim<kBF16><<<blocks, threads, 0, st>>>(pos, pos_cnt, n_cand, ex, n_exp, planes, kappa, max_iter, min_obs,
                                               keep_bits, nu_out, n_out, psi_out, phi_out);
  else
    k_trim<kF16><<<blocks, threads, 0, st>>>(pos, pos_cnt, n_cand, ex, n_exp, planes, kappa, max_iter, min_obs,
                                              keep_bits, nu_out, n_out, psi_out, phi_out);
  return cudaGetLastError();
}

}  // namespace ndt
