// k_stack.cu -- the stacking hot path (paper Algorithm 1: SearchImages,
// FilterGPUIntersections, FindLocalSignal and the constant-flux combination,
// fused into one pass that never materialises an intersection).
//
// One thread owns one orbit and walks its exposures in epoch order.  The
// orbit state is carried from one exposure epoch to the next by a two-body
// step (universal variables), so consecutive steps are short and their
// Stumpff functions are low-order polynomials; the light-time correction is
// a second-order expansion about the geometric state.  Psi, Phi and the
// sample count live in registers (compensated FP32 sums) and the stacked
// statistic is formed in the epilogue.  The FP64 pipe bounds this kernel;
// the gathers move 8 bytes (FP32 planes) or 4 bytes (BF16/FP16) per valid
// sample.
#include <type_traits>

#include "ndt_internal.cuh"

namespace ndt {

namespace {

constexpr int kBlock = 128;
// Resident CTAs per SM requested from the register allocator: 5 x 128
// threads caps the stack kernels at 102 registers (20 warps per SM instead of
// 16 at the unconstrained 120, with ~48 bytes spilled), which hides more of the
// double-float and FP64 dependency latency: 3.6 % faster on the main-belt
// survey, 1.9 % on the batched one.  6 spills ~170 bytes.
#ifndef NDT_STACK_MINB
#define NDT_STACK_MINB 5
#endif
// The double-float walk fits in 72 registers without spilling (no FP64
// state): 7 x 128 threads per SM, 28 warps, 1.6-4 % faster than 5 or 6 on the
// main-belt survey; 8 spills.
#ifndef NDT_STACK_MINB_DF
#define NDT_STACK_MINB_DF 8
#endif

__device__ __forceinline__ void load_state(const double* __restrict__ s, int64_t n, int64_t o,
                                           double r[3], double v[3]) {
  for (int c = 0; c < 3; ++c) {
    r[c] = __ldg(s + c * n + o);
    v[c] = __ldg(s + (c + 3) * n + o);
  }
}

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t* __restrict__ a, int64_t n,
                                                   int64_t key) {
  int64_t lo = 0, hi = n;  // first index with a[i] > key
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Per-thread walk state: what every form carries (orbit constants, sums,
// counts) and the two-body state, in FP64 (Walk) or double-float (WalkDF).
struct WalkBase {
  OrbitConst oc;
  CSum sp, sf;
  int cnt;
  int skipped;         // samples whose FP64 work the off-chip test removed
  int blocked;         // of which the block cone test removed
  bool failed;
};

struct Walk : WalkBase {
  double r[3], v[3], rn, inv_r, t_prev;
  float rf[3], vf[3], tf;   // FP32 copy of the state and its epoch (off-chip test)
};

struct WalkDF : WalkBase {
  StateDF s;
  dfloat tp;           // epoch of the state - t_ref
};

// FP32 view of the state and its epoch (- t_ref) for the off-chip and block tests
__device__ __forceinline__ void fp32_view(const Walk& w, float rf[3], float vf[3], float& tf) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    rf[i] = w.rf[i];
    vf[i] = w.vf[i];
  }
  tf = w.tf;
}
__device__ __forceinline__ void fp32_view(const WalkDF& w, float rf[3], float vf[3], float& tf) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    rf[i] = w.s.r[i].h;
    vf[i] = w.s.v[i].h;
  }
  tf = w.tp.h;
}

__device__ __forceinline__ void walk_fp32_copy(Walk& w, float tf) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    w.rf[i] = d2f_trunc(w.r[i]);
    w.vf[i] = d2f_trunc(w.v[i]);
  }
  w.tf = tf;
}

__device__ __forceinline__ void walk_base_init(WalkBase& w) {
  w.sp = CSum{0.0f, 0.0f};
  w.sf = CSum{0.0f, 0.0f};
  w.cnt = 0;
  w.skipped = 0;
  w.blocked = 0;
  w.failed = false;
}

__device__ __forceinline__ void walk_init(Walk& w, const Phys& ph, const double* __restrict__ states,
                                          int64_t n, int64_t o, double t0, double t_ref = 0.0) {
  load_state(states, n, o, w.r, w.v);
  w.rn = sqrt(w.r[0] * w.r[0] + w.r[1] * w.r[1] + w.r[2] * w.r[2]);
  w.inv_r = 1.0 / w.rn;
  w.oc = orbit_const(ph, w.r, w.v, w.inv_r);
  w.t_prev = t0;
  walk_base_init(w);
  walk_fp32_copy(w, (float)(t0 - t_ref));
}

__device__ __forceinline__ void walk_init(WalkDF& w, const Phys& ph, const double* __restrict__ states,
                                          int64_t n, int64_t o, double t0, double t_ref) {
  double r[3], v[3];
  load_state(states, n, o, r, v);
  const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  const double inv_r = 1.0 / rn;
  w.oc = orbit_const(ph, r, v, inv_r);
  w.s = state_df(r, v, rn, inv_r);
  w.tp = split_df(t0 - t_ref);
  walk_base_init(w);
}

// Persistent form: before the FP64 step, the warp skips the sample when the
// FP32 off-chip test holds for every lane (lanes without work vote yes); the
// state then stays at its last epoch and the next computed step is longer.
// Every lane of the warp must call this (the vote is warp-wide).
template <class W>
__device__ __forceinline__ bool warp_skips(W& w, const Phys& ph, const ExpDev& e, bool active) {
  bool off = !active || w.failed;
  if (!off) {
    float rf[3], vf[3], tf;
    fp32_view(w, rf, vf, tf);
    off = certainly_off_chip(ph, w.oc, rf, vf, tf, e);
  }
  if (!__all_sync(0xffffffffu, off)) return false;
  if (active && !w.failed) w.skipped += 1;
  return true;
}

// Block cone test: the exposures of a staged block (cnt <= 32 records, epoch
// order) that the warp's orbits cannot reach.  Each lane bounds its orbit's
// direction over the block by a cone (block_direction); the warp's cone has
// the first working lane's direction as centre and as radius the largest
// chord angle (2 asin(chord/2) <= 1.05 chord for chord <= 0.5) plus that
// lane's bound.  Exposure jj is unreachable when the angle between the
// warp's centre and its tangent point exceeds the warp radius plus the chip
// cone's radius; lane jj tests exposure jj and a ballot gives the mask.
// Warp-uniform; every lane must call it.
template <class W>
__device__ __forceinline__ unsigned warp_block_mask(const W& w, const Phys& ph, const ExpDev* blk, int cnt,
                                                    bool active) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned all = cnt >= 32 ? full : ((1u << cnt) - 1u);
  const ExpDev& em = blk[cnt >> 1];
  const float tm = em.tf;
  const float h = fmaxf(fabsf(blk[0].tf - tm), fabsf(blk[cnt - 1].tf - tm));
  const float om[3] = {em.obs_f[0], em.obs_f[1], em.obs_f[2]};
  float d = 0.0f;
  if (lane < cnt) {
    const float dx = blk[lane].obs_f[0] - om[0], dy = blk[lane].obs_f[1] - om[1], dz = blk[lane].obs_f[2] - om[2];
    d = sqrtf(dx * dx + dy * dy + dz * dz) * 1.0001f + 1e-7f;
  }
  for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(full, d, o));
  const bool has = active && !w.failed;
  const unsigned act = __ballot_sync(full, has);
  if (act == 0u) return all;                   // no orbit of this warp needs any sample
  float u[3] = {0.0f, 0.0f, 0.0f}, ang = 0.0f;
  if (has) {
    float rf[3], vf[3], tf;
    fp32_view(w, rf, vf, tf);
    ang = block_direction(ph, w.oc, rf, vf, tf, tm, h, om, d, u);
  }
  const int lead = __ffs(act) - 1;
  const float c[3] = {__shfl_sync(full, u[0], lead), __shfl_sync(full, u[1], lead),
                      __shfl_sync(full, u[2], lead)};
  float th = 0.0f;
  if (has) {
    const float ex = u[0] - c[0], ey = u[1] - c[1], ez = u[2] - c[2];
    const float chord = sqrtf(ex * ex + ey * ey + ez * ez);
    th = chord <= 0.5f ? fmaf(1.05f, chord, 1e-6f) + ang : INFINITY;
    if (!(th >= 0.0f)) th = INFINITY;          // NaN
  }
  for (int o = 16; o > 0; o >>= 1) th = fmaxf(th, __shfl_xor_sync(full, th, o));
  if (!(th < 1.0f)) return 0u;
  float sr, cr;
  __sincosf(th, &sr, &cr);                     // abs. error ~1e-6 for |th| < 1, inside the slack below
  bool miss = false;
  if (lane < cnt) {
    const ExpDev& e = blk[lane];
    const float cd = c[0] * e.p0_f[0] + c[1] * e.p0_f[1] + c[2] * e.p0_f[2];
    // cos(th + R) = cos th cos R - sin th sin R, with th + R < 2.5 < pi
    miss = e.chip_cos > 0.0707f && cd < fmaf(cr, e.chip_cos, -sr * e.chip_sin) - 1e-5f;
  }
  return __ballot_sync(full, miss) & all;
}

// GEOM64: light time and TAN projection in FP64 (apparent_rho_d, project_h
// and an FP64 floor) instead of double-float.
template <int PT, bool FP32_COPY = false, bool GEOM64 = false>
__device__ __forceinline__ void walk_sample(Walk& w, const Phys& ph, const ExpDev& e,
                                            const void* __restrict__ planes) {
  if (w.failed) return;
  const double dt = e.t - w.t_prev;
  if (kepler_step(ph, w.oc, dt, w.r, w.v, w.rn, w.inv_r) < 0) {
    w.failed = true;
    return;
  }
  w.t_prev = e.t;
  if (FP32_COPY) walk_fp32_copy(w, e.tf);
  int ix, iy;
  bool in;
  if constexpr (GEOM64) {
    double rho[3], xh, yh;
    apparent_rho_d(ph, w.r, w.v, w.inv_r, e, rho);
    in = project_h(e, rho, xh, yh);
    if (in) {
      const double fx = floor(xh), fy = floor(yh);
      in = fx >= 0.0 && fx < (double)e.W && fy >= 0.0 && fy < (double)e.H;
      ix = (int)fx;
      iy = (int)fy;
    }
  } else {
    dfloat rho[3];
    apparent_rho_df(ph, w.r, w.v, w.inv_r, e, rho);
    in = pixel_of(e, rho, ix, iy);
  }
  if (in) {
    const float2 pv = gather_plane<PT>(planes, e, ix, iy);
    w.sp.add(pv.x);
    w.sf.add(pv.y);
    w.cnt += 1;
  }
}

// The double-float walk: step, light time and projection without FP64
// instructions (the FP32 view of the state is its high parts).
template <int PT, bool FP32_COPY = false, bool GEOM64 = false>
__device__ __forceinline__ void walk_sample(WalkDF& w, const Phys& ph, const ExpDev& e,
                                            const void* __restrict__ planes) {
  static_assert(!GEOM64, "the double-float walk has no FP64 geometry");
  if (w.failed) return;
  const dfloat te = {e.tf, e.tf_l};
  if (kepler_step_df(ph, w.oc, df_sub(te, w.tp), w.s) < 0) {
    w.failed = true;
    return;
  }
  w.tp = te;
  dfloat rho[3];
  apparent_rho_dfs(ph, w.s.r, w.s.v, w.s.ir.h, e, rho);
  int ix, iy;
  if (pixel_of(e, rho, ix, iy)) {
    const float2 pv = gather_plane<PT>(planes, e, ix, iy);
    w.sp.add(pv.x);
    w.sf.add(pv.y);
    w.cnt += 1;
  }
}

__device__ __forceinline__ void walk_finish(const WalkBase& w, const StackArgs& a, int64_t o,
                                            bool active) {
  int valid = 0, fails = 0, skipped = 0, blocked = 0;
  if (active) {
    const float P = w.sp.value(), F = w.sf.value();
    if (a.psi_sum) a.psi_sum[o] = P;
    if (a.phi_sum) a.phi_sum[o] = F;
    if (a.nobs) a.nobs[o] = w.cnt;
    float nu = -INFINITY;
    if (!w.failed && F > 0.0f && w.cnt >= a.min_obs) nu = __fdiv_rn(P, __fsqrt_rn(F));
    if (!(nu == nu)) nu = -INFINITY;
    a.snr[o] = nu;
    valid = w.cnt;
    fails = w.failed ? 1 : 0;
    skipped = w.skipped;
    blocked = w.blocked;
  }
  for (int off = 16; off > 0; off >>= 1) {
    valid += __shfl_xor_sync(0xffffffffu, valid, off);
    fails += __shfl_xor_sync(0xffffffffu, fails, off);
    skipped += __shfl_xor_sync(0xffffffffu, skipped, off);
    blocked += __shfl_xor_sync(0xffffffffu, blocked, off);
  }
  if ((threadIdx.x & 31) == 0 && a.counters) {
    if (valid) atomicAdd(a.counters + 0, (unsigned long long)valid);
    if (fails) atomicAdd(a.counters + 1, (unsigned long long)fails);
    if (skipped) atomicAdd(a.counters + 3, (unsigned long long)skipped);
    if (blocked) atomicAdd(a.counters + 4, (unsigned long long)blocked);
  }
}

// Plain form: one thread per orbit, grid covers all orbits.  GEOM: 0 FP64
// state, double-float light time and projection; 1 FP64 throughout; 2
// double-float state (WalkDF).
template <int PT, int GEOM>
__global__ void __launch_bounds__(kBlock, GEOM == 2 ? NDT_STACK_MINB_DF : NDT_STACK_MINB)
    k_stack_plain(const StackArgs a) {
  using W = typename std::conditional<GEOM == 2, WalkDF, Walk>::type;
  const int64_t slot = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const bool active = slot < a.n;
  const int64_t o = active && a.order ? (int64_t)(uint32_t)__ldg(a.order + slot) : slot;
  W w;
  if (active) {
    walk_init(w, a.ph, a.states, a.n, o, a.t0, a.t_ref);
    int64_t e_begin = 0, e_end = a.n_exp;
    if (a.n_fam > 0) {
      const int64_t f = upper_bound_i64(a.fam_orb_off, a.n_fam + 1, o) - 1;
      e_begin = __ldg(a.fam_exp_off + f);
      e_end = __ldg(a.fam_exp_off + f + 1);
    }
    for (int64_t k = e_begin; k < e_end; ++k) {
      const int j = a.n_fam > 0 ? __ldg(a.fam_exp_pos + k) : (int)k;
      walk_sample<PT, false, GEOM == 1>(w, a.ph, a.ex[j], a.planes);
    }
  }
  walk_finish(w, a, o, active);
}

// Barrier of one team.  The barrier ids are immediates (a team index in a
// register would make the assembler reserve all 16 named barriers per CTA,
// which caps residency at 4 CTAs per SM); the team index is warp-uniform.
template <int TEAM>
__device__ __forceinline__ void team_sync(int team) {
  static_assert(TEAM == 32 || TEAM == 64 || TEAM == kBlock, "teams of 1, 2 or 4 warps");
  if constexpr (TEAM == 32) {
    __syncwarp();
  } else if constexpr (TEAM == kBlock) {
    asm volatile("bar.sync 1, %0;" ::"n"(TEAM) : "memory");
  } else if (team == 0) {
    asm volatile("bar.sync 1, %0;" ::"n"(TEAM) : "memory");
  } else {
    asm volatile("bar.sync 2, %0;" ::"n"(TEAM) : "memory");
  }
}

// Persistent form: teams of TEAM_WARPS warps pop (family, orbit tile) items
// from a global counter in longest-family-first order; each team stages ET
// exposure records at a time in shared memory and walks its orbits through
// them.  The loop ends when the counter passes the last item: no thread ever
// waits on another team.
template <int PT, int TEAM_WARPS, int ET, bool DFS>
__global__ void __launch_bounds__(kBlock, DFS ? NDT_STACK_MINB_DF : NDT_STACK_MINB)
    k_stack_persistent(const StackArgs a) {
  using W = typename std::conditional<DFS, WalkDF, Walk>::type;
  constexpr int TEAM = TEAM_WARPS * 32;
  constexpr int NTEAMS = kBlock / TEAM;
  __shared__ ExpDev stage[NTEAMS][ET];
  __shared__ long long item_sh[NTEAMS];
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x % TEAM;
  for (;;) {
    if (tl == 0) item_sh[team] = (long long)atomicAdd(a.queue_head, 1ull);
    team_sync<TEAM>(team);
    const long long item = item_sh[team];
    if (item >= a.n_items) break;
    const int64_t fq = upper_bound_i64(a.item_off, a.n_fam + 1, item) - 1;
    const int f = __ldg(a.fam_order + fq);
    const int64_t tile = item - __ldg(a.item_off + fq);
    const int64_t o_begin = __ldg(a.fam_orb_off + f), o_end = __ldg(a.fam_orb_off + f + 1);
    const int64_t slot = o_begin + tile * TEAM + tl;
    const bool active = slot < o_end;
    const int64_t o = active && a.order ? (int64_t)(uint32_t)__ldg(a.order + slot) : slot;
    const int64_t e_begin = __ldg(a.fam_exp_off + f), e_end = __ldg(a.fam_exp_off + f + 1);
    W w;
    if (active) {
      walk_init(w, a.ph, a.states, a.n, o, a.t0, a.t_ref);
    } else {
      w.failed = true;   // no orbit: votes "off-chip" and does no work
    }
    constexpr int kWords = (int)(sizeof(ExpDev) / 8);
    int backoff = 0, backoff_left = 0;         // warp-uniform
    for (int64_t eb = e_begin; eb < e_end; eb += ET) {
      const int cnt = (int)min((int64_t)ET, e_end - eb);
      // stage cnt exposure records (kWords 8-byte words each) into shared memory
      double* dst = reinterpret_cast<double*>(&stage[team][0]);
      for (int i = tl; i < cnt * kWords; i += TEAM) {
        const int jj = i / kWords, wd = i % kWords;
        const int j = __ldg(a.fam_exp_pos + eb + jj);
        dst[i] = __ldg(reinterpret_cast<const double*>(a.ex + j) + wd);
      }
      team_sync<TEAM>(team);
      // exposures of the block that no orbit of this warp can reach; after a
      // block where the test removed nothing, the warp skips the test for 1,
      // 2, 4, ... up to 8 blocks (dense fields, where every chip is in reach)
      unsigned miss = 0u;
      if (a.block_test) {
        if (backoff_left > 0) {
          --backoff_left;
        } else {
          miss = warp_block_mask(w, a.ph, stage[team], cnt, active);
          backoff = miss ? 0 : min(2 * backoff + 1, 8);
          backoff_left = backoff;
        }
      }
      // every lane runs the loop: the off-chip vote is warp-wide
#pragma unroll 1
      for (int jj = 0; jj < cnt; ++jj) {
        const ExpDev& e = stage[team][jj];
        if ((miss >> jj) & 1u) {
          if (active && !w.failed) {
            w.skipped += 1;
            w.blocked += 1;
          }
          continue;
        }
        if (a.offchip_test && warp_skips(w, a.ph, e, active)) continue;
        walk_sample<PT, true>(w, a.ph, e, a.planes);
      }
      team_sync<TEAM>(team);
    }
    walk_finish(w, a, o, active);
    team_sync<TEAM>(team);   // every thread has read item_sh before it is rewritten
  }
}

// Bits of x (16 of them) spread to the even positions of a 32-bit word.
__device__ __forceinline__ uint32_t spread_bits16(uint32_t x) {
  x &= 0x0000FFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// Sky-footprint key of each orbit: the Morton interleave of the ecliptic
// longitude and latitude (16 bits each) of its topocentric direction at
// exposure j, from the stack's own step and light time (Track);
// items[o] = key << 32 | o.  An orbit whose step fails sorts last.
template <bool DFS>
__global__ void __launch_bounds__(kBlock)
    k_footprint_key(const double* __restrict__ states, int64_t n, double t0, double t_ref,
                    const ExpDev* __restrict__ ex, int32_t j, Phys ph, unsigned long long* __restrict__ items) {
  const int64_t o = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (o >= n) return;
  Track<DFS> w;
  w.init(ph, states, n, o, t0, t_ref);
  uint32_t key = 0xFFFFFFFFu;
  dfloat rho[3];
  if (w.step(ph, ex[j], rho)) {
    constexpr float kPiF = 3.14159265f;
    const float x = rho[0].h, y = rho[1].h, z = rho[2].h;
    const float lon = atan2f(y, x), lat = atan2f(z, sqrtf(x * x + y * y));
    const float uf = fminf(fmaxf((lon + kPiF) * (65535.0f / (2.0f * kPiF)), 0.0f), 65535.0f);
    const float vf = fminf(fmaxf((lat + 0.5f * kPiF) * (65535.0f / kPiF), 0.0f), 65535.0f);
    key = spread_bits16((uint32_t)uf) | (spread_bits16((uint32_t)vf) << 1);
  }
  items[o] = ((unsigned long long)key << 32) | (unsigned long long)(uint32_t)o;
}

// One step of a walk to exposure e and its topocentric vector; false when
// the step failed.
__device__ __forceinline__ bool walk_step_rho(Walk& w, const Phys& ph, const ExpDev& e, dfloat rd[3]) {
  if (kepler_step(ph, w.oc, e.t - w.t_prev, w.r, w.v, w.rn, w.inv_r) < 0) return false;
  w.t_prev = e.t;
  apparent_rho_df(ph, w.r, w.v, w.inv_r, e, rd);
  return true;
}
__device__ __forceinline__ bool walk_step_rho(WalkDF& w, const Phys& ph, const ExpDev& e, dfloat rd[3]) {
  const dfloat te = {e.tf, e.tf_l};
  if (kepler_step_df(ph, w.oc, df_sub(te, w.tp), w.s) < 0) return false;
  w.tp = te;
  apparent_rho_dfs(ph, w.s.r, w.s.v, w.s.ir.h, e, rd);
  return true;
}

template <bool DFS>
__global__ void __launch_bounds__(kBlock) k_predict(const double* __restrict__ states, int64_t n,
                                                   double t0, double t_ref, const ExpDev* __restrict__ ex,
                                                   const int32_t* __restrict__ pos_to_table,
                                                   int32_t n_exp, Phys ph, double* __restrict__ xy,
                                                   unsigned long long* counters) {
  using W = typename std::conditional<DFS, WalkDF, Walk>::type;
  const int64_t o = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (o >= n) return;
  W w;
  walk_init(w, ph, states, n, o, t0, t_ref);
  for (int j = 0; j < n_exp; ++j) {
    const ExpDev& e = ex[j];
    double* out = xy + ((size_t)o * n_exp + pos_to_table[j]) * 2;
    double x = __longlong_as_double(0x7ff8000000000000ll), y = x;
    if (!w.failed) {
      dfloat rd[3];
      if (!walk_step_rho(w, ph, e, rd)) {
        w.failed = true;
        atomicAdd(counters + 1, 1ull);
      } else {
        const double rho[3] = {f2d_exact(rd[0].h) + f2d_exact(rd[0].l), f2d_exact(rd[1].h) + f2d_exact(rd[1].l),
                               f2d_exact(rd[2].h) + f2d_exact(rd[2].l)};
        double px, py;
        if (project_h(e, rho, px, py)) { x = px - 0.5; y = py - 0.5; }
      }
    }
    out[0] = x;
    out[1] = y;
  }
}

template <int PT, bool DFS>
cudaError_t launch_persistent_pt(const StackArgs& a, int n_sms, cudaStream_t st) {
  // one wave: as many resident CTAs per SM as registers and shared memory allow
#define NDT_CASE(TW, ET)                                                         \
  if (a.orbit_tile == TW * 32 && a.exp_tile == ET) {                             \
    int per_sm = 0;                                                              \
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(               \
        &per_sm, k_stack_persistent<PT, TW, ET, DFS>, kBlock, 0);                \
    if (e != cudaSuccess) return e;                                              \
    const int blocks = n_sms * (per_sm > 0 ? per_sm : 1);                        \
    k_stack_persistent<PT, TW, ET, DFS><<<blocks, kBlock, 0, st>>>(a);           \
    return cudaGetLastError();                                                   \
  }
  NDT_CASE(1, 8) NDT_CASE(1, 16) NDT_CASE(1, 32)
  NDT_CASE(2, 8) NDT_CASE(2, 16) NDT_CASE(2, 32)
  NDT_CASE(4, 8) NDT_CASE(4, 16) NDT_CASE(4, 32)
#undef NDT_CASE
  return cudaErrorInvalidValue;
}

template <int GEOM>
void launch_plain_geom(const StackArgs& a, unsigned blocks, cudaStream_t st) {
  if (a.plane_type == kF32) k_stack_plain<kF32, GEOM><<<blocks, kBlock, 0, st>>>(a);
  else if (a.plane_type == kBF16) k_stack_plain<kBF16, GEOM><<<blocks, kBlock, 0, st>>>(a);
  else k_stack_plain<kF16, GEOM><<<blocks, kBlock, 0, st>>>(a);
}

}  // namespace

cudaError_t launch_stack_plain(const StackArgs& a, cudaStream_t st) {
  const int64_t blocks = (a.n + kBlock - 1) / kBlock;
  if (blocks == 0) return cudaSuccess;
  if (a.state_df) launch_plain_geom<2>(a, (unsigned)blocks, st);
  else if (a.geometry_fp64) launch_plain_geom<1>(a, (unsigned)blocks, st);
  else launch_plain_geom<0>(a, (unsigned)blocks, st);
  return cudaGetLastError();
}

cudaError_t launch_footprint_order(const double* states, int64_t n, double t0, double t_ref, const ExpDev* ex,
                                   int32_t j, Phys ph, bool state_df, unsigned long long* a,
                                   unsigned long long* b, unsigned int* hist, unsigned long long** sorted,
                                   cudaStream_t st) {
  const int64_t blocks = (n + kBlock - 1) / kBlock;
  if (blocks == 0) return cudaSuccess;
  if (state_df)
    k_footprint_key<true><<<(unsigned)blocks, kBlock, 0, st>>>(states, n, t0, t_ref, ex, j, ph, a);
  else
    k_footprint_key<false><<<(unsigned)blocks, kBlock, 0, st>>>(states, n, t0, t_ref, ex, j, ph, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sort_items_hi32(a, b, hist, n, 4, sorted, st);   // the 32-bit key: four 8-bit passes
}

cudaError_t launch_stack_persistent(const StackArgs& a, int n_sms, cudaStream_t st) {
  if (a.state_df) {
    if (a.plane_type == kF32) return launch_persistent_pt<kF32, true>(a, n_sms, st);
    if (a.plane_type == kBF16) return launch_persistent_pt<kBF16, true>(a, n_sms, st);
    return launch_persistent_pt<kF16, true>(a, n_sms, st);
  }
  if (a.plane_type == kF32) return launch_persistent_pt<kF32, false>(a, n_sms, st);
  if (a.plane_type == kBF16) return launch_persistent_pt<kBF16, false>(a, n_sms, st);
  return launch_persistent_pt<kF16, false>(a, n_sms, st);
}

cudaError_t launch_predict(const double* states, int64_t n, double t0, double t_ref, const ExpDev* ex,
                           const int32_t* pos_to_table, int32_t n_exp, Phys ph, bool state_df,
                           double* xy, unsigned long long* counters, cudaStream_t st) {
  const int64_t blocks = (n + kBlock - 1) / kBlock;
  if (blocks == 0) return cudaSuccess;
  if (state_df)
    k_predict<true><<<(unsigned)blocks, kBlock, 0, st>>>(states, n, t0, t_ref, ex, pos_to_table, n_exp, ph,
                                                         xy, counters);
  else
    k_predict<false><<<(unsigned)blocks, kBlock, 0, st>>>(states, n, t0, t_ref, ex, pos_to_table, n_exp, ph,
                                                          xy, counters);
  return cudaGetLastError();
}

}  // namespace ndt
