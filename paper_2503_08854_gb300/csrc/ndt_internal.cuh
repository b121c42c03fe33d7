// ndt_internal.cuh -- device data layout and the per-sample device code of
// the stacking path (propagate -> light time -> project -> gather), shared by
// the stacking and position-prediction kernels of this library.
//
// Paper mapping (arXiv 2503.08854): sec. 3 "SearchImages" (two-body motion
// about the Sun, WCS projection), "FilterGPUIntersections" (keep pixels inside
// the image), "FindLocalSignal" (Gaussian-PSF matched filter, here a gather
// from precomputed planes) and the constant-flux combination.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bitconv.cuh"
#include "dfloat.cuh"

namespace ndt {

constexpr int kTile = 32;          // plane tile edge (pixels); tiles are 32 x 32
constexpr int kTileShift = 5;
constexpr int kMaxPsfRadius = 16;  // R = ceil(4 sigma) with sigma <= 4
constexpr int kMaxKeplerIters = 40;

// Per-exposure constants on the device, derived on the host from the
// exposure table (328 bytes).
struct ExpDev {
  double t;          // epoch (days)
  double obs[3];     // observer, heliocentric ecliptic (AU)
  double p0[3];      // unit vector of the tangent point, ecliptic frame
  double ax[3];      // x + 1/2 = crpix_h[0] + (rho . ax) / (rho . p0)
  double ay[3];      // y + 1/2 = crpix_h[1] + (rho . ay) / (rho . p0)
  double crpix_h[2]; // reference pixel (0-based) + 1/2: pixel i spans [i, i + 1) in x + 1/2
  int64_t plane_off; // first element of this exposure's plane
  int32_t W, H;
  int32_t tiles_x;   // ceil(W / 32)
  float s_psi;       // dequantisation scale of psi (1 for FP32 planes)
  float s_phi;       // dequantisation scale of phi
  float chip_cos;    // cos of the chip cone's radius (largest off-axis angle + 0.01 rad)
  // FP32 copies for the off-chip test of the persistent form
  float tf;          // epoch - t_ref (days), t_ref = earliest exposure epoch
  float obs_f[3], p0_f[3], ax_f[3], ay_f[3], crpix_f[2];
  float ppr;         // largest pixel stretch per radian at the tangent point (||CD^-1|| in px/rad)
  float cos_far;     // cos(largest off-axis angle of the chip + 0.01 rad), or -2 (never)
  // low parts of p0, ax, ay (their high parts are p0_f, ax_f, ay_f)
  float p0_l[3], ax_l[3], ay_l[3];
  // the double-float projection of the stack: rows with the reference pixel
  // folded in, x + 1/2 = (rho . axc) / (rho . p0) with axc = ax + crpix_h[0] p0
  // (and ayc = ay + crpix_h[1] p0), as high/low pairs
  float axc_f[3], axc_l[3], ayc_f[3], ayc_l[3];
  float obs_l[3];    // low parts of obs (high parts: obs_f), for the double-float light time
  float chip_sin;    // sin of the chip cone's radius
  float tf_l;        // epoch - t_ref - tf: the epoch as the double-float pair (tf, tf_l)
  int32_t pad_;
};
static_assert(sizeof(ExpDev) == 328 && sizeof(ExpDev) % 8 == 0, "ExpDev layout");

struct Phys {
  double gm;        // GM_sun (AU^3/day^2); <= 0: force-free motion
  double sqrt_gm;
  double inv_sqrt_gm;
  double inv_gm;
  float inv_c;      // 1 / c (day/AU) for the light-time correction; 0: none
  float inv_c2;     // 1 / c^2
  float gm_f;       // GM_sun in FP32 (light-time acceleration term)
  int32_t force_free;
  float inv_c_l;    // 1/c - inv_c: 1/c as the double-float pair (inv_c, inv_c_l)
  float inv_c3;     // 1 / c^3
  float gm_l;       // GM_sun - gm_f: GM_sun as the double-float pair (gm_f, gm_l)
  float sgm_h, sgm_l;     // sqrt(GM_sun) as a double-float pair
  float isgm_h, isgm_l;   // 1 / sqrt(GM_sun) as a double-float pair
  int32_t pad_;
};

// Plane storage type tags.
enum PlaneType : int32_t { kF32 = 0, kBF16 = 1, kF16 = 2 };

// Element offset of pixel (ix, iy) inside an exposure plane (tile-major).
__host__ __device__ __forceinline__ int64_t tile_offset(int ix, int iy, int tiles_x) {
  return ((int64_t)((iy >> kTileShift) * tiles_x + (ix >> kTileShift)) << (2 * kTileShift)) +
         ((iy & (kTile - 1)) << kTileShift) + (ix & (kTile - 1));
}

// ---------------------------------------------------------------------------
// Compensated FP32 accumulation (Neumaier's variant of Kahan summation).
// ---------------------------------------------------------------------------
struct CSum {
  float s, c;
  __device__ __forceinline__ void add(float x) {
    float t = __fadd_rn(s, x);
    float e = (fabsf(s) >= fabsf(x)) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
    c = __fadd_rn(c, e);
    s = t;
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};

// ---------------------------------------------------------------------------
// FP64 reciprocal by Newton-Raphson refinement of an FP32 seed (the classical
// iteration y <- y + y (1 - x y), which squares the relative error; e.g.
// Knuth, TAOCP vol. 2, sec. 4.3.3).  The seed is the FP32 reciprocal of x
// rounded to FP32 (relative error < 2^-23, conversions on the integer pipe);
// one step gives < 2^-46 (1.5e-14), two steps reach FP64 rounding.  Valid
// for |x| within the FP32 normal range.
// ---------------------------------------------------------------------------
template <int STEPS>
__device__ __forceinline__ double rcp_nr(double x) {
  double y = f2d_exact(__frcp_rn(d2f_rn(x)));
#pragma unroll
  for (int i = 0; i < STEPS; ++i) y = fma(y, fma(-x, y, 1.0), y);
  return y;
}

// ---------------------------------------------------------------------------
// Stumpff functions C(z) = sum (-z)^k/(2k+2)!, S(z) = sum (-z)^k/(2k+3)!.
// Horner evaluation of the Maclaurin series, with the number of terms chosen
// from |z| so that the truncation error stays below 1e-17; closed forms for
// |z| >= 1.5 (Bate, Mueller & White 1971, sec. 4.3).
// ---------------------------------------------------------------------------
// (-1)^k / (2k+2)! and (-1)^k / (2k+3)!, k = 0..10
__device__ __forceinline__ constexpr double stumpff_c_coef(int k) {
  return k == 0 ? 1.0 / 2 : k == 1 ? -1.0 / 24 : k == 2 ? 1.0 / 720 : k == 3 ? -1.0 / 40320
       : k == 4 ? 1.0 / 3628800 : k == 5 ? -1.0 / 479001600 : k == 6 ? 1.0 / 87178291200.0
       : k == 7 ? -1.0 / 20922789888000.0 : k == 8 ? 1.0 / 6402373705728000.0
       : k == 9 ? -1.0 / 2432902008176640000.0 : 1.0 / 1124000727777607680000.0;
}
__device__ __forceinline__ constexpr double stumpff_s_coef(int k) {
  return k == 0 ? 1.0 / 6 : k == 1 ? -1.0 / 120 : k == 2 ? 1.0 / 5040 : k == 3 ? -1.0 / 362880
       : k == 4 ? 1.0 / 39916800 : k == 5 ? -1.0 / 6227020800.0 : k == 6 ? 1.0 / 1307674368000.0
       : k == 7 ? -1.0 / 355687428096000.0 : k == 8 ? 1.0 / 121645100408832000.0
       : k == 9 ? -1.0 / 51090942171709440000.0 : 1.0 / 25852016738884976640000.0;
}

template <int M>
__device__ __forceinline__ void stumpff_series(double z, double& C, double& S) {
  double c = stumpff_c_coef(M - 1), s = stumpff_s_coef(M - 1);
#pragma unroll
  for (int k = M - 2; k >= 0; --k) {
    c = fma(c, z, stumpff_c_coef(k));
    s = fma(s, z, stumpff_s_coef(k));
  }
  C = c;
  S = s;
}

// Closed forms for |z| >= 1.5 (long steps of fast or long-period orbits):
// out of line, so that their library calls stay out of the instruction
// stream of the short steps.
static __device__ __noinline__ double2 stumpff_closed(double z) {
  double C, S;
  if (z > 0.0) {
    double q = sqrt(z), sn, cs;
    sincos(q, &sn, &cs);
    C = (1.0 - cs) / z;
    S = (q - sn) / (z * q);
  } else {
    double q = sqrt(-z);
    double e = exp(q), ei = 1.0 / e;
    double ch = 0.5 * (e + ei), sh = 0.5 * (e - ei);
    C = (ch - 1.0) / (-z);
    S = (sh - q) / ((-z) * q);
  }
  return make_double2(C, S);
}

__device__ __forceinline__ void stumpff(double z, double& C, double& S) {
  // tier choice by an FP32 compare (every boundary has a wide margin)
  const float zf = d2f_trunc(z), az = fabsf(zf);
  if (az < 1e-6f) {
    stumpff_series<3>(z, C, S);
  } else if (az < 1e-3f) {
    stumpff_series<4>(z, C, S);
  } else if (az < 0.05f) {
    stumpff_series<6>(z, C, S);
  } else if (az < 0.3f) {
    stumpff_series<8>(z, C, S);
  } else if (az < 1.5f) {
    stumpff_series<11>(z, C, S);
  } else {
    const double2 cs = stumpff_closed(z);
    C = cs.x;
    S = cs.y;
  }
}

// Per-orbit constants of the two-body motion.
// Products with these replace divisions by 6 and 24 (an FP64 division is a
// multi-instruction sequence on the FP64 pipe); they only scale correction
// terms, so their last-bit rounding does not matter.
constexpr double kInv6 = 1.0 / 6.0;
constexpr double kInv24 = 1.0 / 24.0;

struct OrbitConst {
  double alpha;        // 2/r - v^2/GM (reciprocal semi-major axis), conserved
  // FP32 bounds and thresholds (compared on the FP32 pipe): the series bounds
  // shrunk so that truncated |dt| never passes them wrongly; half a period
  // (bound orbits; steps beyond it are reduced modulo the period in FP64)
  float series_dt_f, tiny_dt_f, half_period_f, alpha_f;
  // bounds along the whole conic for the off-chip test (FP32): |d^3 r/dt^3| / 6,
  // GM / (2 q^2) >= |acceleration| / 2, and the perihelion speed v_q >= |v|
  float jerk6, half_acc, vq;
};

// Bound for the f/g series: along the whole conic |u| = GM/r^3 <= GM/q^3,
// |p| = |r.v|/r^2 <= v_q/q and |w| = |v^2/r^2 - u| <= v_q^2/q^2 + GM/q^3,
// with q the perihelion distance and v_q the speed there (vis-viva).  With
// K = GM/q^3 + v_q^2/q^2 and dt^2 K <= 1e-7 the neglected terms of the
// series stay at FP64 rounding (see fg_series_step).
//
// alpha and the semi-latus rectum p = |r x v|^2 / GM are FP64 (the cross
// product cancels for nearly radial motion); the rest is FP32 and errs only
// on the safe side: e from sqrt(1 - p alpha) with its radicand raised by
// 1e-6 max(1, |p alpha|) (more than its FP32 rounding), q = p / (1 + e)
// lowered by 1e-6, and with that q the vis-viva v_q^2 = GM (2/q - alpha),
// K, |jerk| and |acceleration| are over-estimates, K and the bounds raised
// by a further 1e-5 and the step thresholds lowered by 1e-5 for their own
// FP32 rounding.  Near-circular orbits (radicand ~0) lose ~3e-4 of q this
// way, about 1e-3 of K.
__device__ __forceinline__ OrbitConst orbit_const(const Phys& ph, const double r[3],
                                                  const double v[3], double inv_r) {
  OrbitConst oc;
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  oc.alpha = 2.0 * inv_r - v2 * ph.inv_gm;
  oc.alpha_f = (float)oc.alpha;
  const double hx = r[1] * v[2] - r[2] * v[1], hy = r[2] * v[0] - r[0] * v[2],
               hz = r[0] * v[1] - r[1] * v[0];
  const float semi = (float)((hx * hx + hy * hy + hz * hz) * ph.inv_gm);
  const float gm = ph.gm_f, sa = semi * oc.alpha_f;
  const float ecc = sqrtf(fmaxf(0.0f, 1.0f - sa) + 1e-6f * fmaxf(1.0f, fabsf(sa)));
  const float q = semi / (1.0f + ecc) * (1.0f - 1e-6f);
  const float vq2 = gm * (2.0f / q - oc.alpha_f);
  const float K = (gm / (q * q * q) + vq2 / (q * q)) * (1.0f + 1e-5f);
  const bool ok = q > 0.0f && K > 0.0f && K < INFINITY;
  oc.series_dt_f = ok ? sqrtf(1e-7f / K) * (1.0f - 1e-5f) : 0.0f;
  oc.tiny_dt_f = ok ? sqrtf(3e-10f / K) * (1.0f - 1e-5f) : 0.0f;
  oc.half_period_f = INFINITY;
  if (oc.alpha_f > 0.0f)   // pi / n, n = sqrt(GM) alpha^1.5 (a threshold only)
    oc.half_period_f = 3.14159265f / (sqrtf(gm) * oc.alpha_f * sqrtf(oc.alpha_f));
  // d^3r/dt^3 = -GM (v / r^3 - 3 r (r.v) / r^5), so |d^3r/dt^3| <= 4 GM |v| / r^3
  // <= 4 GM v_q / q^3 anywhere on the conic (r >= q, |v| <= v_q).
  if (ph.force_free) {
    oc.jerk6 = 0.0f;
    oc.half_acc = 0.0f;
    oc.vq = sqrtf((float)v2) * (1.0f + 1e-5f);
  } else if (ok && vq2 >= 0.0f) {
    const float vq = sqrtf(vq2) * (1.0f + 1e-5f);
    oc.jerk6 = 4.0f * gm * vq / (q * q * q) * (1.0f / 6.0f) * (1.0f + 1e-5f);
    oc.half_acc = 0.5f * gm / (q * q) * (1.0f + 1e-5f);
    oc.vq = vq;
  } else {
    oc.jerk6 = INFINITY;   // degenerate conic: never declared off-chip
    oc.half_acc = INFINITY;
    oc.vq = INFINITY;
  }
  return oc;
}

// ---------------------------------------------------------------------------
// Short steps: the Lagrange f and g series about the current state (e.g.
// Bate, Mueller & White 1971, sec. 4.5; Danby 1988, sec. 6.9), with
// u = GM/r^3, p = (r.v)/r^2, w = v^2/r^2 - u:
//   f = 1 - u t^2/2 + u p t^3/2 + u (3w - 15p^2 + u) t^4/24
//   g = t - u t^3/6 + u p t^4/4
//   fdot = -u t + 3 u p t^2/2 + u (3w - 15p^2 + u) t^3/6
//   gdot = 1 - u t^2/2 + u p t^3
// Used only when dt^2 K <= 1e-7 (K bounds u, p^2 and |w| along the conic):
// the neglected terms are then O((dt^2 K)^(5/2)) relative, and a sweep of
// random conics at the bound against a 40-digit universal-variable solution
// shows relative errors of 1.6e-16 in position and 5e-16 in velocity, so the
// step is exact to FP64 rounding without a Kepler solve (about an hour for
// main-belt orbits, seconds near a close perihelion).
//
// Precision split.  Relative to 1, the t^2 terms are below 5e-8 and every
// higher term below 3e-11 (f, g/t, gdot) or 3e-4 of -u t (fdot).  FP64 is
// kept for -u t^2/2, -u t and 3 u p t^2/2 (the last because its error would
// act on the velocity and grow over the following steps), and for the state
// updates themselves (r' = r + (f-1) r + g v, v' = fdot r + v + (gdot-1) v,
// so that the small parts are never added to 1 first).  The other terms are
// formed in FP32, where their rounding (~1e-7 of terms below 3e-11) stays far
// under FP64 rounding of the result; w comes from the vis-viva integral,
// w = u (1 - alpha r).  The FP32 <-> FP64 conversions run on the integer
// pipe (see bitconv.cuh), so the FP64 pipe sees 39 instructions per step.
//
// 1/|r| of the new state starts from the first-order prediction
// y0 = (1/r)(1 - p t), whose relative error e0 = O(dt^2 K) <= 1e-7, and takes
// one third-order step y = y0 (1 + e/2 + 3 e^2/8) with e = 1 - x y0^2
// (remainder 5 e^3 / 16 < 1e-21; the e^2 term, below 4e-15, is formed in
// FP32).
// ---------------------------------------------------------------------------

__device__ __forceinline__ void fg_series_step(const Phys& ph, const OrbitConst& oc, double t,
                                               double r[3], double v[3], double& rn, double& inv_r) {
  const double ir2 = inv_r * inv_r;
  const double u = ph.gm * ir2 * inv_r;
  const double p = (r[0] * v[0] + r[1] * v[1] + r[2] * v[2]) * ir2;
  const double t2 = t * t;
  const double A = u * (-0.5 * t2);                                  // -u t^2 / 2
  // FP32 parts
  const float tf = d2f_rn(t), uf = d2f_rn(u), pf = d2f_rn(p);
  const float wf = uf * fmaf(-oc.alpha_f, d2f_rn(rn), 1.0f);          // u (1 - alpha r)
  const float c4f = uf * fmaf(3.0f, wf, fmaf(-15.0f * pf, pf, uf));   // u (3w - 15p^2 + u)
  const float upf = uf * pf;
  const float t2f = tf * tf, t3f = t2f * tf, t4f = t2f * t2f;
  const float Bf = fmaf(0.5f * upf, t3f, (c4f * (1.0f / 24.0f)) * t4f);   // f - 1 + u t^2/2
  const float Gf = fmaf(-uf * (1.0f / 6.0f), t3f, (0.25f * upf) * t4f);  // g - t
  const float Kf = (c4f * (1.0f / 6.0f)) * t3f;                          // c4 t^3 / 6
  const float Lf = upf * t3f;                                            // gdot - 1 + u t^2/2
  // FP64 parts
  const double fm1 = A + f2d_exact(Bf);
  const double g = t + f2d_exact(Gf);
  const double fdot = fma(-u, t, fma(1.5 * (u * p), t2, f2d_exact(Kf)));
  const double gdm1 = A + f2d_exact(Lf);
  double rr[3];
  for (int i = 0; i < 3; ++i) rr[i] = fma(fm1, r[i], fma(g, v[i], r[i]));
  for (int i = 0; i < 3; ++i) v[i] = fma(fdot, r[i], fma(gdm1, v[i], v[i]));
  for (int i = 0; i < 3; ++i) r[i] = rr[i];
  const double x = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  const double y0 = inv_r * fma(-p, t, 1.0);
  const double e = fma(-x, y0 * y0, 1.0);
  const float ef = d2f_rn(e);
  const double y = fma(y0, fma(0.5, e, f2d_exact(0.375f * ef * ef)), y0);
  inv_r = y;
  rn = x * y;
}

// Very short steps, dt^2 K <= 3e-10 (back-to-back exposures: 90 s for a
// main-belt orbit gives ~1e-10).  Then even u t^2/2 is below 1.5e-10 and its
// FP32 rounding below 1e-17, so f - 1, g - t and gdot - 1 are formed wholly in
// FP32 (p too: its error only reaches terms below 1e-12 of the step).  FP64 is
// kept for -u t in fdot (an error there would act on the velocity and grow
// over the following steps), for the state updates and for 1/|r|, which takes
// one second-order step y0 (1 + e/2) from the first-order prediction
// (e <= ~1e-9, remainder 3 e^2 / 8 < 1e-18).  26 FP64 instructions.
__device__ __forceinline__ void fg_tiny_step(const Phys& ph, const OrbitConst& oc, double t,
                                             double r[3], double v[3], double& rn, double& inv_r) {
  const double ir2 = inv_r * inv_r;
  const double u = ph.gm * ir2 * inv_r;
  const float irf = d2f_rn(inv_r), tf = d2f_rn(t), uf = d2f_rn(u);
  const float rvf = fmaf(d2f_rn(r[0]), d2f_rn(v[0]),
                         fmaf(d2f_rn(r[1]), d2f_rn(v[1]), d2f_rn(r[2]) * d2f_rn(v[2])));
  const float pf = rvf * irf * irf;
  const float upf = uf * pf;
  const float t2f = tf * tf, t3f = t2f * tf;
  const float Af = -0.5f * uf * t2f;                                  // -u t^2 / 2
  const float fm1f = fmaf(0.5f * upf, t3f, Af);                       // f - 1
  const float gm1f = -uf * (1.0f / 6.0f) * t3f;                       // g - t
  // fdot + u t: 3 u p t^2/2 + u (3w - 15p^2 + u) t^3/6 (the last is ~dt^2 K of
  // u t, with the same sign at every step: kept so the velocity does not drift)
  const float wf = uf * fmaf(-oc.alpha_f, d2f_rn(rn), 1.0f);
  const float c4f = uf * fmaf(3.0f, wf, fmaf(-15.0f * pf, pf, uf));
  const float kf = fmaf(1.5f * upf, t2f, (c4f * (1.0f / 6.0f)) * t3f);
  const float gdm1f = fmaf(upf, t3f, Af);                             // gdot - 1
  const double fm1 = f2d_exact(fm1f), g = t + f2d_exact(gm1f);
  const double fdot = fma(-u, t, f2d_exact(kf));
  const double gdm1 = f2d_exact(gdm1f);
  double rr[3];
  for (int i = 0; i < 3; ++i) rr[i] = fma(fm1, r[i], fma(g, v[i], r[i]));
  for (int i = 0; i < 3; ++i) v[i] = fma(fdot, r[i], fma(gdm1, v[i], v[i]));
  for (int i = 0; i < 3; ++i) r[i] = rr[i];
  const double x = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  const double y0 = fma(inv_r, f2d_exact(-pf * tf), inv_r);            // (1/r)(1 - p t)
  const double e = fma(-x, y0 * y0, 1.0);
  const double y = fma(0.5 * y0, e, y0);
  inv_r = y;
  rn = x * y;
}

// ---------------------------------------------------------------------------
// One two-body step of length dt (universal-variable formulation), updating
// the state (r, v) in place together with |r| and 1/|r|.
//
// The universal Kepler equation F(chi) = 0 (F as in Bate, Mueller & White,
// eq. 4.4-14) is solved by the Laguerre-Conway iteration (Conway 1986) from a
// third-order series guess in dt.  F, F' and F'' are evaluated in FP64; only
// the correction ratio is formed in FP32, so every iterate is an FP64 value
// and the converged root satisfies F = 0 to FP64 rounding.
//
// The iteration stops at the first evaluation whose correction delta is below
// kKeplerStop; the Lagrange coefficients are then taken at chi - delta to
// first order in delta (their derivatives in chi are already at hand), so the
// Stumpff functions are never re-evaluated.  The second-order remainder is
// (delta^2 / 2) |d^2 f / d chi^2| r0 <= (1e-14 / 2) * 0.5 * r0, below 1e-14 AU
// for r0 < 4 AU and 1e-13 AU at 50 AU.  With the series guess the first
// evaluation already meets this for steps up to a few days.
// Returns the number of evaluations, or -1 when kMaxKeplerIters is reached.
// ---------------------------------------------------------------------------
constexpr float kKeplerStop = 1e-7f;

__device__ __forceinline__ int kepler_step(const Phys& ph, const OrbitConst& oc, double dt,
                                           double r[3], double v[3], double& rn, double& inv_r) {
  if (ph.force_free) {
    for (int i = 0; i < 3; ++i) r[i] = fma(v[i], dt, r[i]);
    rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    inv_r = 1.0 / rn;
    return 0;
  }
  const float adtf = fabsf(d2f_trunc(dt));   // |dt| truncated: never above |dt|
  if (adtf <= oc.series_dt_f) {
    if (adtf <= oc.tiny_dt_f)
      fg_tiny_step(ph, oc, dt, r, v, rn, inv_r);
    else
      fg_series_step(ph, oc, dt, r, v, rn, inv_r);
    return 0;
  }
  // (reducing a step just under half a period changes nothing: rint gives 0 or +-1)
  if (adtf > oc.half_period_f) {   // bound orbit, step beyond half a period: reduce it
    const double n = ph.sqrt_gm * oc.alpha * sqrt(oc.alpha);       // mean motion
    const double period = 6.283185307179586476925 / n;
    dt = fma(-rint(dt * (n * 0.15915494309189533577)), period, dt);
  }
  const double alpha = oc.alpha;
  const double sig0 = (r[0] * v[0] + r[1] * v[1] + r[2] * v[2]) * ph.inv_sqrt_gm;
  const double a1 = fma(-alpha, rn, 1.0);            // 1 - alpha r0
  const double sdt = ph.sqrt_gm * dt;
  // third-order series of chi(dt): u - sig0 u^2/(2 r0) - u^3/6 (1/r0 - alpha - 3 sig0^2/r0^2)
  // with u = sqrt(GM) dt / r0, in FP32: the guess only starts the iteration,
  // whose residual, stopping test and final correction are FP64 (its FP32
  // rounding, ~1e-7 of chi, is a small part of the first correction)
  const float irf = d2f_rn(inv_r);
  const float uf = d2f_rn(sdt) * irf, sif = d2f_rn(sig0) * irf;
  const float chif =
      uf * fmaf(uf, fmaf(-uf * (1.0f / 6.0f), fmaf(-3.0f * sif, sif, irf - oc.alpha_f), -0.5f * sif), 1.0f);
  double chi;
  if (fabsf(oc.alpha_f) * chif * chif > 0.25f || !(fabsf(chif) < 1e30f)) {
    chi = alpha > 0.0 ? ph.sqrt_gm * alpha * dt : sdt * inv_r;   // far from the series' range
  } else {
    chi = f2d_exact(chif);
  }
  int it;
  for (it = 1; it <= kMaxKeplerIters; ++it) {
    const double chi2 = chi * chi;
    const double z = alpha * chi2;
    double C, S;
    stumpff(z, C, S);
    const double chi2C = chi2 * C;
    const double chi3S = chi2 * chi * S;
    const double chi1mzS = chi * fma(-z, S, 1.0);
    const double omzC = fma(-z, C, 1.0);
    const double F = fma(sig0, chi2C, fma(a1, chi3S, fma(rn, chi, -sdt)));
    const double dF = fma(sig0, chi1mzS, fma(a1, chi2C, rn));        // = |r|
    const double d2F = fma(sig0, omzC, a1 * chi1mzS);
    const float Ff = d2f_trunc(F), dFf = d2f_trunc(dF), d2Ff = d2f_trunc(d2F);
    const float disc = fabsf(16.0f * dFf * dFf - 20.0f * Ff * d2Ff);
    const float delta = 5.0f * Ff / (dFf + sqrtf(disc));
    if (fabsf(delta) <= kKeplerStop) {
      // outputs at chi - delta, to first order in delta
      const double d = f2d_exact(delta);
      const double chi2C_c = fma(-d, chi1mzS, chi2C);
      const double f = fma(-chi2C_c, inv_r, 1.0);
      const double g = fma(-fma(-d, chi2C, chi3S), ph.inv_sqrt_gm, dt);
      const double rc = fma(-d, d2F, dF);
      const double inv_rc = rcp_nr<1>(rc);   // 1.5e-14: f, g, fdot, gdot stay within 1e-13 AU
      const double fdot = -ph.sqrt_gm * fma(-d, omzC, chi1mzS) * (inv_rc * inv_r);
      const double gdot = fma(-chi2C_c, inv_rc, 1.0);
      double rr[3];
      for (int i = 0; i < 3; ++i) rr[i] = fma(f, r[i], g * v[i]);
      for (int i = 0; i < 3; ++i) v[i] = fma(fdot, r[i], gdot * v[i]);
      for (int i = 0; i < 3; ++i) r[i] = rr[i];
      rn = rc;
      inv_r = inv_rc;
      return it;
    }
    chi -= f2d_exact(delta);
  }
  return -1;
}

// ---------------------------------------------------------------------------
// The two-body state in double-float arithmetic (FP32 pairs, ~48 bits).
//
// On this GPU the FP64 pipe retires 1/64 of the FP32 rate, and with an FP64
// state the short steps above spend ~39 FP64 instructions per sample, which
// bound the stacking kernel.  Carried as double-float pairs, the same f and g
// series take ~450 FP32 instructions, about 7 FP64 instructions' worth of
// issue time.  Every term keeps the precision the FP64 step gives it (the
// FP32 parts stay FP32, the FP64 parts become double-float); what changes is
// the rounding unit of the state and of those parts, 2^-48 instead of 2^-53.
// Over n chained steps that adds about sqrt(n) 2^-48 |r| of rounding noise
// to the position (1e-13 AU after 300 steps at 3 AU): 1e-7 px at 0.2 arcsec
// pixels for a main-belt orbit, 1e-6 px for an NEO 0.05 AU away.  Steps
// beyond the series' range (the universal-variable solve, force-free motion)
// convert the state to FP64, take the FP64 step and convert back: they are
// one step per night, not one per sample.
// ---------------------------------------------------------------------------
struct StateDF {
  dfloat r[3], v[3];
  dfloat ir;   // 1 / |r|
  float rn;    // |r| (FP32: it only enters FP32 terms)
};

__device__ __forceinline__ StateDF state_df(const double r[3], const double v[3], double rn, double inv_r) {
  StateDF s;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.r[i] = split_df(r[i]);
    s.v[i] = split_df(v[i]);
  }
  s.ir = split_df(inv_r);
  s.rn = d2f_rn(rn);
  return s;
}

// fg_series_step with the state, u, p, t^2 and the FP64 parts in double-float,
// and one order more, so that it holds for dt^2 K <= 1e-6 (sqrt(10) times the
// FP64 series' range: 0.1-0.2 day for main-belt orbits, the gaps between
// visits of a night).  With f_n, g_n the coefficients of the Lagrange series
// (f_{n+1} = f_n' - u g_n, g_{n+1} = f_n + g_n', u' = -3 u p, p' = w - 2 p^2,
// w' = -p (u + 2 w)):
//   f_5 = 15 p u (7 p^2 - 3 w - u),   g_5 = -u (45 p^2 - 9 w - u),
//   f_6 = -u (945 p^4 - 630 p^2 w - 210 p^2 u + 45 w^2 + 24 w u + u^2),
//   g_6 = 30 p u (14 p^2 - 6 w - u).
// f and g gain f_5 t^5/120 and g_5 t^5/120, fdot and gdot f_5 t^4/24 +
// f_6 t^5/120 and g_5 t^4/24 + g_6 t^5/120.  With |u|, p^2, |w| <= K the sum
// of |coefficients| of f_n is 2.58 K^3 n! at n = 6 and 5.06 K^3.5 n! at n = 7,
// so at dt^2 K <= 1e-6 the neglected terms are below 3e-18 of f, 1e-15 of
// g - t and 5e-17 of the velocity: under the 2^-48 rounding of the state.
// Every new term is below 1e-8 of the quantity it corrects: FP32.
__device__ __forceinline__ void fg_series_step_df(const Phys& ph, const OrbitConst& oc, dfloat t, StateDF& s) {
  const dfloat ir2 = df_mul(s.ir, s.ir);
  const dfloat u = df_mul(df_mul(dfloat{ph.gm_f, ph.gm_l}, ir2), s.ir);
  const dfloat p = df_mul(df_dot3(s.r, s.v), ir2);
  const dfloat t2 = df_mul(t, t);
  const dfloat A = df_scale2(df_mul(u, t2), -0.5f);                     // -u t^2 / 2
  // FP32 parts, as in fg_series_step
  const float tf = t.h, uf = u.h, pf = p.h;
  const float wf = uf * fmaf(-oc.alpha_f, s.rn, 1.0f);
  const float c4f = uf * fmaf(3.0f, wf, fmaf(-15.0f * pf, pf, uf));
  const float upf = uf * pf;
  const float t2f = tf * tf, t3f = t2f * tf, t4f = t2f * t2f, t5f = t4f * tf;
  const float p2f = pf * pf;
  const float f5 = 15.0f * upf * (7.0f * p2f - 3.0f * wf - uf);
  const float g5 = -uf * (45.0f * p2f - 9.0f * wf - uf);
  const float f6 = -uf * (p2f * (945.0f * p2f - 630.0f * wf - 210.0f * uf) + wf * (45.0f * wf + 24.0f * uf) +
                          uf * uf);
  const float g6 = 30.0f * upf * (14.0f * p2f - 6.0f * wf - uf);
  const float Bf = fmaf(0.5f * upf, t3f, fmaf(c4f * (1.0f / 24.0f), t4f, f5 * (1.0f / 120.0f) * t5f));
  const float Gf = fmaf(-uf * (1.0f / 6.0f), t3f, fmaf(0.25f * upf, t4f, g5 * (1.0f / 120.0f) * t5f));
  const float Kf = fmaf(c4f * (1.0f / 6.0f), t3f, fmaf(f5 * (1.0f / 24.0f), t4f, f6 * (1.0f / 120.0f) * t5f));
  const float Lf = fmaf(upf, t3f, fmaf(g5 * (1.0f / 24.0f), t4f, g6 * (1.0f / 120.0f) * t5f));
  // double-float parts
  const dfloat fm1 = df_add_f(A, Bf);
  const dfloat g = df_add_f(t, Gf);
  const dfloat fdot = df_sub(df_add_f(df_mul(df_mul_f(df_mul(u, p), 1.5f), t2), Kf), df_mul(u, t));
  const dfloat gdm1 = df_add_f(A, Lf);
  dfloat rr[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) rr[i] = df_add_prod2(s.r[i], fm1, s.r[i], g, s.v[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.v[i] = df_add_prod2(s.v[i], gdm1, s.v[i], fdot, s.r[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.r[i] = rr[i];
  // 1/|r|: y0 = (1/r)(1 - p t), e = 1 - x y0^2 (|e| = O(dt^2 K) <= 1e-6),
  // y = y0 (1 + e/2 + 3 e^2/8), remainder 5 e^3 / 16 < 1e-18
  const dfloat x = df_dot3(s.r, s.r);
  const dfloat y0 = df_add_prod_small(s.ir, df_neg(s.ir), df_mul(p, t), 0.0f);   // |p t| <= 1e-3
  const dfloat e = df_add_f(df_neg(df_mul(x, df_mul(y0, y0))), 1.0f);
  const dfloat c = df_add_f(df_scale2(e, 0.5f), 0.375f * e.h * e.h);
  s.ir = df_add_prod_small(y0, y0, c, 0.0f);
  s.rn = x.h * s.ir.h;
}

// fg_tiny_step with the state, u and the FP64 parts in double-float
__device__ __forceinline__ void fg_tiny_step_df(const Phys& ph, const OrbitConst& oc, dfloat t, StateDF& s) {
  const dfloat ir2 = df_mul(s.ir, s.ir);
  const dfloat u = df_mul(df_mul(dfloat{ph.gm_f, ph.gm_l}, ir2), s.ir);
  const float irf = s.ir.h, tf = t.h, uf = u.h;
  const float rvf = fmaf(s.r[0].h, s.v[0].h, fmaf(s.r[1].h, s.v[1].h, s.r[2].h * s.v[2].h));
  const float pf = rvf * irf * irf;
  const float upf = uf * pf;
  const float t2f = tf * tf, t3f = t2f * tf;
  const float Af = -0.5f * uf * t2f;
  const float fm1f = fmaf(0.5f * upf, t3f, Af);
  const float gm1f = -uf * (1.0f / 6.0f) * t3f;
  const float wf = uf * fmaf(-oc.alpha_f, s.rn, 1.0f);
  const float c4f = uf * fmaf(3.0f, wf, fmaf(-15.0f * pf, pf, uf));
  const float kf = fmaf(1.5f * upf, t2f, (c4f * (1.0f / 6.0f)) * t3f);
  const float gdm1f = fmaf(upf, t3f, Af);
  const dfloat g = df_add_f(t, gm1f);
  const dfloat fdot = df_add_f(df_neg(df_mul(u, t)), kf);
  // (f - 1) r and (gdot - 1) v are below 1e-9 of the state: FP32 products
  // (rounding below 1e-16 of it) in the low part of the double-float update
  dfloat rr[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) rr[i] = df_add_prod(s.r[i], g, s.v[i], fm1f * s.r[i].h);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.v[i] = df_add_prod(s.v[i], fdot, s.r[i], gdm1f * s.v[i].h);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.r[i] = rr[i];
  const dfloat x = df_dot3(s.r, s.r);
  const dfloat y0 = df_add_scaled_small(s.ir, -pf * tf);
  const dfloat e = df_add_f(df_neg(df_mul(x, df_mul(y0, y0))), 1.0f);
  s.ir = df_add_scaled_small(y0, 0.5f * e.h);   // |e| <= ~1e-9: its low half is below 2^-53 of 1
  s.rn = x.h * s.ir.h;
}

// A step the series do not cover, through FP64: the state is widened (each
// pair summed in FP64), stepped by kepler_step and split again.
static __device__ __noinline__ int kepler_step_df_long(const Phys& ph, const OrbitConst& oc, dfloat dt, StateDF& s) {
  double r[3], v[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r[i] = f2d_exact(s.r[i].h) + f2d_exact(s.r[i].l);
    v[i] = f2d_exact(s.v[i].h) + f2d_exact(s.v[i].l);
  }
  double inv_r = f2d_exact(s.ir.h) + f2d_exact(s.ir.l);
  double rn = (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) * inv_r;
  const int it = kepler_step(ph, oc, f2d_exact(dt.h) + f2d_exact(dt.l), r, v, rn, inv_r);
  s = state_df(r, v, rn, inv_r);
  return it;
}

// The universal-variable step of kepler_step in double-float, for steps
// beyond the series' range with |z| = |alpha chi^2| <= 5e-2 (a day gives
// z ~ 2e-5 for a main-belt orbit, two weeks ~7e-3).  F, F' and the outputs
// are double-float; the Stumpff functions are 1/2 + z (-1/24 + z/720) and
// 1/6 + z (-1/120 + z/5040) in double-float plus the z^3 to z^5 terms in
// FP32 (below 3.1e-9, rounded to 2e-16; the neglected z^6 terms are below
// 2e-19).  An error dC in C moves chi by ~sigma0 chi^2 dC / r0, so the
// position needs dC below ~1e-16 alpha / z: met over the whole range.  The Laguerre-Conway
// correction delta, F'' and the stopping test are FP32 as in kepler_step,
// and the outputs are taken at chi - delta to first order.  Returns the
// number of evaluations, or 0 with the state untouched when |z| leaves the
// range (the guess is held to 3e-2) or 4 evaluations do not converge: the
// caller then takes the FP64 step.
constexpr float kInv6h = (float)(1.0 / 6.0), kInv6l = (float)(1.0 / 6.0 - (double)(float)(1.0 / 6.0));
constexpr float kInv24h = (float)(1.0 / 24.0), kInv24l = (float)(1.0 / 24.0 - (double)(float)(1.0 / 24.0));
constexpr float kInv120h = (float)(1.0 / 120.0),
                kInv120l = (float)(1.0 / 120.0 - (double)(float)(1.0 / 120.0));
constexpr float kInv720h = (float)(1.0 / 720.0),
                kInv720l = (float)(1.0 / 720.0 - (double)(float)(1.0 / 720.0));
constexpr float kInv5040h = (float)(1.0 / 5040.0),
                kInv5040l = (float)(1.0 / 5040.0 - (double)(float)(1.0 / 5040.0));

__device__ __forceinline__ int kepler_uv_df(const Phys& ph, const OrbitConst& oc, dfloat dt, StateDF& s) {
  const dfloat r0 = df_mul(df_dot3(s.r, s.r), s.ir);
  const dfloat sig0 = df_mul(df_dot3(s.r, s.v), dfloat{ph.isgm_h, ph.isgm_l});
  const dfloat al = split_df(oc.alpha);
  const dfloat a1 = df_add_f(df_neg(df_mul(al, r0)), 1.0f);      // 1 - alpha r0
  const dfloat sdt = df_mul(dfloat{ph.sgm_h, ph.sgm_l}, dt);
  // third-order series guess of chi(dt), as in kepler_step
  const float irf = s.ir.h, uf = sdt.h * irf, sif = sig0.h * irf;
  const float chif =
      uf * fmaf(uf, fmaf(-uf * (1.0f / 6.0f), fmaf(-3.0f * sif, sif, irf - oc.alpha_f), -0.5f * sif), 1.0f);
  if (!(fabsf(oc.alpha_f) * chif * chif <= 3e-2f)) return 0;
  dfloat chi = {chif, 0.0f};
#pragma unroll 1
  for (int it = 1; it <= 4; ++it) {
    const dfloat chi2 = df_mul(chi, chi);
    const dfloat z = df_mul(al, chi2);
    const float zf = z.h;
    if (!(fabsf(zf) <= 5e-2f)) return 0;
    // C = 1/2 + z (-1/24 + z/720) + z^3 (-1/40320 + z/3628800 - z^2/479001600),
    // S = 1/6 + z (-1/120 + z/5040) + z^3 (-1/362880 + z/39916800 - z^2/6227020800)
    const float z3 = zf * zf * zf;
    const float tc = z3 * fmaf(zf, fmaf(-zf, 1.0f / 479001600.0f, 1.0f / 3628800.0f), -1.0f / 40320.0f);
    const float ts = z3 * fmaf(zf, fmaf(-zf, 1.0f / 6227020800.0f, 1.0f / 39916800.0f), -1.0f / 362880.0f);
    const dfloat cz = df_mul(z, df_add(dfloat{-kInv24h, -kInv24l}, df_mul(z, dfloat{kInv720h, kInv720l})));
    const dfloat sz = df_mul(z, df_add(dfloat{-kInv120h, -kInv120l}, df_mul(z, dfloat{kInv5040h, kInv5040l})));
    const dfloat C = df_add_f(df_add_f(cz, tc), 0.5f);
    const dfloat S = df_add(df_add_f(sz, ts), dfloat{kInv6h, kInv6l});
    const dfloat chi2C = df_mul(chi2, C);
    const dfloat chi3S = df_mul(df_mul(chi2, chi), S);
    const dfloat chi1mzS = df_mul(chi, df_add_f(df_neg(df_mul(z, S)), 1.0f));   // chi (1 - z S)
    const float omzCf = fmaf(-zf, C.h, 1.0f);                                     // 1 - z C
    const dfloat F = df_add(df_add(df_mul(sig0, chi2C), df_mul(a1, chi3S)), df_sub(df_mul(r0, chi), sdt));
    const dfloat dF = df_add(df_add(df_mul(sig0, chi1mzS), df_mul(a1, chi2C)), r0);   // = |r|
    const float d2Ff = fmaf(sig0.h, omzCf, a1.h * chi1mzS.h);
    const float Ff = F.h, dFf = dF.h;
    const float disc = fabsf(16.0f * dFf * dFf - 20.0f * Ff * d2Ff);
    const float delta = 5.0f * Ff / (dFf + sqrtf(disc));
    if (fabsf(delta) <= kKeplerStop) {
      // outputs at chi - delta, to first order in delta
      const dfloat chi2C_c = df_sub(chi2C, df_mul_f(chi1mzS, delta));
      const dfloat fm1 = df_neg(df_mul(chi2C_c, s.ir));                               // f - 1
      const dfloat g = df_sub(dt, df_mul(df_sub(chi3S, df_mul_f(chi2C, delta)), dfloat{ph.isgm_h, ph.isgm_l}));
      const dfloat rc = df_add_f(dF, -delta * d2Ff);
      const dfloat inv_rc = df_div(dfloat{1.0f, 0.0f}, rc);
      const dfloat fdot = df_neg(df_mul(df_mul(dfloat{ph.sgm_h, ph.sgm_l}, df_add_f(chi1mzS, -delta * omzCf)),
                                        df_mul(inv_rc, s.ir)));
      const dfloat gdm1 = df_neg(df_mul(chi2C_c, inv_rc));                           // gdot - 1
      dfloat rr[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) rr[i] = df_add_prod2(s.r[i], fm1, s.r[i], g, s.v[i]);
#pragma unroll
      for (int i = 0; i < 3; ++i) s.v[i] = df_add_prod2(s.v[i], gdm1, s.v[i], fdot, s.r[i]);
#pragma unroll
      for (int i = 0; i < 3; ++i) s.r[i] = rr[i];
      s.ir = inv_rc;
      s.rn = rc.h;
      return it;
    }
    chi = df_add_f(chi, -delta);
  }
  return 0;
}

// kepler_step for the double-float state: the series steps in double-float
// (fg_series_step_df up to dt^2 K <= 1e-6, i.e. sqrt(10) times the FP64
// series bound), then the double-float universal-variable step where |z| <=
// 5e-2, every other step through FP64.  Returns as kepler_step does.
__device__ __forceinline__ int kepler_step_df(const Phys& ph, const OrbitConst& oc, dfloat dt, StateDF& s) {
  const float adtf = fabsf(dt.h);   // within 2^-24 of |dt|: inside the 1e-5 shrink of the bounds
  // (3.1622775 < sqrt(10); its product's rounding stays inside the 1e-5 shrink)
  if (!ph.force_free && adtf <= oc.series_dt_f * 3.1622775f) {
    if (adtf <= oc.tiny_dt_f)
      fg_tiny_step_df(ph, oc, dt, s);
    else
      fg_series_step_df(ph, oc, dt, s);
    return 0;
  }
  if (!ph.force_free && adtf <= oc.half_period_f) {
    const int it = kepler_uv_df(ph, oc, dt, s);
    if (it > 0) return it;
  }
  return kepler_step_df_long(ph, oc, dt, s);
}

// ---------------------------------------------------------------------------
// Light-time corrected topocentric vector, in double-float arithmetic (FP32
// pairs, ~48 bits; see dfloat.cuh).  With (r, v) the geometric state at the
// exposure epoch, u = GM/|r|^3, p = (r.v)/|r|^2 and d = r - r_obs, the
// emitted position r(t - tau) is expanded to third order in the light time:
//   rho = d - tau v - (tau^2/2) u r + (tau^3/6) u (v - 3 p r)
// (acceleration -u r, jerk -u (v - 3 p r); the fourth-order term is below
// 1e-14 AU for every orbit class in the workloads).  tau is the root of
// |r(t - tau) - r_obs| = c tau expanded to second order in v/c and first in
// the acceleration:
//   tau = |d|/c - (d.v)/c^2 + (|d| v^2 + (d.v)^2/|d| - u |d| (d.r)) / (2 c^3).
// Against the oracle's iterated light time (exact propagation to t - tau)
// this model, evaluated in 40-digit arithmetic on NEO, main-belt, Kuiper-
// belt and hyperbolic orbits, differs by at most 6e-8 px at 0.2 arcsec
// pixels; without the two cubic terms (tau^3 and u (d.r)) by up to 7e-6 px,
// near a close perihelion.  d, |d|^2, |d|, |d|/c and tau v are double-float
// (tau to ~1e-14 relative), the small terms FP32, and the state enters
// through the integer-pipe split of its FP64 values: no FP64 instruction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void apparent_rho_dfs(const Phys& ph, const dfloat R[3], const dfloat V[3],
                                                 float irf, const ExpDev& e, dfloat rho[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) rho[i] = df_add(R[i], {-e.obs_f[i], -e.obs_l[i]});     // d
  if (ph.inv_c == 0.0f) return;
  const dfloat dist = df_sqrt(df_dot3(rho, rho));
  const float dv = fmaf(rho[0].h, V[0].h, fmaf(rho[1].h, V[1].h, rho[2].h * V[2].h));
  const float v2 = fmaf(V[0].h, V[0].h, fmaf(V[1].h, V[1].h, V[2].h * V[2].h));
  const float uf = ph.force_free ? 0.0f : ph.gm_f * irf * irf * irf;
  const float dr = fmaf(rho[0].h, R[0].h, fmaf(rho[1].h, R[1].h, rho[2].h * R[2].h));
  const float pf = fmaf(R[0].h, V[0].h, fmaf(R[1].h, V[1].h, R[2].h * V[2].h)) * irf * irf;
  const float corr = fmaf(-dv, ph.inv_c2,
                          0.5f * ph.inv_c3 * fmaf(dist.h, fmaf(-uf, dr, v2), dv * dv * rcp_approx(dist.h)));
  const dfloat tau = df_fma_small(dist, {ph.inv_c, ph.inv_c_l}, corr);   // |corr| ~ 1e-4 |d|/c
  const float hf = -0.5f * uf * tau.h * tau.h;                    // -(tau^2/2) u
  const float kf = uf * tau.h * tau.h * tau.h * (1.0f / 6.0f);    // (tau^3/6) u
  const dfloat ntau = df_neg(tau);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float small = fmaf(hf, R[i].h, kf * fmaf(-3.0f * pf, R[i].h, V[i].h));
    rho[i] = df_add_prod(rho[i], ntau, V[i], small);
  }
}

// The same from an FP64 state (split into pairs on the integer pipe).
__device__ __forceinline__ void apparent_rho_df(const Phys& ph, const double r[3], const double v[3],
                                                double inv_r, const ExpDev& e, dfloat rho[3]) {
  dfloat R[3], V[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R[i] = split_df(r[i]);
    V[i] = split_df(v[i]);
  }
  apparent_rho_dfs(ph, R, V, d2f_rn(inv_r), e, rho);
}

// The same light-time model in FP64 throughout (the all-FP64 geometry of
// the plain form's reference variant): rho = d - tau v - (tau^2/2) u r +
// (tau^3/6) u (v - 3 p r), tau = |d|/c - (d.v)/c^2 + (|d| v^2 + (d.v)^2/|d|
// - u |d| (d.r)) / (2 c^3).
__device__ __forceinline__ void apparent_rho_d(const Phys& ph, const double r[3], const double v[3],
                                               double inv_r, const ExpDev& e, double rho[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) rho[i] = r[i] - e.obs[i];
  if (ph.inv_c == 0.0f) return;
  const double ic = (double)ph.inv_c + (double)ph.inv_c_l;
  const double dist = sqrt(rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
  const double dv = rho[0] * v[0] + rho[1] * v[1] + rho[2] * v[2];
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double u = ph.force_free ? 0.0 : ph.gm * inv_r * inv_r * inv_r;
  const double dr = rho[0] * r[0] + rho[1] * r[1] + rho[2] * r[2];
  const double p = (r[0] * v[0] + r[1] * v[1] + r[2] * v[2]) * inv_r * inv_r;
  const double tau = dist * ic - dv * ic * ic + 0.5 * ic * ic * ic * (dist * (v2 - u * dr) + dv * dv / dist);
  const double h = -0.5 * u * tau * tau, k = u * tau * tau * tau * kInv6;
#pragma unroll
  for (int i = 0; i < 3; ++i) rho[i] += -tau * v[i] + h * r[i] + k * (v[i] - 3.0 * p * r[i]);
}

// One orbit's walk through exposures in epoch order, for the kernels that
// need its positions (candidate stage): Track<false> carries the FP64 state,
// Track<true> the double-float one, as the stack's two forms do.  step()
// moves the state to the exposure's epoch and gives the light-time corrected
// topocentric vector (double-float); false on a Kepler failure.  fp32() is
// the FP32 view of the state and its epoch - t_ref for the off-chip test.
template <bool DFS>
struct Track;

template <>
struct Track<false> {
  OrbitConst oc;
  double r[3], v[3], rn, inv_r, t;
  float tf;
  __device__ __forceinline__ void init(const Phys& ph, const double* __restrict__ states, int64_t n, int64_t o,
                                       double t0, double t_ref) {
    for (int c = 0; c < 3; ++c) {
      r[c] = states[c * n + o];
      v[c] = states[(c + 3) * n + o];
    }
    rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    inv_r = 1.0 / rn;
    oc = orbit_const(ph, r, v, inv_r);
    t = t0;
    tf = (float)(t0 - t_ref);
  }
  __device__ __forceinline__ bool step(const Phys& ph, const ExpDev& e, dfloat rho[3]) {
    if (kepler_step(ph, oc, e.t - t, r, v, rn, inv_r) < 0) return false;
    t = e.t;
    tf = e.tf;
    apparent_rho_df(ph, r, v, inv_r, e, rho);
    return true;
  }
  __device__ __forceinline__ void fp32(float rf[3], float vf[3], float& tfo) const {
    for (int c = 0; c < 3; ++c) {
      rf[c] = d2f_trunc(r[c]);
      vf[c] = d2f_trunc(v[c]);
    }
    tfo = tf;
  }
};

template <>
struct Track<true> {
  OrbitConst oc;
  StateDF s;
  dfloat tp;
  __device__ __forceinline__ void init(const Phys& ph, const double* __restrict__ states, int64_t n, int64_t o,
                                       double t0, double t_ref) {
    double r[3], v[3];
    for (int c = 0; c < 3; ++c) {
      r[c] = states[c * n + o];
      v[c] = states[(c + 3) * n + o];
    }
    const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const double inv_r = 1.0 / rn;
    oc = orbit_const(ph, r, v, inv_r);
    s = state_df(r, v, rn, inv_r);
    tp = split_df(t0 - t_ref);
  }
  __device__ __forceinline__ bool step(const Phys& ph, const ExpDev& e, dfloat rho[3]) {
    const dfloat te = {e.tf, e.tf_l};
    if (kepler_step_df(ph, oc, df_sub(te, tp), s) < 0) return false;
    tp = te;
    apparent_rho_dfs(ph, s.r, s.v, s.ir.h, e, rho);
    return true;
  }
  __device__ __forceinline__ void fp32(float rf[3], float vf[3], float& tfo) const {
    for (int c = 0; c < 3; ++c) {
      rf[c] = s.r[c].h;
      vf[c] = s.v[c].h;
    }
    tfo = tp.h;
  }
};

// TAN projection through the precomputed per-exposure rows (Calabretta &
// Greisen 2002, sec. 5.1.3, written with the tangent-plane basis vectors).
// Gives the pixel coordinates shifted by one half, (x + 1/2, y + 1/2), so
// that the nearest pixel is their floor.  Returns false when cos c <= 0.
// The reciprocal of rho . p0 needs ~1e-12 relative accuracy (x within 1e-8 px
// at 4096 px from CRPIX): one Newton step from the FP32 seed gives < 1.5e-14.
// The cos c > 0 test is an FP32 compare (the threshold only keeps the
// reciprocal in range).
__device__ __forceinline__ bool project_h(const ExpDev& e, const double rho[3], double& xh, double& yh) {
  const double den = rho[0] * e.p0[0] + rho[1] * e.p0[1] + rho[2] * e.p0[2];
  if (!(d2f_trunc(den) > 1e-30f)) return false;
  const double inv = rcp_nr<1>(den);
  xh = fma(rho[0] * e.ax[0] + rho[1] * e.ax[1] + rho[2] * e.ax[2], inv, e.crpix_h[0]);
  yh = fma(rho[0] * e.ay[0] + rho[1] * e.ay[1] + rho[2] * e.ay[2], inv, e.crpix_h[1]);
  return true;
}

// Nearest pixel of a topocentric vector (double-float, from apparent_rho_df)
// through the TAN projection in double-float arithmetic (~48-bit dot
// products and quotient, the reference pixel folded into the rows): the
// same x + 1/2 and y + 1/2 as project_h to ~2e-8 px at 0.2 arcsec pixels
// (host check against long double), with no FP64 instruction.  False when
// cos c <= 0 or outside the image.
__device__ __forceinline__ bool pixel_of(const ExpDev& e, const dfloat R[3], int& ix, int& iy) {
  const dfloat P[3] = {{e.p0_f[0], e.p0_l[0]}, {e.p0_f[1], e.p0_l[1]}, {e.p0_f[2], e.p0_l[2]}};
  const dfloat den = df_dot3(R, P);
  if (!(den.h > 1e-30f)) return false;
  const dfloat AX[3] = {{e.axc_f[0], e.axc_l[0]}, {e.axc_f[1], e.axc_l[1]}, {e.axc_f[2], e.axc_l[2]}};
  const dfloat AY[3] = {{e.ayc_f[0], e.ayc_l[0]}, {e.ayc_f[1], e.ayc_l[1]}, {e.ayc_f[2], e.ayc_l[2]}};
  const dfloat xh = df_div(df_dot3(R, AX), den);
  const dfloat yh = df_div(df_dot3(R, AY), den);
  ix = df_floor(xh);
  iy = df_floor(yh);
  return (unsigned)ix < (unsigned)e.W && (unsigned)iy < (unsigned)e.H;
}

// Off-chip test of the persistent form (FP32, no FP64 instruction).  From the
// state (r, v) at epoch t_prev (FP32 copies of the FP64 state), the position
// at the exposure epoch is predicted to second order, p = r + v dt + a dt^2/2,
// with the light time to first order.  The Taylor remainder is at most
// jerk6 |dt|^3 (jerk6 bounds |d^3r/dt^3| / 6 on the whole conic); the light-
// time expansion adds at most half_acc tau^2, FP32 rounding of the inputs and
// sums < 1e-6 (|r| + |rho| + v_q |dt|), the FP32 epochs v_q * 1e-4 d.  The
// position error E becomes an angle below E / (|rho| - E), and within 45 deg
// of the tangent point the TAN projection stretches angles by at most
// sec^2 = 2 times ||CD^-1||: the sample is declared off-chip when the
// predicted pixel lies outside the image by more than 2.5 times that bound
// plus 2 px.  Farther out, with an angular error below 0.005 rad, it is
// declared off-chip when its off-axis angle exceeds the chip's largest one
// (a corner) by more than 0.01 rad.  A false "off-chip" would need the bounds
// above to fail; the test never fires for degenerate conics (infinite
// bounds) or NaNs.
__device__ __forceinline__ bool certainly_off_chip(const Phys& ph, const OrbitConst& oc,
                                                   const float rf[3], const float vf[3], float tf,
                                                   const ExpDev& e) {
  const float dt = e.tf - tf;
  const float r2 = rf[0] * rf[0] + rf[1] * rf[1] + rf[2] * rf[2];
  const float ir = rsqrtf(r2);
  const float k = -ph.gm_f * ir * ir * ir;
  float rho[3], vj[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float acc = k * rf[i];
    rho[i] = fmaf(0.5f * acc, dt * dt, fmaf(vf[i], dt, rf[i])) - e.obs_f[i];
    vj[i] = fmaf(acc, dt, vf[i]);
  }
  const float rr2 = rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2];
  const float rr = rr2 * rsqrtf(rr2);   // NaN for rho = 0: the test then declines
  const float tau = rr * ph.inv_c;
#pragma unroll
  for (int i = 0; i < 3; ++i) rho[i] = fmaf(-vj[i], tau, rho[i]);
  const float adt = fabsf(dt);
  const float err = oc.jerk6 * adt * adt * adt + oc.half_acc * tau * tau +
                    1e-6f * (r2 * ir + rr) + oc.vq * fmaf(1e-6f, adt, 1e-4f);
  const float den = rho[0] * e.p0_f[0] + rho[1] * e.p0_f[1] + rho[2] * e.p0_f[2];
  if (!(rr > 2.0f * err)) return false;
  // fast intrinsics (a few ulp): their error is far inside the 1e-6 slack
  const float eps = __fdividef(err, rr - err);       // angular error bound (rad)
  // (0.005 rad of the 0.01 rad angle margin is left for FP32 rounding of den / rr)
  if (!(den > 0.70710678f * rr)) return eps <= 0.005f && den < e.cos_far * rr;
  const float m = fmaf(2.5f * e.ppr, eps, 2.0f);
  const float x = e.crpix_f[0] + __fdividef(rho[0] * e.ax_f[0] + rho[1] * e.ax_f[1] + rho[2] * e.ax_f[2], den);
  const float y = e.crpix_f[1] + __fdividef(rho[0] * e.ay_f[0] + rho[1] * e.ay_f[1] + rho[2] * e.ay_f[2], den);
  return x < -0.5f - m || x > (float)e.W - 0.5f + m || y < -0.5f - m || y > (float)e.H - 0.5f + m;
}

// Block cone test of the persistent form (FP32).  For a block of exposures
// (epochs within h of the middle one, observers within d_obs of its
// observer), each lane predicts its orbit's position at the middle epoch tm
// from its last FP64 state, as in certainly_off_chip, and bounds the angle
// between that direction from the middle observer and the true direction of
// any sample of the block: the Taylor remainder jerk6 |dt|^3 and the FP32
// slack of certainly_off_chip, the motion over the block (v_q h), the
// observer offset d_obs, light time (|rho| v_q / c plus its acceleration
// term).  Returns the unit direction u and that angular radius (INFINITY
// when the bound is unusable).
__device__ __forceinline__ float block_direction(const Phys& ph, const OrbitConst& oc, const float rf[3],
                                                 const float vf[3], float tf, float tm, float h,
                                                 const float obs_mid[3], float d_obs, float u[3]) {
  const float dt = tm - tf;
  const float r2 = rf[0] * rf[0] + rf[1] * rf[1] + rf[2] * rf[2];
  const float ir = rsqrtf(r2);
  const float k = -ph.gm_f * ir * ir * ir;
  float rho[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) rho[i] = fmaf(0.5f * k * rf[i], dt * dt, fmaf(vf[i], dt, rf[i])) - obs_mid[i];
  const float rr2 = rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2];
  const float rr = rr2 * rsqrtf(rr2);
  const float tau = fmaf(rr, 1.01f, 1e-3f) * ph.inv_c;   // covers |rho| of every sample
  const float adt = fabsf(dt) + h;
  const float err = oc.jerk6 * adt * adt * adt + oc.half_acc * tau * tau + 1e-6f * (r2 * ir + rr) +
                    oc.vq * fmaf(1e-6f, adt, 1e-4f) + oc.vq * (h + tau) + d_obs;
  const float inv = __frcp_rn(rr);
#pragma unroll
  for (int i = 0; i < 3; ++i) u[i] = rho[i] * inv;
  if (!(rr > 2.0f * err)) return INFINITY;
  // arcsin(err / (rr - err)) <= 1.6 err / (rr - err) for err / (rr - err) <= 1
  return 1.6f * __fdividef(err, rr - err);
}

template <int PT>
__device__ __forceinline__ float2 gather_plane(const void* __restrict__ planes, const ExpDev& e,
                                               int ix, int iy) {
  const int64_t off = e.plane_off + tile_offset(ix, iy, e.tiles_x);
  if (PT == kF32) {
    return __ldg(reinterpret_cast<const float2*>(planes) + off);
  } else if (PT == kBF16) {
    __nv_bfloat162 q = __ldg(reinterpret_cast<const __nv_bfloat162*>(planes) + off);
    float2 f = __bfloat1622float2(q);
    return make_float2(f.x * e.s_psi, f.y * e.s_phi);
  } else {
    __half2 q = __ldg(reinterpret_cast<const __half2*>(planes) + off);
    float2 f = __half22float2(q);
    return make_float2(f.x * e.s_psi, f.y * e.s_phi);
  }
}

// ---------------------------------------------------------------------------
// Launchers (defined in the kernel translation units).
// ---------------------------------------------------------------------------
struct PlaneJob {
  // TMA descriptor of the image (2-D, W x H FP32, zero fill outside) when
  // `tma` != 0 (the window radius its box was encoded for): constant
  // variance, W a multiple of 4, 16-byte aligned image
  CUtensorMap tmap;     // 128-byte aligned by its own declaration
  int32_t tma;
  int32_t n_strips;     // TMA form: strips of 4 tiles (0 for the general form)
  const float* image;   // row-major H x W
  const float* var;     // row-major H x W, or null (constant variance)
  float var_c;
  float sigma;
  int32_t W, H, tiles_x, tiles_y;
  int64_t plane_off;    // element offset in the plane buffer
  int32_t R;            // window radius ceil(4 sigma)
  float s_psi, s_phi;   // a-priori scales of the BF16 planes (noise sigma of psi, interior phi)
  float g[2 * kMaxPsfRadius + 1];    // unit-sum 1-D Gaussian window (host FP64, rounded)
  float g2[2 * kMaxPsfRadius + 1];   // its square
  float pre[2 * kMaxPsfRadius + 2];  // pre[i] = sum of g2 over taps < i (FP32, in order)
};

// Plane kernel outputs: FP32 pairs, or (two passes) the largest |psi| and phi
// of each plane, then BF16/FP16 pairs scaled by those maxima.
enum PlaneMode : int32_t { kPlaneStoreF32 = 0, kPlaneAbsMax = 1, kPlaneStoreBF16 = 2, kPlaneStoreF16 = 3 };

// CTAs of the planes kernel per exposure of tiles_x x tiles_y tiles; a launch
// takes the largest over its exposures as grid.x ("max_ctas" below).
// Fill J.tmap and set J.tma (to the launch's window radius, from max_R of
// all jobs) when the job can take the TMA form (constant variance, W % 4 ==
// 0, 16-byte aligned image, TMA available); else J.tma = 0.
void plane_job_try_tma(PlaneJob& J, int max_R);
// plane_job_try_tma for every job, its strip count and prefix sums of g^2.
void plane_jobs_prepare(PlaneJob* jobs, int n_jobs, int max_R);
// Launch the planes of every job: the TMA form for jobs with J.tma set, the
// general form for the others.  `jobs_host` mirrors `jobs_dev`; `err` (device
// word, zeroed by the caller) counts CTAs whose bounded TMA wait gave up.
cudaError_t launch_planes(const PlaneJob* jobs_dev, const PlaneJob* jobs_host, int n_jobs, int max_R,
                          bool any_var, int mode, void* out, unsigned int* absmax2,
                          unsigned int* err, cudaStream_t st);
cudaError_t launch_plane_decode(const void* planes, int plane_type, const ExpDev* e_host_copy,
                                float* psi, float* phi, cudaStream_t st);

struct StackArgs {
  const double* states;        // SoA 6 x n
  int64_t n;
  double t0;
  const ExpDev* ex;            // sorted by epoch
  int32_t n_exp;
  const void* planes;
  int32_t plane_type;
  // families (CSR over sorted exposure positions); n_fam = 0: all x all
  int32_t n_fam;
  const int64_t* fam_orb_off;
  const int64_t* fam_exp_off;
  const int32_t* fam_exp_pos;
  // persistent queue
  const int64_t* item_off;     // n_fam + 1 prefix of items per family (queue order)
  const int32_t* fam_order;    // queue order -> family
  int64_t n_items;
  unsigned long long* queue_head;
  int32_t orbit_tile, exp_tile;
  // outputs (per orbit, any may be null except snr)
  float* psi_sum;
  float* phi_sum;
  int32_t* nobs;
  float* snr;
  int32_t min_obs;
  unsigned long long* counters;  // [0] valid samples, [1] Kepler failures, [3] skipped samples,
                                 // [4] of which the block test skipped
  Phys ph;
  double t_ref;                // epoch origin of ExpDev::tf
  int32_t offchip_test;        // persistent form: skip FP64 work of certainly off-chip samples
  int32_t block_test;          // persistent form: warp cone test per staged exposure block
  int32_t geometry_fp64;       // plain form: FP64 light time and TAN projection
  int32_t state_df;            // two-body state in double-float (WalkDF) instead of FP64
  // footprint order (no families): slot o of the walk takes orbit
  // (uint32) order[o]; null: slot o is orbit o
  const unsigned long long* order;
};

cudaError_t launch_stack_plain(const StackArgs& a, cudaStream_t st);
// Footprint order of n orbits (n < 2^32): keys of their sky direction at
// exposure j (Morton interleave of ecliptic longitude and latitude, 16 bits
// each) sorted with their indices; *sorted points into a or b, each n items.
cudaError_t launch_footprint_order(const double* states, int64_t n, double t0, double t_ref, const ExpDev* ex,
                                   int32_t j, Phys ph, bool state_df, unsigned long long* a,
                                   unsigned long long* b, unsigned int* hist, unsigned long long** sorted,
                                   cudaStream_t st);
cudaError_t launch_stack_persistent(const StackArgs& a, int n_sms, cudaStream_t st);
cudaError_t launch_predict(const double* states, int64_t n, double t0, double t_ref, const ExpDev* ex,
                           const int32_t* exp_pos_to_table, int32_t n_exp, Phys ph, bool state_df,
                           double* xy, unsigned long long* counters, cudaStream_t st);

// Number of values of nu (n of them) at least thr, into *out (device).
cudaError_t launch_count_ge(const float* nu, int64_t n, float thr, unsigned long long* out, cudaStream_t st);

// Stable LSD radix sort (k_topk.cu) of k 64-bit items on bits 32 .. 32 + 8
// passes - 1, ping-ponging between a and b; *sorted is the buffer that holds
// the result.  hist needs sort_hist_bytes(k).
cudaError_t sort_items_hi32(unsigned long long* a, unsigned long long* b, unsigned int* hist, int64_t k,
                            int passes, unsigned long long** sorted, cudaStream_t st);
size_t sort_hist_bytes(int64_t k);

// duplicate suppression of ranked candidates (k_dedup.cu)
uint32_t dedup_table_size(int64_t n_cand);
size_t dedup_scratch_bytes(int64_t n_cand, int n_ref, uint32_t table);
cudaError_t launch_dedup(const double* states, int64_t n, double t0, double t_ref, bool state_df,
                         const int64_t* cand, int64_t n_cand, const ExpDev* ex, const int32_t* ref_dev,
                         int n_ref, Phys ph, float radius, void* scratch, unsigned long long* counters,
                         int64_t* out, int* n_keep_dev, cudaStream_t st);

// vetting (stamps + CNN)
int cnn_param_count();
size_t cnn_smem_bytes();
int cnn_backward_blocks(int64_t n, int n_sms);
// Compacted track positions of candidates: pos[i * n_exp + k], k < cnt[i],
// = (ix << 16 | exposure, iy) of the k-th exposure (epoch order) whose
// nearest pixel is inside the image (exposures < 2^16, widths <= 2^15).
cudaError_t launch_stamp_positions(const double* states, int64_t n, double t0, double t_ref, bool state_df,
                                   const int64_t* cand, int64_t n_cand, const ExpDev* ex, int32_t n_exp,
                                   Phys ph, int2* pos, int* cnt, unsigned long long* counters,
                                   cudaStream_t st);
cudaError_t launch_stamps(const int2* pos, const int* pos_cnt, int64_t n_cand, const ExpDev* ex,
                          int32_t n_exp, const void* planes, int plane_type, float* out_f32,
                          __nv_bfloat16* out_bf16, int n_sms, cudaStream_t st);
// Iterative-MAD noise estimate (k_mad.cu): one image and its round state.
struct MadImage {
  const float* x;
  int64_t n;
};
struct MadState {
  int32_t done, round, rounds;
  int32_t what;              // selection in progress: 0 median of S_i, 1 its MAD
  int32_t phase;             // next pass: 1 histogram, 2 compaction of the band
  int32_t level;             // histogram level of this selection (0: the window)
  int32_t shift;             // histogram bins are 2^shift keys wide
  int32_t passes;            // image passes so far
  uint32_t lo;               // first key of the first inner bin
  uint32_t blo, bhi;         // band: only keys in [blo, bhi] are counted or copied
  uint32_t slo, shi;         // speculative copy range of a histogram pass (none if slo > shi)
  uint32_t pad_;
  long long n_kept;          // |S_i|
  unsigned long long krem;   // rank wanted among the keys of the band
  float m_prev, thr_prev;    // S_i = { |x - m_prev| <= thr_prev } (round > 0)
  float m_cur;               // median of this round
  float m_last, sigma;       // the last completed round's (median, sigma)
  float rho[2];              // keys per key unit near the last median / MAD
  uint32_t kpred[2];         // key of the last median / MAD
};
constexpr int kNoiseMaxRounds = 10;
// keys a selection may copy out per image (the buffer holds cap per image)
constexpr uint32_t kMadCap = 1u << 18;
MadState mad_initial_state();
// n_pairs (pass, pick) launches of the iterative-MAD selection (k_mad.cu)
cudaError_t launch_mad_passes(const MadImage* imgs, MadState* st, uint32_t* hist, uint32_t* cnt, uint32_t* buf,
                              uint32_t cap, int n_images, int64_t max_pixels, int max_rounds, int n_pairs,
                              cudaStream_t stream);
size_t mad_hist_words(int n_images);

size_t trim_scratch_words(int64_t n_cand, int32_t n_exp);
cudaError_t launch_trim(const int2* pos, const int* pos_cnt, int64_t n_cand, const ExpDev* ex, int32_t n_exp,
                        const void* planes,
                        int plane_type, float kappa, int32_t max_iter, int32_t min_obs, uint32_t* keep_bits,
                        float* nu_out, int32_t* n_out, float* psi_out, float* phi_out, int n_sms,
                        cudaStream_t st);
cudaError_t launch_cnn_forward_tc(const float* th, const __nv_bfloat16* x, int64_t n, float* logits,
                                  int* err, int n_sms, cudaStream_t st, int withhold_first_layer = 0);
cudaError_t launch_cnn_backward(const float* th, const __nv_bfloat16* x, const float* labels,
                                int64_t n, float* grad, float* loss_sum, float* a1_scratch,
                                float* logits, int n_sms, cudaStream_t st);
cudaError_t launch_sigmoid(float* z, int64_t n, cudaStream_t st);
cudaError_t launch_adam(float* th, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, int step, cudaStream_t st);

// top-k
struct TopkScratch {
  unsigned int* hist;          // 256 bins
  unsigned int* sel_state;     // [prefix, k_remaining, n_less, mask]
  unsigned int* block_counts;  // 2 * max_blocks
  unsigned long long* items;   // k composite keys (key32 << 32 | idx32)
  int max_blocks;
};
size_t topk_scratch_bytes(int64_t n, int64_t k);
cudaError_t launch_topk(const float* snr, int64_t n, int64_t k, void* scratch, size_t scratch_bytes,
                        int64_t* idx_out, float* snr_out, int* launches, cudaStream_t st);

}  // namespace ndt
