// Host check of the double-float helpers of the stacking kernel against long
// double: the FP64 split, the dot product, the quotient and the floor, and
// the whole TAN projection at 0.2 arcsec pixels (1e6 px per radian) against
// its long double value.  Prints the worst errors and exits non-zero
// when one exceeds its bound.
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <random>

#include "dfloat.cuh"

using ndt::dfloat;
typedef long double LD;

static LD val(dfloat a) { return (LD)a.h + (LD)a.l; }

int main() {
  std::mt19937_64 rng(4242);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  int bad = 0;
  // 1. split: hi is d2f_rn(v) and hi + lo = v to 2^-48 relative
  double worst_split = 0.0;
  for (int i = 0; i < 2000000; ++i) {
    const double v = std::ldexp(U(rng), (int)(rng() % 120) - 60);
    const dfloat s = ndt::split_df(v);
    if (s.h != ndt::d2f_rn(v)) { std::printf("split: hi mismatch at %.17g\n", v); return 1; }
    // (below 2^-73 lo is 0 by design: negligible next to any term it meets)
    if (std::fabs(v) >= std::ldexp(1.0, -72))
      worst_split = std::fmax(worst_split, (double)(std::fabs(val(s) - (LD)v) / std::fabs((LD)v)));
    if (std::fabs((LD)s.l) > std::ldexp(std::fabs((LD)s.h), -23)) { std::printf("split: lo too big\n"); return 1; }
  }
  if (worst_split > std::ldexp(1.0, -48)) ++bad;
  std::printf("split: worst relative error %.3g (bound 2^-48 = %.3g)\n", worst_split, std::ldexp(1.0, -48));
  // 2. dot products with cancellation
  double worst_dot = 0.0;
  for (int i = 0; i < 1000000; ++i) {
    double a[3], b[3];
    dfloat A[3], B[3];
    LD exact = 0, mag = 0;
    for (int k = 0; k < 3; ++k) {
      a[k] = (U(rng) + (U(rng) > 0 ? 1e-3 : -1e-3)) * std::ldexp(1.0, (int)(rng() % 8));
      b[k] = U(rng) * 1e6;
      A[k] = ndt::split_df(a[k]);
      B[k] = ndt::split_df(b[k]);
    }
    if (i % 2) a[2] = -(a[0] * b[0] + a[1] * b[1]) / b[2], A[2] = ndt::split_df(a[2]);   // near-orthogonal
    for (int k = 0; k < 3; ++k) {
      exact += (LD)a[k] * (LD)b[k];
      mag += std::fabs((LD)a[k] * (LD)b[k]);
    }
    const dfloat d = ndt::df_dot3(A, B);
    worst_dot = std::fmax(worst_dot, (double)(std::fabs(val(d) - exact) / mag));
  }
  // about six roundings of order 2^-48 of the terms: 2^-45.4; bound with a factor 2
  if (worst_dot > std::ldexp(1.0, -44)) ++bad;
  std::printf("dot: worst error / sum|a b| %.3g (bound 2^-44 = %.3g)\n", worst_dot, std::ldexp(1.0, -44));
  // 3. TAN projection: x + 1/2 = crpix_h + (rho . ax) / (rho . p0), formed as
  //    the kernel does, (rho . (ax + crpix_h p0)) / (rho . p0)
  double worst_px = 0.0;
  const double ppr = 1.0 / (0.2 / 3600.0 * M_PI / 180.0);   // px per radian at 0.2 arcsec
  for (int i = 0; i < 1000000; ++i) {
    // tangent point p0, orthonormal basis (e1, e2) of the tangent plane
    double p0[3] = {U(rng), U(rng), U(rng)};
    const double n0 = std::sqrt(p0[0] * p0[0] + p0[1] * p0[1] + p0[2] * p0[2]);
    for (double& c : p0) c /= n0;
    double e1[3] = {-p0[1], p0[0], 0.0};
    const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
    for (double& c : e1) c /= n1;
    const double e2[3] = {p0[1] * e1[2] - p0[2] * e1[1], p0[2] * e1[0] - p0[0] * e1[2], p0[0] * e1[1] - p0[1] * e1[0]};
    double ax[3], ay[3];
    for (int k = 0; k < 3; ++k) {
      ax[k] = -ppr * e1[k];
      ay[k] = ppr * e2[k];
    }
    const double crh[2] = {2048.5 + 0.25 * U(rng), 2048.5 + 0.25 * U(rng)};
    // rho within ~1.5 deg of the tangent point, 0.02 to 60 AU away
    const double dist = std::exp(std::log(0.02) + (std::log(60.0) - std::log(0.02)) * 0.5 * (U(rng) + 1.0));
    const double ox = 0.026 * U(rng), oy = 0.026 * U(rng);
    double rho[3];
    for (int k = 0; k < 3; ++k) rho[k] = dist * (p0[k] + ox * e1[k] + oy * e2[k]);
    // the kernel's rows carry the reference pixel: axc = ax + crh[0] p0
    dfloat R[3], P[3], AX[3], AY[3];
    for (int k = 0; k < 3; ++k) {
      R[k] = ndt::split_df(rho[k]);
      P[k] = ndt::split_df(p0[k]);
      AX[k] = ndt::split_df((double)((LD)ax[k] + (LD)crh[0] * (LD)p0[k]));
      AY[k] = ndt::split_df((double)((LD)ay[k] + (LD)crh[1] * (LD)p0[k]));
    }
    const dfloat den = ndt::df_dot3(R, P);
    const dfloat xh = ndt::df_div(ndt::df_dot3(R, AX), den);
    const dfloat yh = ndt::df_div(ndt::df_dot3(R, AY), den);
    LD D = 0, NX = 0, NY = 0;
    for (int k = 0; k < 3; ++k) {
      D += (LD)rho[k] * (LD)p0[k];
      NX += (LD)rho[k] * (LD)ax[k];
      NY += (LD)rho[k] * (LD)ay[k];
    }
    const LD xr = (LD)crh[0] + NX / D, yr = (LD)crh[1] + NY / D;
    worst_px = std::fmax(worst_px, (double)std::fmax(std::fabs(val(xh) - xr), std::fabs(val(yh) - yr)));
    // floor agrees with the exact value unless that is within 1e-8 px of an integer
    const int fx = ndt::df_floor(xh);
    const LD flx = std::floor(xr);
    if (fx != (int)flx && std::fabs(xr - std::round(xr)) > 5e-8L) {
      std::printf("floor mismatch: %d vs %.12Lf\n", fx, xr);
      return 1;
    }
  }
  // ~2^-47 relative per term of rho . ax, whose terms are ~|rho| ppr: about
  // 3 2^-47 ppr = 2e-8 px at 1e6 px/rad, 50x below the 1e-6 px band inside
  // which the parity tests accept either neighbouring pixel
  if (worst_px > 5e-8) ++bad;
  std::printf("projection: worst |x - x_exact| %.3g px (bound 5e-8 px)\n", worst_px);
  // 4. floor at integer boundaries: hi an integer, lo of either sign
  for (int n = -3000; n <= 3000; ++n) {
    const float h = (float)n;
    const float eps[4] = {0.0f, 1e-6f, -1e-6f, -1e-12f};
    for (float e : eps) {
      const dfloat x = ndt::fast_two_sum(h, e);
      const int want = (int)std::floor((LD)x.h + (LD)x.l);
      if (ndt::df_floor(x) != want) {
        std::printf("floor at %d%+g: %d vs %d\n", n, (double)e, ndt::df_floor(x), want);
        return 1;
      }
    }
  }
  // 5. increments by products (the two-body and light-time updates):
  //    x + (a b + c), x + (a u + b w), x (1 + f), against long double, with
  //    increments from 1 down to 1e-12 of x (the _small forms) and of any
  //    size (the general ones); error relative to |x| + |increments|
  double worst_inc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < 1000000; ++i) {
    const double xv = U(rng) * std::ldexp(1.0, (int)(rng() % 12) - 6);
    const double sm = std::ldexp(1.0, -(int)(rng() % 40));           // |increment| / |x| scale
    const double big = std::ldexp(1.0, (int)(rng() % 40) - 20);      // any ratio
    const double av = U(rng) * sm, bv = xv * U(rng), cv = xv * sm * 1e-8 * U(rng);
    const double a2 = U(rng) * big, u2 = xv * U(rng), b2 = U(rng) * big, w2 = U(rng);
    const dfloat X = ndt::split_df(xv), A = ndt::split_df(av), B = ndt::split_df(bv);
    const dfloat A2 = ndt::split_df(a2), U2 = ndt::split_df(u2), B2 = ndt::split_df(b2), W2 = ndt::split_df(w2);
    const float c = (float)cv, f = (float)(0.5 * U(rng) * sm);
    const LD x = val(X), a = val(A), b = val(B);
    // |a b| <= |x| here: the _small form applies
    LD want = x + (a * b + (LD)c);
    LD mag = std::fabs(x) + std::fabs(a * b) + std::fabs((LD)c);
    worst_inc[0] = std::fmax(worst_inc[0], (double)(std::fabs(val(ndt::df_add_prod_small(X, A, B, c)) - want) / mag));
    worst_inc[1] = std::fmax(worst_inc[1], (double)(std::fabs(val(ndt::df_add_prod(X, A, B, c)) - want) / mag));
    // general magnitudes
    want = x + (val(A2) * val(U2) + val(B2) * val(W2));
    mag = std::fabs(x) + std::fabs(val(A2) * val(U2)) + std::fabs(val(B2) * val(W2));
    worst_inc[2] = std::fmax(worst_inc[2], (double)(std::fabs(val(ndt::df_add_prod2(X, A2, U2, B2, W2)) - want) / mag));
    want = x * (1.0L + (LD)f);
    worst_inc[3] = std::fmax(worst_inc[3], (double)(std::fabs(val(ndt::df_add_scaled_small(X, f)) - want) / std::fabs(x)));
  }
  // a b + c with |c| <= |a b| / 2 (the light time |d| / c + corr)
  double worst_fma = 0.0;
  for (int i = 0; i < 1000000; ++i) {
    const dfloat A = ndt::split_df(U(rng) * std::ldexp(1.0, (int)(rng() % 20) - 10));
    const dfloat B = ndt::split_df(U(rng) * std::ldexp(1.0, (int)(rng() % 20) - 10));
    const LD ab = val(A) * val(B);
    const float c = (float)(0.5 * (double)ab * U(rng) * std::ldexp(1.0, -(int)(rng() % 30)));
    const LD want = ab + (LD)c;
    worst_fma = std::fmax(worst_fma, (double)(std::fabs(val(ndt::df_fma_small(A, B, c)) - want) / std::fabs(ab)));
  }
  if (!(worst_fma <= std::ldexp(1.0, -45))) ++bad;
  std::printf("a b + c: worst error / |a b| %.3g (bound 2^-45 = %.3g)\n", worst_fma, std::ldexp(1.0, -45));
  const char* inc_names[4] = {"x + (a b + c), small", "x + (a b + c)", "x + (a u + b w)", "x (1 + f)"};
  for (int k = 0; k < 4; ++k) {
    // a handful of roundings of order 2^-48 of the largest term
    if (!(worst_inc[k] <= std::ldexp(1.0, -45))) ++bad;
    std::printf("%s: worst error / magnitude %.3g (bound 2^-45 = %.3g)\n", inc_names[k], worst_inc[k],
                std::ldexp(1.0, -45));
  }
  std::printf("%s\n", bad ? "FAILED" : "ok");
  return bad ? 1 : 0;
}
