// Host check of the integer-pipe conversions used by the stacking kernel:
// each helper against the host's own conversion over special
// values, values next to every rounding boundary that matters, and random bit
// patterns.  Prints the number of cases checked and exits non-zero on the
// first mismatch.
#include <cinttypes>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <random>
#include <vector>

#include "bitconv.cuh"

static long long n_checked = 0;

static double dbl(uint64_t b) { double d; std::memcpy(&d, &b, 8); return d; }
static uint64_t bits(double d) { uint64_t b; std::memcpy(&b, &d, 8); return b; }
static uint32_t fbits(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

static bool fail(const char* what, double d, double got, double want) {
  std::printf("MISMATCH %s: input %.17g (0x%016" PRIx64 ") got %.17g want %.17g\n", what, d, bits(d),
              got, want);
  return false;
}

// truncation toward zero to FP32, for inputs in the normal FP32 range
static bool check_trunc(double d) {
  ++n_checked;
  const float f = ndt::d2f_trunc(d);
  if (std::isnan(d)) return std::isinf(f) ? true : fail("d2f_trunc nan", d, f, INFINITY);
  const double a = std::fabs(d);
  if (a < 0x1p-126) return (f == 0.0f && std::signbit(f) == std::signbit(d)) ? true : fail("d2f_trunc small", d, f, 0.0);
  if (a >= 0x1p128) return (std::isinf(f) && std::signbit(f) == std::signbit(d)) ? true : fail("d2f_trunc big", d, f, d);
  const double fa = std::fabs((double)f);
  const float up = std::nextafter(std::fabs(f), INFINITY);
  if (std::signbit(f) != std::signbit(d) || fa > a || (double)up <= a) return fail("d2f_trunc", d, f, d);
  return true;
}

// round to nearest, ties away from zero; equals the host's round-to-nearest-
// even conversion except at exact ties
static bool check_rn(double d) {
  ++n_checked;
  const float f = ndt::d2f_rn(d);
  const double a = std::fabs(d);
  if (std::isnan(d) || a < 0x1p-126 || a >= 0x1p127) return true;   // outside the helper's claim
  const float h = (float)d;
  if (f == h) return true;
  // differing results must be a tie, resolved away from zero
  const double lo = std::fabs((double)h), hi = std::fabs((double)f);
  if (hi > lo && (a - lo) == (hi - a) && std::signbit(f) == std::signbit(d)) return true;
  return fail("d2f_rn", d, f, h);
}

static bool check_exact(float f) {
  ++n_checked;
  const double d = ndt::f2d_exact(f);
  if (std::isnan(f)) return std::isnan(d) ? true : fail("f2d_exact nan", f, d, f);
  if (std::fpclassify(f) == FP_SUBNORMAL) return d == 0.0 ? true : fail("f2d_exact subnormal", f, d, 0.0);
  if (bits(d) != bits((double)f)) return fail("f2d_exact", f, d, (double)f);
  return true;
}

static bool check_all(double d) {
  return check_trunc(d) && check_rn(d) && check_exact((float)d);
}

int main() {
  std::vector<double> special = {0.0, -0.0, 0.5, -0.5, 1.0, -1.0, 1.5, -1.5, 2.5, -2.5,
                                 std::numeric_limits<double>::denorm_min(),
                                 -std::numeric_limits<double>::denorm_min(),
                                 std::numeric_limits<double>::min(), INFINITY, -INFINITY, NAN,
                                 0x1p30, -0x1p30, 0x1p-11, -0x1p-11, 0x1p-12, -0x1p-12,
                                 0x1p-126, 0x1p127, 0x1p128, -0x1p128, 4095.5, 4096.0, 1e300};
  for (double d : special) {
    if (!check_all(d)) return 1;
    if (!check_all(std::nextafter(d, INFINITY)) || !check_all(std::nextafter(d, -INFINITY))) return 1;
  }
  // integers and half-integers of the image range, with their neighbours
  for (int i = -70000; i <= 70000; ++i) {
    for (double base : {(double)i, i + 0.5}) {
      double d = base;
      for (int k = 0; k < 3; ++k) d = std::nextafter(d, -INFINITY);
      for (int k = 0; k < 7; ++k, d = std::nextafter(d, INFINITY))
        if (!check_all(d)) return 1;
    }
  }
  // values around 2^29 and 2^30 (large pixel coordinates)
  for (double base : {0x1p30, -0x1p30, 0x1p29, -0x1p29}) {
    double d = base;
    for (int k = 0; k < 4; ++k) d = std::nextafter(d, -INFINITY);
    for (int k = 0; k < 9; ++k, d = std::nextafter(d, INFINITY))
      if (!check_all(d)) return 1;
  }
  // FP32 rounding boundaries: every FP64 value next to a tie between two
  // FP32 neighbours, over all FP32 exponents of the normal range
  std::mt19937_64 rng(20250311);
  for (int e = -125; e < 127; ++e) {
    for (int r = 0; r < 200; ++r) {
      const uint32_t m = (uint32_t)(rng() & 0x7FFFFFu);
      const float f = std::ldexp(1.0f + m * 0x1p-23f, e);
      const double tie = (double)f + std::ldexp(1.0, e - 24);
      for (double d : {tie, std::nextafter(tie, 0.0), std::nextafter(tie, INFINITY), -tie, (double)f, -(double)f})
        if (!check_all(d)) return 1;
    }
  }
  // random bit patterns (all exponents), and random pixel coordinates
  for (int r = 0; r < 4000000; ++r) {
    if (!check_all(dbl(rng()))) return 1;
    const double x = std::ldexp((double)(int64_t)rng(), -(int)(rng() % 80));   // |x| up to 2^63
    if (!check_all(x)) return 1;
    const double px = (double)(rng() % 20000) / 4.0 - 2500.0 + std::ldexp((double)(rng() >> 11), -60);
    if (!check_all(px) || !check_all(-px)) return 1;
  }
  // every FP32 exponent and sign for the widening conversion
  for (uint32_t hi = 0; hi < 512; ++hi) {
    for (int r = 0; r < 64; ++r) {
      const uint32_t u = (hi << 23) | (uint32_t)(rng() & 0x7FFFFFu);
      float f;
      std::memcpy(&f, &u, 4);
      if (!check_exact(f)) return 1;
    }
  }
  (void)fbits;
  std::printf("ok %lld\n", n_checked);
  return 0;
}
