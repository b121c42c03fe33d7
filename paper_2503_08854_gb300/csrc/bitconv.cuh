// Number conversions on the integer pipe, from the IEEE-754 bit patterns.
//
// The stacking kernel is bound by the FP64 pipe, which on this GPU also
// executes every conversion that reads or writes an FP64 value.  These
// helpers do the same conversions with integer and logic instructions, which
// run on other pipes with plenty of spare issue slots.  They compile for the
// host too (plain C++), so that they can be checked there against the
// hardware conversions.
#pragma once

#include <climits>
#include <cstring>

#ifdef __CUDACC__
#define NDT_HD __host__ __device__ __forceinline__
#else
#define NDT_HD inline
#endif

namespace ndt {

NDT_HD unsigned hi_word(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(d);
#else
  unsigned long long b;
  std::memcpy(&b, &d, 8);
  return (unsigned)(b >> 32);
#endif
}

NDT_HD unsigned lo_word(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(d);
#else
  unsigned long long b;
  std::memcpy(&b, &d, 8);
  return (unsigned)b;
#endif
}

NDT_HD double from_words(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const unsigned long long b = ((unsigned long long)hi << 32) | lo;
  double d;
  std::memcpy(&d, &b, 8);
  return d;
#endif
}

NDT_HD float float_of_bits(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

NDT_HD unsigned bits_of_float(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}

// FP64 -> FP32 by truncation toward zero (exponent rebias and mantissa
// shift).  Relative error < 2^-23; magnitudes below 2^-126 become 0, above
// FP32 range infinity (NaN too).
NDT_HD float d2f_trunc(double d) {
  const unsigned hi = hi_word(d), lo = lo_word(d);
  const unsigned sign = hi & 0x80000000u;
  const int ex = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (ex <= 0) return float_of_bits(sign);
  if (ex >= 255) return float_of_bits(sign | 0x7F800000u);
  return float_of_bits(sign | ((unsigned)ex << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// FP64 -> FP32 rounded to nearest, ties away from zero: half an FP32 ulp is
// added to the FP64 bit pattern (a carry moves into the exponent as it
// should), then the pattern is truncated.  Relative error <= 2^-24, as for
// the hardware conversion (which differs only at exact ties).
NDT_HD float d2f_rn(double d) {
  const unsigned lo = lo_word(d);
  const unsigned lo2 = lo + (1u << 28);
  const unsigned hi2 = hi_word(d) + (lo2 < lo ? 1u : 0u);
  return d2f_trunc(from_words(hi2, lo2));
}

// FP32 -> FP64 exactly; subnormal FP32 values become 0, infinities and NaNs
// stay so.
NDT_HD double f2d_exact(float f) {
  const unsigned u = bits_of_float(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned eh = e == 0u ? 0u : (e == 255u ? 0x7FFu : e + 896u);   // 896 = 1023 - 127
  const unsigned hi = sign | (eh << 20) | (e == 0u ? 0u : m >> 3);
  const unsigned lo = e == 0u ? 0u : m << 29;
  return from_words(hi, lo);
}

}  // namespace ndt
