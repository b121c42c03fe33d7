// Double-float arithmetic: a value carried as an unevaluated sum hi + lo of
// two FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits, with
// error-free transformations built on the FP32 FMA (Dekker 1971; Knuth, TAOCP
// vol. 2, sec. 4.2.2; Ogita, Rump & Oishi 2005).  The stacking kernel uses it
// for the TAN projection: a one-shot, non-accumulating computation whose
// nearest-pixel decision needs ~1e-9 px, which 48 bits give, while every FP64
// instruction it would otherwise take is on the pipe that bounds the kernel.
// Compiles for the host too, where tests check it against long double.
#pragma once

#include <cmath>

#include "bitconv.cuh"

namespace ndt {

struct dfloat {
  float h, l;
};

// correctly rounded FP32 operations that the compiler may not contract
NDT_HD float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float s = a + b;
  return s;
#endif
}
NDT_HD float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  volatile float s = a - b;
  return s;
#endif
}
NDT_HD float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  volatile float s = a * b;
  return s;
#endif
}
NDT_HD float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}
// 1/a to about an ulp (the hardware approximation on the device, one
// instruction; subnormal inputs and results flush to zero): the quotient
// and square-root corrections below need no more
NDT_HD float rcp_approx(float a) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
#else
  return 1.0f / a;
#endif
}

// s + e = a + b exactly (Knuth's two-sum)
NDT_HD dfloat two_sum(float a, float b) {
  const float s = add_rn(a, b);
  const float bb = sub_rn(s, a);
  const float e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
  return {s, e};
}
// s + e = a + b exactly when |a| >= |b| or a == 0
NDT_HD dfloat fast_two_sum(float a, float b) {
  const float s = add_rn(a, b);
  return {s, sub_rn(b, sub_rn(s, a))};
}
// p + e = a b exactly (FMA two-product)
NDT_HD dfloat two_prod(float a, float b) {
  const float p = mul_rn(a, b);
  return {p, fma_rn(a, b, -p)};
}

// An FP64 value as hi + lo on the integer pipe: hi = d2f_rn(v) (24 bits of
// the significand, rounded) and lo = the remaining 29 bits of the significand
// rounded to FP32, so hi + lo = v to 2^-48 relative.  lo is 0 when v is zero,
// below 2^-73 in magnitude (negligible here) or outside the FP32 range.
NDT_HD dfloat split_df(double v) {
  const float h = d2f_rn(v);
  const unsigned hi = hi_word(v), lo32 = lo_word(v);
  const int ex = (int)((hi >> 20) & 0x7FFu);
  const int r29 = (int)(lo32 & 0x1FFFFFFFu);                 // significand bits below hi's
  const int rem = r29 >= (1 << 28) ? r29 - (1 << 29) : r29;  // d2f_rn rounded up at >= half
  const int se = ex - 1075 + 127;                           // FP32 exponent of 2^(ex - 1075)
  float l = 0.0f;
  if (ex != 0 && se > 0 && se < 255) l = (float)rem * float_of_bits((unsigned)se << 23);
  if (hi & 0x80000000u) l = -l;
  return {h, l};
}

// a . b for 3-vectors of double-floats; error ~2^-47 sum |a_i b_i|
NDT_HD dfloat df_dot3(const dfloat a[3], const dfloat b[3]) {
  dfloat p[3];
  float low = 0.0f;
  for (int i = 0; i < 3; ++i) {
    p[i] = two_prod(a[i].h, b[i].h);
    low = fma_rn(a[i].h, b[i].l, fma_rn(a[i].l, b[i].h, add_rn(low, p[i].l)));
  }
  const dfloat s1 = two_sum(p[0].h, p[1].h);
  const dfloat s2 = two_sum(s1.h, p[2].h);
  return fast_two_sum(s2.h, add_rn(low, add_rn(s1.l, s2.l)));
}

// n / d (d != 0); relative error ~2^-45
NDT_HD dfloat df_div(dfloat n, dfloat d) {
  const float r = rcp_approx(d.h);
  const float q1 = mul_rn(n.h, r);
  const dfloat p = two_prod(q1, d.h);
  // n - q1 d: n.h - p.h is exact (Sterbenz), the rest are small corrections
  const float rem = fma_rn(-q1, d.l, sub_rn(add_rn(sub_rn(n.h, p.h), n.l), p.l));
  return fast_two_sum(q1, mul_rn(rem, r));
}

// sqrt(a) to about an ulp (the hardware approximation on the device): the
// Newton correction of df_sqrt removes its error
NDT_HD float sqrt_rn(float a) {
#ifdef __CUDA_ARCH__
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
#else
  return std::sqrt(a);
#endif
}

// a b; relative error ~2^-46
NDT_HD dfloat df_mul(dfloat a, dfloat b) {
  const dfloat p = two_prod(a.h, b.h);
  return fast_two_sum(p.h, fma_rn(a.h, b.l, fma_rn(a.l, b.h, p.l)));
}

// sqrt(a) for a > 0: the FP32 root s and one Newton correction
// (a - s^2) / (2 s), with s^2 formed exactly; relative error ~2^-46
NDT_HD dfloat df_sqrt(dfloat a) {
  const float s = sqrt_rn(a.h);
  const dfloat sq = two_prod(s, s);
  const float res = add_rn(sub_rn(sub_rn(a.h, sq.h), sq.l), a.l);
  return fast_two_sum(s, mul_rn(res, 0.5f * rcp_approx(s)));
}

NDT_HD dfloat df_add(dfloat a, dfloat b) {
  const dfloat s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, add_rn(s.l, add_rn(a.l, b.l)));
}

NDT_HD dfloat df_neg(dfloat a) { return {-a.h, -a.l}; }

NDT_HD dfloat df_sub(dfloat a, dfloat b) { return df_add(a, df_neg(b)); }

// a + b for an FP32 b
NDT_HD dfloat df_add_f(dfloat a, float b) {
  const dfloat s = two_sum(a.h, b);
  return fast_two_sum(s.h, add_rn(s.l, a.l));
}

// a b for an FP32 b; relative error ~2^-47
NDT_HD dfloat df_mul_f(dfloat a, float b) {
  const dfloat p = two_prod(a.h, b);
  return fast_two_sum(p.h, fma_rn(a.l, b, p.l));
}

// Increments of a double-float by products: x + (a b + c), with the product
// a.h b.h formed exactly, its cross terms and the FP32 term c gathered in the
// low part, and one normalisation at the end (16 FP32 instructions, where a
// product, a sum and a second sum take 29).  c is a correction below 2^-24 of
// |x| + |a b| (it is rounded with the low part); the error is then ~2^-47
// (|x| + |a b|).
// The _small form needs |a b| <= |x|, which a vector component need not meet
// even when the vector's increment is small (a component of x may vanish):
// it serves updates of one quantity by a fraction of itself.  The others
// hold for any magnitudes.
NDT_HD dfloat df_add_prod_small(dfloat x, dfloat a, dfloat b, float c) {
  const dfloat p = two_prod(a.h, b.h);
  const float lo = fma_rn(a.h, b.l, fma_rn(a.l, b.h, add_rn(p.l, c)));
  const dfloat s = fast_two_sum(x.h, p.h);
  return fast_two_sum(s.h, add_rn(s.l, add_rn(x.l, lo)));
}
NDT_HD dfloat df_add_prod(dfloat x, dfloat a, dfloat b, float c) {
  const dfloat p = two_prod(a.h, b.h);
  const float lo = fma_rn(a.h, b.l, fma_rn(a.l, b.h, add_rn(p.l, c)));
  const dfloat s = two_sum(x.h, p.h);
  return fast_two_sum(s.h, add_rn(s.l, add_rn(x.l, lo)));
}
// x + (a u + b w)
NDT_HD dfloat df_add_prod2(dfloat x, dfloat a, dfloat u, dfloat b, dfloat w) {
  const dfloat p = two_prod(a.h, u.h);
  const dfloat q = two_prod(b.h, w.h);
  const dfloat t = two_sum(p.h, q.h);
  const float lo =
      fma_rn(a.h, u.l, fma_rn(a.l, u.h, fma_rn(b.h, w.l, fma_rn(b.l, w.h, add_rn(p.l, add_rn(q.l, t.l))))));
  const dfloat s = two_sum(x.h, t.h);
  return fast_two_sum(s.h, add_rn(s.l, add_rn(x.l, lo)));
}
// a b + c for an FP32 c with |c| <= |a b| / 2
NDT_HD dfloat df_fma_small(dfloat a, dfloat b, float c) {
  const dfloat p = two_prod(a.h, b.h);
  const dfloat s = fast_two_sum(p.h, c);
  return fast_two_sum(s.h, fma_rn(a.h, b.l, fma_rn(a.l, b.h, add_rn(p.l, s.l))));
}
// x (1 + f) for an FP32 f with |f| <= 1/2
NDT_HD dfloat df_add_scaled_small(dfloat x, float f) {
  const dfloat p = two_prod(x.h, f);
  const float lo = fma_rn(x.l, f, p.l);
  const dfloat s = fast_two_sum(x.h, p.h);
  return fast_two_sum(s.h, add_rn(s.l, add_rn(x.l, lo)));
}

// a 2^k (s = 2^k): exact
NDT_HD dfloat df_scale2(dfloat a, float s) { return {mul_rn(a.h, s), mul_rn(a.l, s)}; }

// floor(hi + lo) for a normalised pair: floor(hi), one lower when hi is an
// integer and lo < 0; INT_MIN when |hi| >= 2^30 or not finite
NDT_HD int df_floor(dfloat x) {
  if (!(std::fabs(x.h) < 1073741824.0f)) return INT_MIN;
  const float f = std::floor(x.h);
  return (int)f - ((f == x.h && x.l < 0.0f) ? 1 : 0);
}

}  // namespace ndt
