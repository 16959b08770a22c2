// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  GB300 issues FP32
// at roughly 70x its FP64 rate, so the mixed-precision path carries the
// quantities that need more than FP32 -- phase-space momenta, resonant
// invariants -- as double-floats on the FP32 pipe instead of in FP64.
//
// Building blocks are the error-free transformations of Knuth (TwoSum),
// Dekker (FastTwoSum) and the FMA form of TwoProduct, combined as in Joldes,
// Muller, Popescu, "Tight and rigorous error bounds for basic building blocks
// of double-word arithmetic", ACM TOMS 44 (2017) (sum: AccurateDWPlusDW;
// product: DWTimesDW with an FMA).  The logarithm is Tang's table-driven
// method (ACM TOMS 16 (1990) 378) with a 128-entry table and a short log1p
// series; sine and cosine of pi x use a 257-entry table of pi j/128 and
// Taylor series on |theta| < pi/256.  Tables: dfloat_tables.h (generated).
#pragma once
#include <cstdint>
#include <cstring>
#include <cmath>

#include "dfloat_tables.h"

#define DF_HD __host__ __device__ __forceinline__

namespace me {

struct df {
  float hi, lo;
};

#ifdef __CUDA_ARCH__
DF_HD float df_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
DF_HD float df_add_rn(float a, float b) { return __fadd_rn(a, b); }
DF_HD float df_sub_rn(float a, float b) { return __fsub_rn(a, b); }
DF_HD float df_mul_rn(float a, float b) { return __fmul_rn(a, b); }
#else
DF_HD float df_fma(float a, float b, float c) { return fmaf(a, b, c); }
DF_HD float df_add_rn(float a, float b) { volatile float s = a + b; return s; }
DF_HD float df_sub_rn(float a, float b) { volatile float s = a - b; return s; }
DF_HD float df_mul_rn(float a, float b) { volatile float s = a * b; return s; }
#endif

// Knuth TwoSum: s + e = a + b exactly
DF_HD df two_sum(float a, float b) {
  const float s = df_add_rn(a, b);
  const float bb = df_sub_rn(s, a);
  const float e = df_add_rn(df_sub_rn(a, df_sub_rn(s, bb)), df_sub_rn(b, bb));
  return df{s, e};
}
// Dekker FastTwoSum (|a| >= |b|)
DF_HD df fast_two_sum(float a, float b) {
  const float s = df_add_rn(a, b);
  const float e = df_sub_rn(b, df_sub_rn(s, a));
  return df{s, e};
}
// TwoProduct with an FMA: p + e = a b exactly
DF_HD df two_prod(float a, float b) {
  const float p = df_mul_rn(a, b);
  return df{p, df_fma(a, b, -p)};
}

DF_HD df dfs(float a) { return df{a, 0.0f}; }
DF_HD df operator-(df a) { return df{-a.hi, -a.lo}; }
DF_HD df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  const df v = fast_two_sum(s.hi, df_add_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, df_add_rn(t.lo, v.lo));
}
DF_HD df operator-(df a, df b) { return a + (-b); }
// Sloppy sum (Dekker; SloppyDWPlusDW in Joldes, Muller, Popescu): one TwoSum, error
// below 2^-47 (|a| + |b|) rather than 2^-47 |a + b|.  For sums whose accuracy is
// needed relative to their operands' scale (momentum components against sqrt(s)).
DF_HD df sadd(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, df_add_rn(s.lo, df_add_rn(a.lo, b.lo)));
}
DF_HD df ssub(df a, df b) { return sadd(a, df{-b.hi, -b.lo}); }
DF_HD df operator*(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  const float t = df_fma(a.hi, b.lo, df_mul_rn(a.lo, b.hi));
  return fast_two_sum(p.hi, df_add_rn(p.lo, t));
}
DF_HD df operator*(df a, float b) {
  const df p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, df_fma(a.lo, b, p.lo));
}
DF_HD df operator+(df a, float b) {
  const df s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, df_add_rn(s.lo, a.lo));
}
DF_HD df sqr(df a) {
  const df p = two_prod(a.hi, a.hi);
  return fast_two_sum(p.hi, df_fma(df_add_rn(a.hi, a.hi), a.lo, p.lo));
}
// 1/x to about one ulp: on the device the fast reciprocal and one Newton step
// (FMA form), on the host IEEE division.  Normal, finite x.
DF_HD float df_recip(float x) {
#ifdef __CUDA_ARCH__
  const float r = __fdividef(1.0f, x);
  return df_fma(r, df_fma(-x, r, 1.0f), r);
#else
  return 1.0f / x;
#endif
}
// a / b: an FP32 quotient corrected by the double-float residual, both from one
// reciprocal of b.hi (the residual a - b q1 is formed exactly, so q1 need not be
// correctly rounded; q2 carries an error of about one ulp of itself, 2^-47 of a / b)
DF_HD df operator/(df a, df b) {
  const float rb = df_recip(b.hi);
  const float q1 = df_mul_rn(a.hi, rb);
  const df r = a - b * q1;
  const float q2 = df_mul_rn(r.hi, rb);
  return fast_two_sum(q1, q2);
}
DF_HD df df_sqrt(df a) {
  if (!(a.hi > 0.0f)) return df{0.0f, 0.0f};
  const float s = sqrtf(a.hi);
  const df r = a - two_prod(s, s);
  return fast_two_sum(s, r.hi / (2.0f * s));
}
DF_HD float to_float(df a) { return df_add_rn(a.hi, a.lo); }
DF_HD double to_double(df a) { return (double)a.hi + (double)a.lo; }

// FP64 -> double-float without FP64 arithmetic: hi = x truncated to 24 bits
// (exponent and top mantissa bits moved by integer operations), lo = the
// remaining 29 mantissa bits rounded to FP32.  Finite |x| in [2^-100, 2^120] or 0.
DF_HD df from_double(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  const uint32_t sign = (uint32_t)(b >> 63);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return df{0.0f, 0.0f};
  const uint64_t man = b & 0xfffffffffffffull;
  const uint32_t hib = (sign << 31) | ((uint32_t)(e - 1023 + 127) << 23) | (uint32_t)(man >> 29);
  float hi;
  memcpy(&hi, &hib, 4);
  const uint32_t rest = (uint32_t)(man & 0x1fffffffull);  // 29 bits, weight 2^(e-1023-52)
  // lo = (rest 2^-52) 2^(e-1023): both scalings by exactly representable powers of two
  const int pe = e - 1023 + 127;
  float lo = 0.0f;
  if (rest && pe > 0 && pe < 255) {
    const uint32_t pb = (uint32_t)pe << 23;
    float p2;
    memcpy(&p2, &pb, 4);
    lo = ((float)rest * 0x1p-52f) * p2;
    if (sign) lo = -lo;
  }
  return df{hi, lo};
}

// Uniform deviate (w + 1/2) 2^-32 of a 32-bit word as an exact double-float: hi
// = the top 24 bits (w with its low 8 bits cleared, exact in FP32), lo = the low
// 8 bits plus 1/2; FastTwoSum normalises the pair (|hi| >= |lo| or hi = 0).
DF_HD df unit_df32(uint32_t w) {
  const float hi = (float)(w & 0xffffff00u) * 0x1p-32f;
  const float lo = ((float)(w & 0xffu) + 0.5f) * 0x1p-32f;
  return fast_two_sum(hi, lo);
}

// ---------------------------------------------------------------------------
// log(x), x > 0 (Tang): x = 2^k m, m in [1, 2); j from the top 7 mantissa bits;
// r = m c_j - 1 (|r| < 2^-8); log x = k ln2 + L_j + log1p(r) with
// log1p(r) = r - r^2/2 + r^3/3 + r^4 (-1/4 + r/5 - r^2/6 + r^3/7), the first three
// terms in double-float, the tail (below 2^-33) in FP32.
// ---------------------------------------------------------------------------
DF_HD df df_log(df x) {
  uint32_t bits;
  memcpy(&bits, &x.hi, 4);
  const int k = (int)((bits >> 23) & 0xff) - 127;
  const uint32_t sb = (uint32_t)(127 - k) << 23;  // 2^-k, exact for the ranges used here
  float scale;
  memcpy(&scale, &sb, 4);
  const df m = df{x.hi * scale, x.lo * scale};
  const int j = (int)((bits >> 16) & 0x7f);
  const float c = ME_TAB(kLogC)[j];
  // r = m c - 1 (the product is within 2^-8 of 1, so the subtraction is exact)
  const df mc = m * c;
  const df r = fast_two_sum(df_sub_rn(mc.hi, 1.0f), mc.lo);
  const float rh = r.hi;
  const float tail = df_fma(df_fma(df_fma(1.0f / 7.0f, rh, -1.0f / 6.0f), rh, 0.2f), rh, -0.25f);
  const df r2 = sqr(r);
  const df r3 = (r2 * rh) * df{kThirdHi, kThirdLo};
  df l1p = (r - r2 * 0.5f) + r3;
  l1p = l1p + (r2.hi * r2.hi) * tail;
  const df kl = two_prod((float)k, kLn2Hi) + (float)k * kLn2Lo;
  const df L = df{ME_TAB(kLogLhi)[j], ME_TAB(kLogLlo)[j]};
  return (kl + L) + l1p;
}

// sin(pi x), cos(pi x) for x in [0, 2]: x = j/128 + d, theta = pi d, |theta| <= pi/256.
DF_HD void df_sincospi(df x, df& s, df& c) {
  const float jf = rintf(x.hi * 128.0f);
  const int j = (int)jf;
  const df d = fast_two_sum(df_sub_rn(x.hi, jf * 0.0078125f), x.lo);  // exact subtraction (Sterbenz)
  const df th = d * df{kPiHi, kPiLo};
  const df t2 = sqr(th);
  const float t2h = t2.hi;
  // sin(theta) = theta - theta^3/6 + theta^5 (1/120 - theta^2/5040)
  const df t3 = t2 * th;
  const float t5 = t2h * t2h * th.hi;
  const df sn = (th - t3 * df{kSixthHi, kSixthLo}) + t5 * df_fma(-t2h, 1.0f / 5040.0f, 1.0f / 120.0f);
  // cos(theta) = 1 - theta^2/2 + theta^4 (1/24 - theta^2/720 + theta^4/40320)
  const float t4 = t2h * t2h;
  const df cs = (dfs(1.0f) - t2 * 0.5f) + t4 * df_fma(df_fma(t2h, 1.0f / 40320.0f, -1.0f / 720.0f), t2h, 1.0f / 24.0f);
  const df cj = df{ME_TAB(kCosHi)[j], ME_TAB(kCosLo)[j]};
  const df sj = df{ME_TAB(kSinHi)[j], ME_TAB(kSinLo)[j]};
  s = sj * cs + cj * sn;
  c = cj * cs - sj * sn;
}

}  // namespace me
