// Double-FP32 ("df32") arithmetic for the FP64-accurate operator on the FP32
// pipe. A real number is an unevaluated sum h + l of two floats; products of
// the leading parts are exact through FMA (p = a*b, e = fma(a, b, -p)), sums
// of leading parts are exact through Knuth's TwoSum (six additions), and the
// trailing parts and cross terms are carried in plain FP32, where their
// rounding is 2^-24 of quantities already 2^-23 smaller than the result.
//
// FP64 inputs are split without FP64 instructions: h takes the sign, the
// exponent and the top 23 stored mantissa bits of the double (truncated); l
// is the remaining 29 bits rounded to 23, built as a float whose implicit one
// is subtracted again. The split is exact to 2^-47 relative (|d| between
// 2^-103 and 2^127; smaller magnitudes keep h only, which still holds
// them to 2^-24, and zero and subnormals give 0). Results go back to FP64
// as double(h) + double(l) (three FP64 operations per value).
#pragma once

#include <stdint.h>

#include "sq_device.cuh"

namespace sq {

struct df {
  float h, l;
};

__device__ __forceinline__ df split64(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const unsigned s = bh & 0x80000000u;
  const int E = (int)((bh >> 20) & 0x7FFu);
  df r;
  if (E < 897 || E > 1150) {  // zero, subnormal, tiny or huge: no float split
    r.h = E > 1150 ? __uint_as_float(s | 0x7F800000u) : __uint_as_float(s);
    r.l = 0.0f;
    return r;
  }
  const unsigned m23 = ((bh & 0xFFFFFu) << 3) | (bl >> 29);
  r.h = __uint_as_float(s | ((unsigned)(E - 896) << 23) | m23);
  if (E < 920) {
    r.l = 0.0f;
    return r;
  }
  // 29 remaining bits, rounded to 23 (a carry into the exponent field still
  // gives the right value after the implicit one is taken away)
  const unsigned rem = ((bl & 0x1FFFFFFFu) + 32u) >> 6;
  const unsigned base = s | ((unsigned)(E - 919) << 23);
  r.l = __uint_as_float(base + rem) - __uint_as_float(base);
  return r;
}

__device__ __forceinline__ double to64(df a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly (a, b floats)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// a + b
__device__ __forceinline__ df df_add(df a, df b) {
  df r;
  float e;
  two_sum(a.h, b.h, r.h, e);
  r.l = e + (a.l + b.l);
  return r;
}

// a - b
__device__ __forceinline__ df df_sub(df a, df b) {
  df r;
  float e;
  two_sum(a.h, -b.h, r.h, e);
  r.l = e + (a.l - b.l);
  return r;
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }

// acc + a * b
__device__ __forceinline__ df df_fma(df a, df b, df acc) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.h, -p);
  const float c = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  df r;
  float t;
  two_sum(acc.h, p, r.h, t);
  r.l = acc.l + (t + c);
  return r;
}

// complex df32: re and im, each h + l; stored as float4 (re.h, im.h, re.l, im.l)
struct cdf {
  df re, im;
};

__device__ __forceinline__ cdf cdf_of(float4 q) { return cdf{df{q.x, q.z}, df{q.y, q.w}}; }
__device__ __forceinline__ float4 float4_of(cdf a) { return make_float4(a.re.h, a.im.h, a.re.l, a.im.l); }
__device__ __forceinline__ cdf cdf_split(double2 d) { return cdf{split64(d.x), split64(d.y)}; }
__device__ __forceinline__ double2 double2_of(cdf a) { return make_double2(to64(a.re), to64(a.im)); }

__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cdf{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
// i a
__device__ __forceinline__ cdf citimes(cdf a) { return cdf{df_neg(a.im), a.re}; }
// acc + u * v
__device__ __forceinline__ cdf cfma_df(cdf u, cdf v, cdf acc) {
  acc.re = df_fma(u.re, v.re, acc.re);
  acc.re = df_fma(df_neg(u.im), v.im, acc.re);
  acc.im = df_fma(u.re, v.im, acc.im);
  acc.im = df_fma(u.im, v.re, acc.im);
  return acc;
}
// acc + conj(u) * v
__device__ __forceinline__ cdf cjfma_df(cdf u, cdf v, cdf acc) {
  acc.re = df_fma(u.re, v.re, acc.re);
  acc.re = df_fma(u.im, v.im, acc.re);
  acc.im = df_fma(u.re, v.im, acc.im);
  acc.im = df_fma(df_neg(u.im), v.re, acc.im);
  return acc;
}
// s * a for a real df32 scalar s
__device__ __forceinline__ cdf cscale(df s, cdf a) {
  const df z{0.0f, 0.0f};
  return cdf{df_fma(s, a.re, z), df_fma(s, a.im, z)};
}

}  // namespace sq
