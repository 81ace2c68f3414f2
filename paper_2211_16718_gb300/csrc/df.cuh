// Double-float ("f32x2") arithmetic on the FP32 pipe for quantities that need
// ~1e-13 relative accuracy but not the FP64 pipe (on GB300 FP32 runs 63x faster
// than FP64).  Each value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significant bits.
//
// Building blocks are the classical error-free transformations: Knuth's TwoSum,
// Dekker's Fast2Sum and the FMA-based TwoProd; df_add/df_mul/df_div follow the
// usual double-word algorithms (Dekker 1971; Joldes, Muller, Popescu 2017).
// Conversions from and to FP64 use integer bit manipulation only, so they do
// not occupy the FP64 pipe.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ns3d {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) { return df{hi, lo}; }

// Fast2Sum (Dekker): exact s + e = a + b when |a| >= |b| (or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df{s, e};
}

// TwoSum (Knuth): exact s + e = a + b, no ordering requirement.
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

// TwoProd with FMA: exact p + e = a * b (barring underflow).
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return df{p, e};
}

// Accurate double-word addition (two TwoSums), safe under cancellation.
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  df t = two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

// Double-word addition with one TwoSum: absolute error ~2^-47 (|x| + |y|), i.e.
// accurate relative to the inputs (not to the result under cancellation).  Used
// where the result only ever enters through such absolute bounds (differences
// feeding the smoothness indicators and the interface offsets).
__device__ __forceinline__ df df_add_fast(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, s.lo);
}

// Addition of two non-negative double-words (no cancellation possible).
__device__ __forceinline__ df df_add_pos(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, s.lo);
}

// The same, left unnormalised (see df_mul_u below): with both operands non-negative
// there is no cancellation, so |lo| stays within ~1.5 ulp(hi).
__device__ __forceinline__ df df_add_pos_u(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return df{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}

// Double-word addition when |x| >= c |y| is known with a margin c > 1 well above the
// relative size of the lo parts (then |x.hi| >= |y.hi| and Fast2Sum on the hi parts is
// exact).  Left unnormalised like df_mul_u; with the margin, x + y can cancel at most by
// the factor c/(c-1), so |lo| stays within a few ulp(hi).
__device__ __forceinline__ df df_add_ordered_u(df x, df y) {
  const df s = fast_two_sum(x.hi, y.hi);
  return df{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}

// The same, renormalised (for sums that are squared next, where a larger |lo| would cost
// accuracy).
__device__ __forceinline__ df df_add_ordered(df x, df y) {
  const df s = df_add_ordered_u(x, y);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }

__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.lo, p.lo);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_sqr(df x) {
  df p = two_prod(x.hi, x.hi);
  const float e = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, p.lo);
  return fast_two_sum(p.hi, e);
}

// Multiplication by a float (exact small integers, or any float).
__device__ __forceinline__ df df_mul_f(df x, float c) {
  df p = two_prod(x.hi, c);
  const float e = __fmaf_rn(x.lo, c, p.lo);
  return fast_two_sum(p.hi, e);
}

// Products left unnormalised.  (hi, lo) holds exactly the sum that the normalised
// form would hold (Fast2Sum is an exact transformation), only with |lo| up to a few
// ulp(hi) instead of ulp(hi)/2.  The operations in this file accept such operands
// with error bounds larger by that small factor, so a product that feeds straight
// into another double-float operation skips the three additions of renormalising.
__device__ __forceinline__ df df_mul_u(df x, df y) {
  const df p = two_prod(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.lo, p.lo);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df{p.hi, e};
}

__device__ __forceinline__ df df_sqr_u(df x) {
  const df p = two_prod(x.hi, x.hi);
  return df{p.hi, __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, p.lo)};
}

__device__ __forceinline__ df df_mul_f_u(df x, float c) {
  const df p = two_prod(x.hi, c);
  return df{p.hi, __fmaf_rn(x.lo, c, p.lo)};
}

// Exact scaling by 2 (barring overflow).
__device__ __forceinline__ df df_twice(df x) { return df{2.0f * x.hi, 2.0f * x.lo}; }

// Reciprocal and square root seeds from the special-function unit (PTX rcp.approx /
// sqrt.approx, relative error about 2^-23); the double-float operations below correct
// them, so their results do not depend on the seeds being correctly rounded.
__device__ __forceinline__ float rcp_seed(float y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}

__device__ __forceinline__ float sqrt_seed(float y) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}

// Division x / y (y a normal float magnitude): float quotient q1 from the reciprocal
// seed, exact remainder x - q1*y (TwoProd), one correction q2 = remainder / y.  Error
// about eps_seed^2 + 2^-48 relative (eps_seed ~ 2^-23).
__device__ __forceinline__ df df_div(df x, df y) {
  const float r = rcp_seed(y.hi);
  const float q1 = __fmul_rn(x.hi, r);
  // remainder x - q1*y, evaluated with TwoProd
  df p = two_prod(q1, y.hi);
  float rem = __fsub_rn(x.hi, p.hi);
  rem = __fsub_rn(rem, p.lo);
  rem = __fadd_rn(rem, x.lo);
  rem = __fmaf_rn(-q1, y.lo, rem);
  const float q2 = __fmul_rn(rem, r);
  return fast_two_sum(q1, q2);
}

// Square root of a positive double-word (hi a normal float): float seed r, one
// correction (x - r^2)/(2r) with the exact square of the seed (Dekker's method).
__device__ __forceinline__ df df_sqrt(df x) {
  const float r = sqrt_seed(x.hi);
  const df p = two_prod(r, r);
  float d = __fsub_rn(x.hi, p.hi);
  d = __fsub_rn(d, p.lo);
  d = __fadd_rn(d, x.lo);
  return fast_two_sum(r, __fmul_rn(d, __fmul_rn(0.5f, rcp_seed(r))));
}

__device__ __forceinline__ df df_abs(df x) { return (x.hi < 0.0f) ? df_neg(x) : x; }

// x < y for double-words in canonical form (|lo| <= ulp(hi)/2).
__device__ __forceinline__ bool df_lt(df x, df y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }

// ---- conversions by bit manipulation (no FP64 instructions) -----------------
// float -> double, exact for normal floats; zero and subnormals map to signed 0,
// infinities and NaNs keep their class.  Branch-free: the float exponent is rebased
// from 127 to 1023 by one integer addition on the shifted bit pattern.
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t mag = b & 0x7fffffffu;
  const uint32_t sign = b & 0x80000000u;
  uint32_t hi = (mag >> 3) + (896u << 20);       // (e8 + 896) << 20 | top 20 mantissa bits
  hi = (mag >= 0x7f800000u) ? hi + (896u << 20) : hi;  // e8 = 255 -> e11 = 2047
  const bool zero = mag < 0x00800000u;           // zero or subnormal
  hi = zero ? sign : (hi | sign);
  const uint32_t lo = zero ? 0u : (b << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// Power of two 2^k as a float for -126 <= k <= 127.
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

// double -> double-float: hi = x truncated to 24 significant bits, lo = the next
// 29 bits rounded to a float.  Values below 2^-126 in magnitude become (+-0, 0); the lo
// part of values below 2^-74 is dropped (relative error 2^-24 only for such tiny x);
// values beyond the float range become +-inf.  Branch-free integer arithmetic.
__device__ __forceinline__ df d2df_bits(double x) {
  const uint32_t h = (uint32_t)__double2hiint(x);
  const uint32_t l = (uint32_t)__double2loint(x);
  const uint32_t sign = h & 0x80000000u;
  const int e11 = (int)((h >> 20) & 0x7ffu);
  // (h:l) << 3 keeps the low 9 exponent bits and the top 23 mantissa bits; adding
  // 2^30 (= -896 << 23 modulo 2^32) rebases the exponent for 897 <= e11 <= 1150
  uint32_t hb = (__funnelshift_l(l, h, 3) + 0x40000000u) | sign;
  // lo = (29 remaining bits) * 2^(e11 - 1075), signed; scale 0 below the float range
  const uint32_t ks = (uint32_t)max(e11 - 948, 0);
  float lo = __uint2float_rn(l & 0x1fffffffu) * __uint_as_float((ks << 23) | sign);
  const bool tiny = e11 <= 896, huge = e11 >= 1151;
  hb = tiny ? sign : (huge ? (sign | 0x7f800000u) : hb);
  lo = (tiny || huge) ? 0.0f : lo;
  return df{__uint_as_float(hb), lo};
}

// Round-to-nearest FP64 -> FP32 by bit manipulation (finite values in the float
// range; smaller magnitudes flush to zero, larger ones saturate to infinity).
__device__ __forceinline__ float d2f_rn(double x) {
  const uint32_t h = (uint32_t)__double2hiint(x);
  const uint32_t l = (uint32_t)__double2loint(x);
  const uint32_t sign = h & 0x80000000u;
  const int e8 = (int)((h >> 20) & 0x7ffu) - 896;
  if (e8 <= 0) return __uint_as_float(sign);
  if (e8 >= 255) return __uint_as_float(sign | 0x7f800000u);
  uint32_t bits = ((uint32_t)e8 << 23) | ((h & 0xfffffu) << 3) | (l >> 29);
  bits += (l >> 28) & 1u;  // round half up on the first dropped bit (carry may bump the exponent)
  return __uint_as_float(sign | bits);
}

// Nearest-float of a double (truncated to 24 bits; enough for correction terms).
__device__ __forceinline__ float d2f_trunc(double x) { return d2df_bits(x).hi; }

// Largest power of two not above |x| (x finite, nonzero, normal float).
__device__ __forceinline__ int exponent_of(float x) { return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127; }

// ---- FP64 reciprocal and reciprocal square root by Newton-Raphson -------------
// Seeds from the FP32 MUFU approximations (relative error ~2^-22 after the
// truncating conversion); each Newton step squares the error, two steps reach
// FP64 rounding.  For x in the normal float range (positive for rsqrt).
__device__ __forceinline__ double rcp_newton(double x) {
  double r = f2d_bits(__frcp_rn(d2f_trunc(x)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

__device__ __forceinline__ double rsqrt_newton(double x) {
  double r = f2d_bits(rsqrtf(d2f_trunc(x)));
  const double hx = 0.5 * x;
  double e = fma(-hx * r, r, 0.5);  // (1 - x r^2)/2
  r = fma(r, e, r);
  e = fma(-hx * r, r, 0.5);
  return fma(r, e, r);
}

}  // namespace ns3d
