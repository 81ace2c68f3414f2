// Double-float arithmetic on two independent lanes at once, with the packed FP32
// instructions of sm_100-class GPUs (FADD2 / FMUL2 / FFMA2 through the CUDA builtins
// __fadd2_rn, __fmul2_rn, __ffma2_rn).  A packed instruction does the work of two
// scalar ones in one issue slot (it holds the FP32 pipe for two cycles, so the FP32
// throughput is unchanged; what it saves is instruction issue, which bounds the
// direction passes).  Operand negations, including per-lane ones, fold into the
// packed instructions.
//
// Every operation here except df2_div performs, in each lane, exactly the IEEE
// operations of its scalar counterpart in df.cuh in the same order (a - b as a + (-b),
// which IEEE 754 defines identically), so a two-lane result equals the two scalar
// results bit for bit (tests/test_gpu_df2.py: a million random lane pairs, operation by
// operation and for the compositions the direction pass uses); df2_div differs from
// df_div in its last step (see there).
// Layout: hi = (hi of lane 0, hi of lane 1), lo = (lo of lane 0, lo of lane 1).
#pragma once

#include <cuda_runtime.h>

#include "df.cuh"

namespace ns3d {

struct df2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, f2neg(b)); }
// The product as an explicit PTX mul.rn.f32x2.  Where a fused multiply-add of such a
// product with the following addition would round differently and was observed (the
// last step of the division below), the fused form is written out instead.
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2splat(float c) { return make_float2(c, c); }

// Lane views and packing.
__device__ __forceinline__ df df2_lane0(df2 x) { return df{x.hi.x, x.lo.x}; }
__device__ __forceinline__ df df2_lane1(df2 x) { return df{x.hi.y, x.lo.y}; }
__device__ __forceinline__ df2 df2_pack(df a, df b) { return df2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ df2 df2_splat(df a) { return df2{f2splat(a.hi), f2splat(a.lo)}; }
// The shared-memory form of a lane pair: (hi0, hi1, lo0, lo1).
__device__ __forceinline__ df2 df2_from4(float4 v) { return df2{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 df2_to4(df2 x) { return make_float4(x.hi.x, x.hi.y, x.lo.x, x.lo.y); }

__device__ __forceinline__ df2 df2_neg(df2 x) { return df2{f2neg(x.hi), f2neg(x.lo)}; }

// Fast2Sum, TwoSum, TwoProd (as fast_two_sum, two_sum, two_prod).
__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = f2add(a, b);
  return df2{s, f2sub(b, f2sub(s, a))};
}
__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = f2add(a, b);
  const float2 bb = f2sub(s, a);
  return df2{s, f2add(f2sub(a, f2sub(s, bb)), f2sub(b, bb))};
}
__device__ __forceinline__ df2 two_prod2(float2 a, float2 b) {
  const float2 p = f2mul(a, b);
  return df2{p, f2fma(a, b, f2neg(p))};
}

// As df_add_fast, df_add_pos_u, df_add_ordered_u, df_add_ordered.
__device__ __forceinline__ df2 df2_add_fast(df2 x, df2 y) {
  df2 s = two_sum2(x.hi, y.hi);
  s.lo = f2add(s.lo, f2add(x.lo, y.lo));
  return fast_two_sum2(s.hi, s.lo);
}
__device__ __forceinline__ df2 df2_add_pos_u(df2 x, df2 y) {
  const df2 s = two_sum2(x.hi, y.hi);
  return df2{s.hi, f2add(s.lo, f2add(x.lo, y.lo))};
}
__device__ __forceinline__ df2 df2_add_ordered_u(df2 x, df2 y) {
  const df2 s = fast_two_sum2(x.hi, y.hi);
  return df2{s.hi, f2add(s.lo, f2add(x.lo, y.lo))};
}
__device__ __forceinline__ df2 df2_add_ordered(df2 x, df2 y) {
  const df2 s = df2_add_ordered_u(x, y);
  return fast_two_sum2(s.hi, s.lo);
}

// As df_mul_u, df_sqr_u, df_mul_f_u (unnormalised products), df_twice.
__device__ __forceinline__ df2 df2_mul_u(df2 x, df2 y) {
  const df2 p = two_prod2(x.hi, y.hi);
  float2 e = f2fma(x.hi, y.lo, p.lo);
  e = f2fma(x.lo, y.hi, e);
  return df2{p.hi, e};
}
// As df_mul (normalised product).
__device__ __forceinline__ df2 df2_mul(df2 x, df2 y) {
  const df2 p = two_prod2(x.hi, y.hi);
  float2 e = f2fma(x.hi, y.lo, p.lo);
  e = f2fma(x.lo, y.hi, e);
  return fast_two_sum2(p.hi, e);
}
__device__ __forceinline__ df2 df2_sqr_u(df2 x) {
  const df2 p = two_prod2(x.hi, x.hi);
  return df2{p.hi, f2fma(f2add(x.hi, x.hi), x.lo, p.lo)};
}
__device__ __forceinline__ df2 df2_mul_f_u(df2 x, float c) {
  const float2 cc = f2splat(c);
  const df2 p = two_prod2(x.hi, cc);
  return df2{p.hi, f2fma(x.lo, cc, p.lo)};
}
__device__ __forceinline__ df2 df2_twice(df2 x) {
  const float2 two = f2splat(2.0f);
  return df2{f2mul(two, x.hi), f2mul(two, x.lo)};
}
// Exact scaling of both parts by per-lane powers of two.
__device__ __forceinline__ df2 df2_scale(df2 x, float2 s) { return df2{f2mul(x.hi, s), f2mul(x.lo, s)}; }

// Division as df_div (per-lane reciprocal seeds from the special-function unit, the rest
// packed), except for the last step: the correction q1 + rem * r is renormalised with its
// error term taken from the exact product, e = fma(rem, r, -(s - q1)) with s = q1 + q2,
// instead of q2 - (s - q1).  (The compiler fuses the packed product into that subtraction
// anyway; written out, the operation is the same whatever it decides.)  s + e is then
// q1 + rem * r up to one rounding of e, at least as accurate as the Fast2Sum of df_div.
__device__ __forceinline__ df2 df2_div(df2 x, df2 y) {
  const float2 r = make_float2(rcp_seed(y.hi.x), rcp_seed(y.hi.y));
  const float2 q1 = f2mul(x.hi, r);
  const df2 p = two_prod2(q1, y.hi);
  float2 rem = f2sub(x.hi, p.hi);
  rem = f2sub(rem, p.lo);
  rem = f2add(rem, x.lo);
  rem = f2fma(f2neg(q1), y.lo, rem);
  const float2 s = f2add(q1, f2mul(rem, r));
  return df2{s, f2fma(rem, r, f2neg(f2sub(s, q1)))};
}

}  // namespace ns3d
