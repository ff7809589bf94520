// Float-float arithmetic for the dense stages of FP32 steps.
//
// GB300's FP64 pipe issues about 1.7 FMAs per clock per SM against 128 FP32
// FMAs, so the slice products of the dense stages (Grams of the cores and of
// the rank-2r cores, the new cores) are FP64-throughput bound.  In an FP32
// step they run on the FP32 pipe instead, with every operand held as an
// unevaluated sum of two floats (hi + lo, 48 significant bits) and every dot
// product accumulated by the compensated scheme of Ogita, Rump and Oishi
// ("Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005,
// algorithm Dot2): the product of the high parts is split exactly by an FMA
// (TwoProduct), the running sum exactly by Knuth's TwoSum, and the rounding
// errors plus the cross terms hi*lo and lo*hi are summed in a second float.
// The result is as accurate as a dot product in twice FP32's precision: the
// error is about u |a.b| + (n u)^2 sum |a_i b_i| with u = 2^-24 (for n = 64,
// ~2e-11 relative to sum |a_i b_i|), far below what an FP32 step needs and
// about 1/12 of the FP64 cost per FMA on this GPU.
//
// The error-free transformations must be evaluated exactly as written, so the
// products and sums use the _rn intrinsics, which the compiler never fuses
// into FMAs.  Values outside FP32's exponent range (|x| >= 2^128 or below
// 2^-126) keep only their FP32 rounding; FP32 steps accept FP32's range.
#pragma once

#include <cuda_runtime.h>

namespace ffa {

// x = hi + lo exactly up to the 53-bit significand: hi is x truncated to 24
// significant bits (built from the exponent and fraction fields with integer
// operations: conversions from FP64 run on the slow FP64 pipe), lo the
// remaining 29 bits rounded to a float.
__device__ __forceinline__ float2 split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 1023 - 126 || e > 1023 + 127) return make_float2(__double2float_rn(x), 0.f);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long frac = b & 0xfffffffffffffULL;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(frac >> 29));
  // lo = rem * 2^(e - 1075), rem < 2^29, scaled in two exact steps so that
  // no factor leaves the normal range (e - 1075 >= -228 here)
  const float rem = __uint2float_rn((unsigned)(frac & 0x1fffffffu));
  const int s = e - 1075;
  const int s1 = s < -100 ? s + 100 : s;
  float lo = __fmul_rn(rem, __uint_as_float((unsigned)(s1 + 127) << 23));
  if (s < -100) lo = __fmul_rn(lo, __uint_as_float((unsigned)(-100 + 127) << 23));
  return make_float2(hi, sign ? -lo : lo);
}

// (hi, lo) back to a double: two exact conversions and one FP64 add
__device__ __forceinline__ double join(float s, float c) { return (double)s + (double)c; }

// Knuth's TwoSum: a + b = t + err exactly
__device__ __forceinline__ void two_sum(float a, float b, float& t, float& err) {
  t = __fadd_rn(a, b);
  const float z = __fsub_rn(t, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(t, z)), __fsub_rn(b, z));
}

// one step of Dot2 on float-float operands: (s, c) += a * b
__device__ __forceinline__ void dot_step(float& s, float& c, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);      // TwoProduct: a.x b.x = p + e exactly
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// (s, c) renormalised to a float-float value (hi, lo), |lo| <= ulp(hi) / 2
__device__ __forceinline__ float2 renorm(float s, float c) {
  float t, err;
  two_sum(s, c, t, err);
  return make_float2(t, err);
}

// (s, c) += w * (u, v), w = (wh, wl) a float-float weight; the product's
// terms below 2^-48 of it are dropped
__device__ __forceinline__ void acc_scaled(float& s, float& c, float2 w, float u, float v) {
  const float p = __fmul_rn(w.x, u);
  float e = __fmaf_rn(w.x, u, -p);
  e = __fmaf_rn(w.x, v, e);
  e = __fmaf_rn(w.y, u, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// sum_t x[t] y[t] over K float-float pairs with unit stride, two independent
// Dot2 chains, returned as (s, c)
__device__ __forceinline__ void dot(const float2* x, const float2* y, int K, float& s, float& c) {
  float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
  int t = 0;
  for (; t + 1 < K; t += 2) {
    dot_step(s0, c0, x[t], y[t]);
    dot_step(s1, c1, x[t + 1], y[t + 1]);
  }
  if (t < K) dot_step(s0, c0, x[t], y[t]);
  float tt, err;
  two_sum(s0, s1, tt, err);
  s = tt;
  c = __fadd_rn(__fadd_rn(c0, c1), err);
}

}  // namespace ffa
