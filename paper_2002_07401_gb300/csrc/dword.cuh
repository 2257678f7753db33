// dword.cuh -- double-word ("float-float") arithmetic on FP32 for the mixed
// path's orbital evaluation.  A value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits, computed
// with FP32 instructions only (GB300 issues FP32 at ~58x its FP64 rate).
//
// Building blocks: the error-free sum of two numbers (Knuth's TwoSum; the
// branch-free FastTwoSum of Dekker 1971 when |a| >= |b|), the error-free
// product by one fused multiply-add, and double-word sums and products built
// from them as analysed by Joldes, Muller and Popescu (ACM TOMS 2017).  The
// _rn intrinsics keep the compiler from contracting or reordering the steps.
#pragma once

#include <cuda_runtime.h>

namespace jagp {

struct fdw {
  float hi, lo;
};

__device__ __forceinline__ fdw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}

// requires |a| >= |b| (or a = 0)
__device__ __forceinline__ fdw fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ fdw two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ fdw dw_neg(fdw x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ fdw dw_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - static_cast<double>(h))};
}

// x + y, both double-words: two TwoSums and two renormalisations (relative
// error a few units of 2^-48 even with cancellation between x and y)
__device__ __forceinline__ fdw dw_add(fdw x, fdw y) {
  const fdw s = two_sum(x.hi, y.hi);
  const fdw t = two_sum(x.lo, y.lo);
  const fdw v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ fdw dw_add_f(fdw x, float y) {
  const fdw s = two_sum(x.hi, y);
  return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}

__device__ __forceinline__ fdw dw_mul(fdw x, fdw y) {
  const fdw c = two_prod(x.hi, y.hi);
  float t = __fmul_rn(x.lo, y.lo);
  t = __fmaf_rn(x.hi, y.lo, t);
  t = __fmaf_rn(x.lo, y.hi, t);
  return fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}

__device__ __forceinline__ fdw dw_mul_f(fdw x, float y) {
  const fdw c = two_prod(x.hi, y);
  return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}

// square root: s = sqrt(hi) refined by one Newton step on the residual
__device__ __forceinline__ fdw dw_sqrt(fdw x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  const float s = sqrtf(x.hi);
  const float res = __fadd_rn(__fmaf_rn(-s, s, x.hi), x.lo);  // x - s^2, the fma exact
  return fast_two_sum(s, __fdiv_rn(res, __fmul_rn(2.0f, s)));
}

// 1 / x as a double-word: the FP32 reciprocal y refined by one Newton step,
// y' = y + y e with the residual e = 1 - x y formed exactly by an fma
__device__ __forceinline__ fdw dw_recip(fdw x) {
  const float y = __frcp_rn(x.hi);
  const float e = __fadd_rn(__fmaf_rn(-x.hi, y, 1.0f), -__fmul_rn(x.lo, y));
  return fast_two_sum(y, __fmul_rn(y, e));
}

// e^x for x <= 0 as a double-word, relative error ~1e-9:
// Cody-Waite reduction x = k ln2 + r, |r| <= ln2/2, with ln2 split into three
// FP32 parts (the first with 16 significant bits, so that k * part1 and the
// first subtraction are exact for |k| <= 150); then the Taylor series
// e^r = 1 + r + r^2/2 + r^3 q(r), q(r) = sum_{n=3..8} r^(n-3)/n!, the first
// three terms in double-word, the tail (< 0.0073) in FP32; the scaling by 2^k
// is exact.  Arguments below -104 (where e^x is below the FP32 range) give 0.
__device__ __forceinline__ fdw dw_exp_neg(fdw x) {
  if (!(x.hi > -104.0f)) return {x.hi != x.hi ? x.hi : 0.0f, 0.0f};
  const float kLn2a = 0.693145751953125f;        // 16 significant bits
  const float kLn2b = 1.428606765330187e-06f;     // ln2 - kLn2a, rounded
  const float kLn2c = 5.497923148e-14f;           // the remainder, rounded
  const float k = rintf(__fmul_rn(x.hi, 1.44269504f));
  fdw r = two_sum(__fmaf_rn(-k, kLn2a, x.hi), x.lo);
  r = dw_add(r, dw_neg(two_prod(k, kLn2b)));
  r = dw_add_f(r, __fmul_rn(-k, kLn2c));
  const float rh = r.hi;
  float q = 1.0f / 40320.0f;
  q = __fmaf_rn(q, rh, 1.0f / 5040.0f);
  q = __fmaf_rn(q, rh, 1.0f / 720.0f);
  q = __fmaf_rn(q, rh, 1.0f / 120.0f);
  q = __fmaf_rn(q, rh, 1.0f / 24.0f);
  q = __fmaf_rn(q, rh, 1.0f / 6.0f);
  const float tail = __fmul_rn(q, __fmul_rn(__fmul_rn(rh, rh), rh));
  fdw h = dw_mul(r, r);
  h.hi = __fmul_rn(h.hi, 0.5f);
  h.lo = __fmul_rn(h.lo, 0.5f);
  fdw e = dw_add(r, h);
  e = dw_add_f(e, tail);
  e = dw_add_f(e, 1.0f);
  const int ki = static_cast<int>(k);
  if (ki >= -126) {
    const float p = __int_as_float((127 + ki) << 23);
    return {__fmul_rn(e.hi, p), __fmul_rn(e.lo, p)};
  }
  return {ldexpf(e.hi, ki), ldexpf(e.lo, ki)};
}

}  // namespace jagp
