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

// 1/k! as a double-word (the FP32 rounding and the remainder, both formed at
// compile time)
struct DwConst {
  float hi, lo;
};
constexpr DwConst dw_inv_fact(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  const double v = 1.0 / f;
  const float h = static_cast<float>(v);
  return {h, static_cast<float>(v - static_cast<double>(h))};
}

// e^x for x <= 0 as a double-word, relative error a few units of 2^-46:
// Cody-Waite reduction x = k ln2 + r, |r| <= ln2/2, with ln2 split into three
// FP32 parts (the first with 16 significant bits, so that k * part1 and the
// first subtraction are exact for |k| <= 150); then the Taylor series of e^r
// by Horner's rule in double-word arithmetic through r^6/6!, the terms
// r^7/7! .. r^12/12! (together below 1.2e-7) in FP32, the truncation after
// r^12/12! below 3e-16; the scaling by 2^k is exact.  Arguments below -104
// (where e^x is below the FP32 range) give 0.
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
  // FP32 tail: sum_{n=7..12} r^(n-7) / n!
  float q = 1.0f / 479001600.0f;
  q = __fmaf_rn(q, rh, 1.0f / 39916800.0f);
  q = __fmaf_rn(q, rh, 1.0f / 3628800.0f);
  q = __fmaf_rn(q, rh, 1.0f / 362880.0f);
  q = __fmaf_rn(q, rh, 1.0f / 40320.0f);
  q = __fmaf_rn(q, rh, 1.0f / 5040.0f);
  // Horner in double-word: p = 1/6! + r q, then p = 1/n! + r p for n = 5 .. 0
  constexpr DwConst c6 = dw_inv_fact(6), c5 = dw_inv_fact(5), c4 = dw_inv_fact(4), c3 = dw_inv_fact(3);
  fdw p = dw_add(fdw{c6.hi, c6.lo}, dw_mul_f(r, q));
  p = dw_add(fdw{c5.hi, c5.lo}, dw_mul(r, p));
  p = dw_add(fdw{c4.hi, c4.lo}, dw_mul(r, p));
  p = dw_add(fdw{c3.hi, c3.lo}, dw_mul(r, p));
  p = dw_add_f(dw_mul(r, p), 0.5f);
  p = dw_add_f(dw_mul(r, p), 1.0f);
  p = dw_add_f(dw_mul(r, p), 1.0f);
  const int ki = static_cast<int>(k);
  if (ki >= -126) {
    const float sc = __int_as_float((127 + ki) << 23);
    return {__fmul_rn(p.hi, sc), __fmul_rn(p.lo, sc)};
  }
  return {ldexpf(p.hi, ki), ldexpf(p.lo, ki)};
}

}  // namespace jagp
