// Float-float ("double-float") arithmetic: a value is hi + lo with two
// float32 numbers, |lo| <= ulp(hi)/2, giving ~48 significant bits. Built from
// the error-free transformations of Knuth (two-sum) and Dekker (two-product,
// here with a fused multiply-add), with division by long division and square
// root by one Newton correction, as in the double-double algorithms of Hida,
// Li and Bailey (2001) carried over to float32. Used for the SAV scalar
// algebra of the float32-bulk path: this GPU issues float64 slowly (measured
// ~69-cycle dependent FMA, ~580-cycle divide), float32 quickly.
#pragma once

#include <cuda_runtime.h>

namespace spfc {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo = 0.f) { return ff{hi, lo}; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// p + e = a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const ff s = two_sum(x.hi, y.hi);
  const ff t = two_sum(x.lo, y.lo);
  ff r = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(r.hi, __fadd_rn(r.lo, t.lo));
}
__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const ff p = two_prod(x.hi, y.hi);
  const float c = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  return fast_two_sum(p.hi, __fadd_rn(p.lo, c));
}
__device__ __forceinline__ ff ff_mulf(ff x, float y) {
  const ff p = two_prod(x.hi, y);
  return fast_two_sum(p.hi, __fmaf_rn(x.lo, y, p.lo));
}

// x / y: three-term long division
__device__ __forceinline__ ff ff_div(ff x, ff y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  ff r = ff_sub(x, ff_mulf(y, q1));
  const float q2 = __fdiv_rn(r.hi, y.hi);
  r = ff_sub(r, ff_mulf(y, q2));
  const float q3 = __fdiv_rn(r.hi, y.hi);
  const ff q = fast_two_sum(q1, q2);
  return ff_add(q, ff_make(q3));
}

// sqrt(x), x > 0: float32 root refined by one Newton step in float-float
__device__ __forceinline__ ff ff_sqrt(ff x) {
  const float s = __fsqrt_rn(x.hi);
  const ff s2 = two_prod(s, s);
  const float e = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(x.hi, s2.hi), s2.lo), x.lo), __fmul_rn(2.f, s));
  return fast_two_sum(s, e);
}

__device__ __forceinline__ bool ff_isfinite(ff x) { return isfinite(x.hi) && isfinite(x.lo); }

}  // namespace spfc
