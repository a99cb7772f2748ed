// Double-float ("dd") arithmetic: a value is hi + lo with two float32s,
// |lo| <= ulp(hi)/2, about 48 significant bits.  GB300 runs float32 at many
// times its float64 rate, so the elementwise stages of the fast form (the
// Eq. A7 regulariser, the 2-RDM dressing, the digit staging) use these
// operations.  The error-free transformations are Knuth's TwoSum and the
// fused-multiply-add TwoProduct; additions and products follow the standard
// double-float construction (Dekker 1971).
#pragma once
#include <cuda_runtime.h>

namespace dsrg {

struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_make(float h) { return {h, 0.0f}; }

__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ dd quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dd two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

// a + b with an absolute error of a few units of 2^-48 max(|a|, |b|) (no
// relative accuracy when the high parts cancel); for sums whose terms keep
// their sign or whose cancellation the caller does not need resolved.
__device__ __forceinline__ dd dd_add_fast(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_sub_fast(dd a, dd b) { return dd_add_fast(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ dd dd_add_f(dd a, float b) {
  dd s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_mul_f(dd a, float b) {
  dd p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// a / b: float reciprocal estimate, one dd correction step
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dd r = dd_sub(a, dd_mul_f(b, q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  const dd r2 = dd_sub(r, dd_mul_f(b, q2));
  const float q3 = __fdiv_rn(r2.hi, b.hi);
  dd q = quick_two_sum(q1, q2);
  return dd_add_f(q, q3);
}

// 1 / b: float reciprocal (one rounding), then one Newton step in
// double-float, r1 = r0 + r0 (1 - b r0), with 1 - b r0 formed exactly enough
// (TwoProduct of the high parts): relative error about 2^-46.
__device__ __forceinline__ dd dd_recip(dd b) {
  const float r0 = __frcp_rn(b.hi);
  const dd p = two_prod(b.hi, r0);
  const float e = __fmaf_rn(-b.lo, r0, __fsub_rn(__fsub_rn(1.0f, p.hi), p.lo));
  return quick_two_sum(r0, __fmul_rn(r0, e));
}

__device__ __forceinline__ dd dd_ldexp(dd a, int e) { return {ldexpf(a.hi, e), ldexpf(a.lo, e)}; }

__device__ __forceinline__ dd dd_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

}  // namespace dsrg
