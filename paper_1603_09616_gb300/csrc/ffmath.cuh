// Float-float ("FP32 pair") arithmetic for the mixed-precision path.
//
// GB300 runs FP32 FMAs ~58x faster than FP64 ones, so the reduced-precision
// path keeps values that must stay FP64-accurate (the seed Krylov vectors, the
// product H p, the inner-solve residual and the dot products) as unevaluated
// sums hi + lo of two floats, with ~48 significand bits.  The primitives are the
// classical error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum and
// the FMA-based exact product (TwoProd).  Every primitive uses the explicit
// round-to-nearest intrinsics so the compiler cannot contract or reassociate
// the operations the error terms depend on.
#pragma once
#include <cuda_runtime.h>

namespace gbff {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_from_double(double d) {
  const float hi = __double2float_rn(d);
  const float lo = __double2float_rn(d - (double)hi);
  return {hi, lo};
}
__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

// Compensated accumulator: s = hi + lo + err, fed with exact products.
struct acc {
  float hi, err;
};
__device__ __forceinline__ void acc_init(acc& a) { a.hi = 0.f; a.err = 0.f; }
// a += x * y with x, y float-float (products of the low parts dropped: 2^-48 relative)
__device__ __forceinline__ void acc_mul_add(acc& a, ff x, ff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const ff s = two_sum(a.hi, p);
  a.hi = s.hi;
  a.err = __fadd_rn(a.err, __fadd_rn(s.lo, e));
}
// a += x * y with x float-float, y float
__device__ __forceinline__ void acc_mul_add(acc& a, ff x, float y) {
  const float p = __fmul_rn(x.hi, y);
  float e = __fmaf_rn(x.hi, y, -p);
  e = __fmaf_rn(x.lo, y, e);
  const ff s = two_sum(a.hi, p);
  a.hi = s.hi;
  a.err = __fadd_rn(a.err, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ void acc_add(acc& a, ff x) {
  const ff s = two_sum(a.hi, x.hi);
  a.hi = s.hi;
  a.err = __fadd_rn(a.err, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ ff acc_get(const acc& a) { return fast_two_sum(a.hi, a.err); }
__device__ __forceinline__ double acc_to_double(const acc& a) { return (double)a.hi + (double)a.err; }

// complex float-float: stored as float4 {re.hi, re.lo, im.hi, im.lo}
struct cff {
  ff re, im;
};
__device__ __forceinline__ cff cff_load(const float4& v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 cff_store(const cff& c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }
__device__ __forceinline__ cff cff_add(cff a, cff b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__device__ __forceinline__ cff cff_sub(cff a, cff b) { return {ff_sub(a.re, b.re), ff_sub(a.im, b.im)}; }
__device__ __forceinline__ cff cff_mul(cff a, cff b) {
  return {ff_sub(ff_mul(a.re, b.re), ff_mul(a.im, b.im)), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
__device__ __forceinline__ cff cff_from(double2 d) { return {ff_from_double(d.x), ff_from_double(d.y)}; }
__device__ __forceinline__ cff cff_scale_pow2(cff a, float s) {
  return {{a.re.hi * s, a.re.lo * s}, {a.im.hi * s, a.im.lo * s}};
}

}  // namespace gbff
