// Float-float (unevaluated sum hi + lo of two FP32 numbers) arithmetic for
// the single-precision apply.  GB300 runs FP64 at 1/64 of its FP32 rate, so
// the local solves, the coarse restriction and the prolongation keep their
// operands in FP32 (or FP16) storage but evaluate their sums with error-free
// transformations on the FP32 pipe:
//  * TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and FastTwoSum (Dekker 1971);
//  * the exact product error fma(a, b, -a*b) (Ogita, Rump, Oishi, "Accurate
//    sum and dot product", SIAM J. Sci. Comput. 26, 2005: Dot2);
//  * a biased accumulator: with hi kept near a power of two A >= 3 * (the sum
//    of |terms| so far), s = fl(hi + v x) and hi are within a factor two, so
//    d = hi - s is exact (Sterbenz) and fma(v, x, d) is the rounding error of
//    s, correct to one FP32 rounding.  Five operations per product instead of
//    the eleven of Dot2; A is raised by powers of two as the bound grows.
// Every operation goes through the _rn intrinsics so the compiler cannot
// contract or reassociate them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace asmgpu {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// (hi, lo) += (bh, bl), both normalised float-float numbers
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  fast_two_sum(s, e, hi, lo);
}

// smallest power of two >= m (m >= 0, finite; 0 for m = 0)
__device__ __forceinline__ float pow2_ceil(float m) {
  return __uint_as_float((__float_as_uint(m) + 0x7fffffu) & 0x7f800000u);
}

// Biased accumulator: value = (hi - A) + lo; bnd >= the sum of |v * xh| of
// the terms taken so far (FP32, rounded up by the factor checks below).
struct BiasAcc {
  float hi, lo, A, bnd;
};

__device__ __forceinline__ void bias_init(BiasAcc& a) {
  a.hi = 0.f;
  a.lo = 0.f;
  a.A = 0.f;
  a.bnd = 0.f;
}

// Account for the next terms, whose |v * xh| sum to tb, before adding them:
// keeps A >= 4 * bnd (three is what the exactness argument needs), moving
// the value to a new power of two with 8x headroom when it does not.
__device__ __forceinline__ void bias_reserve(BiasAcc& a, float tb) {
  a.bnd = __fadd_rn(a.bnd, tb);
  if (__fmul_rn(4.f, a.bnd) > a.A) {
    const float An = pow2_ceil(__fmul_rn(8.f, a.bnd));
    const float P = __fsub_rn(a.hi, a.A);  // exact
    float s, e;
    fast_two_sum(An, P, s, e);  // |An| >= 4 |P|
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
    a.A = An;
  }
}

// hi + lo += v * (xh + xl)
__device__ __forceinline__ void bias_step(BiasAcc& a, float v, float xh, float xl) {
  const float s = __fmaf_rn(v, xh, a.hi);
  const float d = __fsub_rn(a.hi, s);      // exact
  const float r = __fmaf_rn(v, xh, d);     // rounding error of s (one rounding)
  a.hi = s;
  a.lo = __fadd_rn(a.lo, r);
  a.lo = __fmaf_rn(v, xl, a.lo);
}

// keep lo small: hi + lo unchanged, |lo| <= ulp(hi)
__device__ __forceinline__ void bias_renorm(BiasAcc& a) {
  float s, e;
  fast_two_sum(a.hi, a.lo, s, e);
  a.hi = s;
  a.lo = e;
}

// the accumulated value as a normalised float-float pair
__device__ __forceinline__ void bias_value(const BiasAcc& a, float& h, float& l) {
  two_sum(__fsub_rn(a.hi, a.A), a.lo, h, l);
}

// Dot2 step: (hi, lo) += v * (xh + xl)
__device__ __forceinline__ void dot2_step(float& hi, float& lo, float v, float xh, float xl) {
  const float p = __fmul_rn(v, xh);
  const float pe = __fmaf_rn(v, xh, -p);
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
  lo = __fmaf_rn(v, xl, lo);
}

// the biased step and renormalisation on a bare (hi, lo) pair whose bias is
// kept by the caller
__device__ __forceinline__ void bias_step1(float& hi, float& lo, float v, float xh, float xl) {
  const float s = __fmaf_rn(v, xh, hi);
  const float d = __fsub_rn(hi, s);   // exact
  const float r = __fmaf_rn(v, xh, d);
  hi = s;
  lo = __fadd_rn(lo, r);
  lo = __fmaf_rn(v, xl, lo);
}
__device__ __forceinline__ void bias_renorm1(float& hi, float& lo) {
  float s, e;
  fast_two_sum(hi, lo, s, e);
  hi = s;
  lo = e;
}

// split a double into hi + lo (exact up to 2^-48 relative)
__device__ __forceinline__ float2 split_ff(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

__device__ __forceinline__ double ff_to_double(float h, float l) { return (double)h + (double)l; }

}  // namespace asmgpu
