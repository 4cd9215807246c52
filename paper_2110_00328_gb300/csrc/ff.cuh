// ff.cuh -- float-float ("double-single") arithmetic for the fine-level
// residual of the mixed-precision solver.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// carrying ~48 significant bits.  The operations are built from the classical
// error-free transformations: Knuth's two-sum, Dekker's fast two-sum (|a| >=
// |b|) and the FMA-based two-product (the rounding error of a*b is
// fma(a, b, -a*b) exactly).  Every step is a single-precision instruction with
// explicit round-to-nearest intrinsics, so the compiler neither contracts nor
// reorders them.  On GB300 single precision runs at 64 times the FP64 rate,
// which makes ~10 float operations per double operation the cheaper way to
// carry the residual's 1e-13 relative accuracy.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) { return ff{hi, lo}; }

// a + b = s + e exactly (Knuth)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}

// a + b = s + e exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a * b = p + e exactly (FMA two-product)
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const ff p = two_prod(x.hi, y.hi);
  const float c = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  return fast_two_sum(p.hi, __fadd_rn(p.lo, c));
}

// x * f for a float f
__device__ __forceinline__ ff ff_mul_f(ff x, float f) {
  const ff p = two_prod(x.hi, f);
  return fast_two_sum(p.hi, __fmaf_rn(x.lo, f, p.lo));
}

__device__ __forceinline__ ff ff_sqr(ff x) {
  const ff p = two_prod(x.hi, x.hi);
  return fast_two_sum(p.hi, __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, p.lo));
}

__device__ __forceinline__ float ff_to_float(ff x) { return __fadd_rn(x.hi, x.lo); }

// x / y: the quotient's leading float q1 from the approximate reciprocal, then
// one correction q2 = (x - q1 y) / y with the remainder formed exactly to first
// order (q1 y.hi by two-product; x.hi - (q1 y.hi).hi is exact since the two
// agree to a few ulp).  Unnormalised: |q2| <= ~2^-22 |q1|.
__device__ __forceinline__ ff ff_div(ff x, ff y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y.hi));
  const float q1 = __fmul_rn(x.hi, r);
  const ff p = two_prod(q1, y.hi);
  const float rem = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo), __fmul_rn(q1, y.lo));
  return ff{q1, __fmul_rn(rem, r)};
}

// Unnormalised float-float accumulator: the value is s + e, where s is the
// running float sum of the leading parts and e collects, in single precision,
// the exact rounding errors of those sums together with the low parts.  One
// two-sum per term and no renormalisation: after m terms the error is at most
// ~m^2 2^-48 of the largest partial sum.
struct ffacc {
  float s, e;
};

__device__ __forceinline__ ffacc acc_of(ff x) { return ffacc{x.hi, x.lo}; }

// a += hi + lo
__device__ __forceinline__ void acc_add(ffacc& a, float hi, float lo) {
  const ff t = two_sum(a.s, hi);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, lo));
}

__device__ __forceinline__ void acc_add(ffacc& a, ff x) { acc_add(a, x.hi, x.lo); }

__device__ __forceinline__ ff acc_ff(const ffacc& a) { return two_sum(a.s, a.e); }

__device__ __forceinline__ float acc_float(const ffacc& a) { return __fadd_rn(a.s, a.e); }

// Exact split of a double into hi + lo by integer operations on its bits (no
// double-precision instruction): hi keeps the leading 24 bits of the
// significand, lo the next 29 rounded to 24.  Valid for |d| in [2^-74, 2^128);
// smaller magnitudes give hi = lo = 0, which the residual never needs, and
// larger ones (inf, NaN) give NaN, so that a diverging solve is still seen.
__device__ __forceinline__ ff ff_from_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7FF);        // biased exponent
  if (ex < 1023 - 74) return ff{0.f, 0.f};
  if (ex > 1023 + 127) return ff{__int_as_float(0x7fffffff), 0.f};  // |d| >= 2^128, inf, NaN: NaN
  const unsigned mhi = (unsigned)((b >> 29) & 0x7FFFFFu);  // 23 fraction bits after the leading one
  const float hi = __uint_as_float(sign | ((unsigned)(ex - 1023 + 127) << 23) | mhi);
  const unsigned rest = (unsigned)(b & 0x1FFFFFFFull);     // remaining 29 bits, units 2^(ex-1023-52)
  // rest * 2^(ex - 1075) with the scale built as a float (exponent ex - 1075 >= -126)
  const float scale = __uint_as_float((unsigned)(ex - 1075 + 127) << 23);
  const float lo = __fmul_rn(__uint2float_rn(rest), scale);
  return ff{hi, sign ? -lo : lo};
}

}  // namespace mg
