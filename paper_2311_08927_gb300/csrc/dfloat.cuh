// Two-float ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the error-free
// transformations of Knuth (TwoSum: the rounding error of a float addition,
// six operations) and of Dekker / Ogita-Rump-Oishi with a fused multiply-add
// (TwoProd: the rounding error of a float product, two operations), combined
// as in the double-double arithmetic of Hida, Li and Bailey (2001).
//
// GB300 runs FP32 at 64 times its FP64 rate, so a residual formed with a
// dozen FP32 operations per term still costs a fraction of the FP64 pipe
// time of the same residual in binary64.  Used for the refinement residual
// r = b - W x of the mixed form, where b - x cancels and W x must be formed
// to well below the FP32 rounding level.
//
// The operations below need IEEE float arithmetic without reassociation
// (nvcc's default; no fast-math flags).  FMA contraction of a*b + c is
// harmless: every product here is already an explicit fmaf.
#pragma once
#include <cuda_runtime.h>

#ifndef CHAD_HD
#define CHAD_HD __host__ __device__ __forceinline__
#endif

namespace chad {

struct df {
  float hi, lo;
};

CHAD_HD df df_of(float a) { return df{a, 0.0f}; }

// s + e = a + b exactly (any magnitudes)
CHAD_HD df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df{s, e};
}
// s + e = a + b exactly, for |a| >= |b| (or a = 0)
CHAD_HD df quick_two_sum(float a, float b) {
  const float s = a + b;
  return df{s, b - (s - a)};
}
// p + e = a * b exactly (barring underflow)
CHAD_HD df two_prod(float a, float b) {
  const float p = a * b;
  return df{p, fmaf(a, b, -p)};
}

// a + b with the low parts added in float ("sloppy" addition of Hida, Li
// and Bailey): its error is O(2^-44 (|a| + |b|)), absolute, even when a and
// b cancel -- the bound a refinement residual needs (its terms cancel by
// design and its error must be small against them, not against the result).
CHAD_HD df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
CHAD_HD df df_neg(df a) { return df{-a.hi, -a.lo}; }
CHAD_HD df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
CHAD_HD df df_add_f(df a, float b) {
  const df s = two_sum(a.hi, b);
  return quick_two_sum(s.hi, s.lo + a.lo);
}
// a * b with b a float
CHAD_HD df df_mul_f(df a, float b) {
  const df p = two_prod(a.hi, b);
  return quick_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
CHAD_HD df df_mul(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  return quick_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
// acc + a * b (a, b floats): the product exactly, then the two-float sum
CHAD_HD df df_fma_ff(df acc, float a, float b) { return df_add(acc, two_prod(a, b)); }
// acc + a * b (a two-float, b float)
CHAD_HD df df_fma_f(df acc, df a, float b) { return df_add(acc, df_mul_f(a, b)); }

// binary64 <-> two-float.  hi is d rounded to float, lo the float nearest
// the remainder d - hi (exact in binary64), so hi + lo carries ~48 bits.
CHAD_HD df df_of_double(double d) {
  const float hi = float(d);
  return df{hi, float(d - double(hi))};
}
CHAD_HD double df_to_double(df a) { return double(a.hi) + double(a.lo); }

// A two-float accumulator as a scalar type, so that the templated model
// routines (the Jacobian-vector product and the stoichiometry) run in it
// unchanged: hi is the float sum of the terms, lo the float sum of the
// rounding errors that TwoSum and TwoProd recover (the cascaded summation
// "Sum2" of Ogita, Rump and Oishi, 2005).  lo is not renormalised into hi
// after each operation; the value is hi + lo, accurate to O(2^-44) times
// the sum of the magnitudes of the terms.  Products are only of a float
// coefficient and an accumulator (three operations); a sum of two
// accumulators is eight.
struct DF {
  float hi, lo;
  DF() = default;
  CHAD_HD DF(float a) : hi(a), lo(0.0f) {}
  CHAD_HD DF(float h, float l) : hi(h), lo(l) {}
  CHAD_HD df v() const { return df{hi, lo}; }
};
CHAD_HD DF operator+(DF a, DF b) {
  const df s = two_sum(a.hi, b.hi);
  return DF(s.hi, s.lo + (a.lo + b.lo));
}
CHAD_HD DF operator-(DF a) { return DF(-a.hi, -a.lo); }
CHAD_HD DF operator-(DF a, DF b) { return a + (-b); }
CHAD_HD DF operator*(float c, DF a) {
  const df p = two_prod(c, a.hi);
  return DF(p.hi, fmaf(c, a.lo, p.lo));
}
CHAD_HD DF operator*(DF a, float c) { return c * a; }
CHAD_HD DF& operator+=(DF& a, DF b) {
  a = a + b;
  return a;
}

}  // namespace chad
