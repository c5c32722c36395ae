// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits.  On this GPU the
// float pipes issue 64 times more operations per clock than the float64
// pipe, so the residual of the refinement (which needs ~1e-14 relative
// accuracy, not float64 exactly) runs in this format.
//
// Error-free transformations:
//  * two_sum: Knuth's branch-free sum, s + e = a + b exactly
//    (D. E. Knuth, The Art of Computer Programming, vol. 2, 4.2.2).
//  * two_prod: with a fused multiply-add, p + e = a * b exactly
//    (the FMA form of Dekker's product, T. J. Dekker, Numer. Math. 18, 1971).
// df_add / df_fma renormalise once per operation ("sloppy" double-float
// addition: the relative error is a small multiple of 2^-48 unless the
// operands cancel, when the absolute error is bounded by the larger
// operand's 2^-48).
//
// split_f64 converts a float64 value to hi + lo with integer operations
// only (no float64 instruction, not even on the overflow path): hi takes the
// top 24 significant bits (truncated), lo the next 29 bits rounded to 24.
// Values below 2^-126 in magnitude map to zero; the fields here are many
// orders of magnitude larger.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace femfft {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
// exact scaling by a power of two
__device__ __forceinline__ df df_scale2(df a, float p2) { return {a.hi * p2, a.lo * p2}; }

// acc + a * b
__device__ __forceinline__ df df_fma(df a, df b, df acc) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  df s = two_sum(acc.hi, p);
  s.lo += acc.lo + e;
  return quick_two_sum(s.hi, s.lo);
}

// One term of a compensated dot product of double-float vectors (Dot2 of
// T. Ogita, S. M. Rump, S. Oishi, "Accurate sum and dot product", SIAM J.
// Sci. Comput. 26, 2005, with double-float operands): (s, c) += a * b.  The
// hi parts of the products are summed into s with two_sum; every rounding
// error and the cross terms go into the float correction c.  The carried
// dependency is one float addition per term; the running value is the
// unnormalised pair (s, c).
__device__ __forceinline__ void dot2_step(df a, df b, float& s, float& c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float t = s + p;
  const float z = t - s;
  const float sig = (s - (t - z)) + (p - z);
  s = t;
  c += sig + e;
}

__device__ __forceinline__ df split_f64(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(bits >> 32);
  const int e = (int)((hi32 >> 20) & 0x7ffu);   // biased float64 exponent
  if (e > 1150) {   // |x| >= 2^128 rounds to infinity in float; nan stays nan
    const bool nan = e == 2047 && (bits & 0x000fffffffffffffull) != 0;
    return {__uint_as_float((hi32 & 0x80000000u) | 0x7f800000u | (nan ? 0x00400000u : 0u)), 0.0f};
  }
  if (e < 897) return {0.0f, 0.0f};                   // |x| < 2^-126
  const unsigned sign = hi32 & 0x80000000u;
  const unsigned long long mant = bits & 0x000fffffffffffffull;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(mant >> 29));
  // x - hi = rem * 2^-52 * 2^(e-1023), rem the low 29 bits of the significand
  const unsigned rem = (unsigned)(mant & 0x1fffffffu);
  const float scale = __uint_as_float(sign | ((unsigned)(e - 896) << 23));   // +-2^(e-1023)
  const float lo = (__uint2float_rn(rem) * 2.220446049250313080847263336181640625e-16f) * scale;
  return {hi, lo};
}

// the value rounded to float
__device__ __forceinline__ float df_to_float(df a) { return a.hi + a.lo; }

}  // namespace femfft
