// Double-double arithmetic for the plan precompute (host only).
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 106 significant bits.  The
// error-free transformations are Knuth's two-sum and the FMA-based two-product
// (Dekker/Knuth, as used by Hida, Li and Bailey's double-double library).  The
// translation unit that includes this header must be compiled without
// floating-point contraction (-ffp-contract=off) so that the compiler does not
// fuse the operations these transformations rely on; the results are then
// bit-identical on any IEEE-754 host with a correctly rounded fma().
#pragma once
#include <cmath>

namespace femfft {

struct dd {
  double hi, lo;
  dd() : hi(0.0), lo(0.0) {}
  dd(double h) : hi(h), lo(0.0) {}
  dd(double h, double l) : hi(h), lo(l) {}
  double to_double() const { return hi + lo; }
};

inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return dd(s, b - (s - a));
}
inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  return dd(s, (a - (s - bb)) + (b - bb));
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  return dd(p, std::fma(a, b, -p));
}
inline dd operator+(const dd& a, const dd& b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  double e = s.lo + t.hi;
  s = quick_two_sum(s.hi, e);
  e = s.lo + t.lo;
  return quick_two_sum(s.hi, e);
}
inline dd operator-(const dd& a) { return dd(-a.hi, -a.lo); }
inline dd operator-(const dd& a, const dd& b) { return a + (-b); }
inline dd operator*(const dd& a, const dd& b) {
  dd p = two_prod(a.hi, b.hi);
  double e = p.lo + (a.hi * b.lo + a.lo * b.hi);
  return quick_two_sum(p.hi, e);
}
inline dd operator/(const dd& a, const dd& b) {
  double q1 = a.hi / b.hi;
  dd r = a - dd(q1) * b;
  double q2 = r.hi / b.hi;
  r = r - dd(q2) * b;
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return q + dd(q3);
}
inline dd& operator+=(dd& a, const dd& b) { a = a + b; return a; }
inline dd& operator-=(dd& a, const dd& b) { a = a - b; return a; }
inline dd& operator*=(dd& a, const dd& b) { a = a * b; return a; }
inline bool operator<(const dd& a, const dd& b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline dd dd_abs(const dd& a) { return a.hi < 0.0 ? -a : a; }
inline dd dd_sqrt(const dd& a) {
  if (a.hi <= 0.0) return dd(0.0);
  double x = std::sqrt(a.hi);
  dd xx = two_prod(x, x);
  double corr = ((a - xx).hi) / (2.0 * x);
  return quick_two_sum(x, corr);
}

// pi to double-double precision
inline dd dd_pi() { return dd(3.141592653589793116e+00, 1.224646799147353207e-16); }

// sin and cos of pi * num / den for integers, |result| accurate to ~1e-30.
// Exact rational reduction to an octant, then Taylor series on |x| <= pi/4.
void dd_sincospi_frac(long long num, long long den, dd* s, dd* c);

}  // namespace femfft
