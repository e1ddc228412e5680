// Double-double arithmetic for the host-side operator builder.
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 106 significant bits.  The
// error-free transformations are Knuth's TwoSum and the FMA-based TwoProduct;
// the compound operations follow Dekker (1971) and Hida, Li & Bailey,
// "Algorithms for quad-double precision floating point arithmetic" (2001).
// Only IEEE double operations and std::fma are used, so results are identical
// on every IEEE-754 host (this file must be compiled without FP contraction).
#pragma once
#include <cmath>

namespace ddm {

struct dd {
    double hi, lo;
    dd() : hi(0.0), lo(0.0) {}
    dd(double h) : hi(h), lo(0.0) {}
    dd(double h, double l) : hi(h), lo(l) {}
    explicit operator double() const { return hi + lo; }
};

inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return dd(s, e);
}
inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return dd(s, e);
}
inline dd two_prod(double a, double b) {
    double p = a * b;
    double e = std::fma(a, b, -p);
    return dd(p, e);
}

inline dd operator+(const dd& a, const dd& b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(const dd& a) { return dd(-a.hi, -a.lo); }
inline dd operator-(const dd& a, const dd& b) { return a + (-b); }
inline dd operator*(const dd& a, const dd& b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
inline dd operator/(const dd& a, const dd& b) {
    double q1 = a.hi / b.hi;
    dd r = a - b * dd(q1);
    double q2 = r.hi / b.hi;
    r = r - b * dd(q2);
    double q3 = r.hi / b.hi;
    dd q = quick_two_sum(q1, q2);
    return q + dd(q3);
}
inline dd& operator+=(dd& a, const dd& b) { a = a + b; return a; }
inline dd& operator-=(dd& a, const dd& b) { a = a - b; return a; }
inline dd& operator*=(dd& a, const dd& b) { a = a * b; return a; }
inline bool operator<(const dd& a, const dd& b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline dd ddabs(const dd& a) { return a.hi < 0 || (a.hi == 0 && a.lo < 0) ? -a : a; }

// pi to double-double precision
inline dd dd_pi() { return dd(3.141592653589793116e+00, 1.224646799147353207e-16); }

// sin and cos of a double-double argument by their Taylor series after the
// reductions x -> x - 2 pi k and sin(x) = cos(pi/2 - x); |x| <= pi/4 needs 28 terms
// for full double-double accuracy.
inline dd taylor_sin(const dd& x) {
    dd x2 = x * x, term = x, sum = x;
    for (int k = 1; k < 30; ++k) {
        term = term * x2 / dd((double)((2 * k) * (2 * k + 1)));
        sum = (k & 1) ? sum - term : sum + term;
    }
    return sum;
}
inline dd taylor_cos(const dd& x) {
    dd x2 = x * x, term(1.0), sum(1.0);
    for (int k = 1; k < 30; ++k) {
        term = term * x2 / dd((double)((2 * k - 1) * (2 * k)));
        sum = (k & 1) ? sum - term : sum + term;
    }
    return sum;
}
// sin(pi * p / q) and cos(pi * p / q) for integers, reduced exactly in the integers
// to an angle in [0, pi/4] before the series.
inline void sincos_pi_rational(long long p, long long q, dd* s, dd* c) {
    // reduce p/q to [0, 2): angle = pi * p / q
    long long twoq = 2 * q;
    p %= twoq;
    if (p < 0) p += twoq;
    // octant: angle in units of pi/4 is 4p/q
    long long oct = (4 * p) / q;           // 0..7
    long long rem = 4 * p - oct * q;       // angle = (pi/4) (oct + rem/q)
    dd r = dd_pi() * dd((double)rem) / dd((double)(4 * q));   // in [0, pi/4)
    dd sr = taylor_sin(r), cr = taylor_cos(r);
    // angle = oct * pi/4 + r
    dd h = dd(0.70710678118654757, -4.8336466567264567e-17);  // sqrt(1/2)
    dd sa, ca;
    switch (oct) {
        case 0: sa = sr; ca = cr; break;
        case 1: sa = h * (sr + cr); ca = h * (cr - sr); break;
        case 2: sa = cr; ca = -sr; break;
        case 3: sa = h * (cr - sr); ca = -(h * (sr + cr)); break;
        case 4: sa = -sr; ca = -cr; break;
        case 5: sa = -(h * (sr + cr)); ca = -(h * (cr - sr)); break;
        case 6: sa = -cr; ca = sr; break;
        default: sa = -(h * (cr - sr)); ca = h * (sr + cr); break;
    }
    *s = sa; *c = ca;
}

}  // namespace ddm
