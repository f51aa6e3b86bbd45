// Double-double ("dd") arithmetic for the host-side plan builder: a value is
// the unevaluated sum hi + lo of two doubles with |lo| <= ulp(hi)/2, built
// from the error-free transformations TwoSum (Knuth) and TwoProd (fma).
// Used only while building plan tables, so that every stored FP64 constant
// is correctly rounded from a ~1e-32-accurate value.
#pragma once

#include <cmath>

namespace shtb {

struct DD {
    double hi, lo;
};

inline DD dd(double a) { return {a, 0.0}; }

inline DD two_sum(double a, double b)
{
    double s = a + b;
    double v = s - a;
    return {s, (a - (s - v)) + (b - v)};
}

inline DD fast_two_sum(double a, double b)    // requires |a| >= |b|
{
    double s = a + b;
    return {s, b - (s - a)};
}

inline DD operator+(DD x, DD y)
{
    DD s = two_sum(x.hi, y.hi);
    DD t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

inline DD operator-(DD x) { return {-x.hi, -x.lo}; }
inline DD operator-(DD x, DD y) { return x + (-y); }

inline DD operator*(DD x, DD y)
{
    double p = x.hi * y.hi;
    double e = std::fma(x.hi, y.hi, -p);
    e += x.hi * y.lo + x.lo * y.hi;
    return fast_two_sum(p, e);
}

inline DD operator*(DD x, double d)
{
    double p = x.hi * d;
    double e = std::fma(x.hi, d, -p);
    e += x.lo * d;
    return fast_two_sum(p, e);
}

inline DD operator/(DD x, DD y)
{
    double q1 = x.hi / y.hi;
    DD r = x - y * q1;
    double q2 = r.hi / y.hi;
    r = r - y * q2;
    double q3 = r.hi / y.hi;
    return fast_two_sum(q1, q2) + dd(q3);
}

inline DD sqrt(DD x)
{
    if (x.hi <= 0.0) return dd(0.0);
    double s = std::sqrt(x.hi);
    double p = s * s;
    double e = std::fma(s, s, -p);
    double r = ((x.hi - p) - e + x.lo) / (2.0 * s);
    return fast_two_sum(s, r);
}

// exact product of two integers below 2^53 as a dd
inline DD ddmul(double a, double b)
{
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}

inline double to_double(DD x) { return x.hi + x.lo; }

// pi as a dd
constexpr double kPiHi = 3.141592653589793116e+00;
constexpr double kPiLo = 1.224646799147353207e-16;

}  // namespace shtb
