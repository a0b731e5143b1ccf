/* Forward-mode dual numbers for the oracle's derivative build (test infrastructure only).
 *
 * A dual x = (v, d) carries a value and its derivative with respect to one seeded input; every
 * operation applies the chain rule of calculus to the pair, so a program evaluated on duals
 * returns the exact derivative of its own floating-point arithmetic (up to the rounding of the
 * derivative's arithmetic).  Comparisons look at the value only: a branch, a clamp or a max picks
 * the branch of the value and differentiates that branch (one-sided at a kink, which has measure
 * zero). */
#pragma once
#include <cmath>

struct dual {
    double v, d;
    dual() = default;
    dual(double x) : v(x), d(0.0) {}
    dual(double x, double y) : v(x), d(y) {}
    dual &operator+=(const dual &b) { d += b.d; v += b.v; return *this; }
    dual &operator-=(const dual &b) { d -= b.d; v -= b.v; return *this; }
    dual &operator*=(const dual &b) { d = d * b.v + v * b.d; v *= b.v; return *this; }
    /* (a / b)' = (a' - (a / b) b') / b, written without b^2 (which underflows for tiny b) */
    dual &operator/=(const dual &b) { v /= b.v; d = (d - v * b.d) / b.v; return *this; }
};

inline dual operator-(const dual &a) { return dual(-a.v, -a.d); }
inline dual operator+(const dual &a, const dual &b) { return dual(a.v + b.v, a.d + b.d); }
inline dual operator-(const dual &a, const dual &b) { return dual(a.v - b.v, a.d - b.d); }
inline dual operator*(const dual &a, const dual &b) { return dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline dual operator/(const dual &a, const dual &b)
{
    const double q = a.v / b.v;
    return dual(q, (a.d - q * b.d) / b.v);
}
inline dual operator+(const dual &a, double b) { return dual(a.v + b, a.d); }
inline dual operator+(double a, const dual &b) { return dual(a + b.v, b.d); }
inline dual operator-(const dual &a, double b) { return dual(a.v - b, a.d); }
inline dual operator-(double a, const dual &b) { return dual(a - b.v, -b.d); }
inline dual operator*(const dual &a, double b) { return dual(a.v * b, a.d * b); }
inline dual operator*(double a, const dual &b) { return dual(a * b.v, a * b.d); }
inline dual operator/(const dual &a, double b) { return dual(a.v / b, a.d / b); }
inline dual operator/(double a, const dual &b)
{
    const double q = a / b.v;
    return dual(q, -q * b.d / b.v);
}

inline bool operator<(const dual &a, const dual &b) { return a.v < b.v; }
inline bool operator>(const dual &a, const dual &b) { return a.v > b.v; }
inline bool operator<=(const dual &a, const dual &b) { return a.v <= b.v; }
inline bool operator>=(const dual &a, const dual &b) { return a.v >= b.v; }
inline bool operator<(const dual &a, double b) { return a.v < b; }
inline bool operator>(const dual &a, double b) { return a.v > b; }
inline bool operator<=(const dual &a, double b) { return a.v <= b; }
inline bool operator>=(const dual &a, double b) { return a.v >= b; }
inline bool operator<(double a, const dual &b) { return a < b.v; }
inline bool operator>(double a, const dual &b) { return a > b.v; }

/* d sqrt(x) = dx / (2 sqrt(x)); d cbrt(x) = dx / (3 cbrt(x)^2); d exp(x) = exp(x) dx;
   d erf(x) = (2 / sqrt(pi)) exp(-x^2) dx; d log(x) = dx / x */
inline dual sqrt(const dual &a)
{
    const double s = std::sqrt(a.v);
    return dual(s, a.d / (2.0 * s));
}
inline dual cbrt(const dual &a)
{
    const double c = std::cbrt(a.v);
    return dual(c, a.d / (3.0 * c * c));
}
inline dual exp(const dual &a)
{
    const double e = std::exp(a.v);
    return dual(e, e * a.d);
}
inline dual erf(const dual &a)
{
    return dual(std::erf(a.v), 1.1283791670955126 * std::exp(-a.v * a.v) * a.d);
}
inline dual log(const dual &a) { return dual(std::log(a.v), a.d / a.v); }
/* d x^y = x^y (y dx / x + log(x) dy) */
inline dual pow(double x, const dual &y)
{
    const double p = std::pow(x, y.v);
    return dual(p, y.d == 0.0 ? 0.0 : p * std::log(x) * y.d);
}
inline dual pow(const dual &x, double y)
{
    return dual(std::pow(x.v, y), x.d == 0.0 ? 0.0 : y * std::pow(x.v, y - 1.0) * x.d);
}
inline dual pow(const dual &x, const dual &y)
{
    const double p = std::pow(x.v, y.v);
    double d = 0.0;
    if (x.d != 0.0) d += y.v * std::pow(x.v, y.v - 1.0) * x.d;
    if (y.d != 0.0) d += p * std::log(x.v) * y.d;
    return dual(p, d);
}
inline dual fabs(const dual &a) { return a.v < 0.0 ? -a : a; }
inline dual fmax(const dual &a, const dual &b) { return a.v >= b.v ? a : b; }
inline dual fmin(const dual &a, const dual &b) { return a.v <= b.v ? a : b; }
