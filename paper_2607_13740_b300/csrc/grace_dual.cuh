// Forward-mode dual numbers for the exact parameter derivative of the FP64 precompute.
//
// A Dual carries a value and its derivative with respect to one physics parameter; the kernel
// and breakage functions and the flux quadrature, instantiated on Dual, produce dT_r/dtheta by
// the chain rule applied to the very operations that build T_r (no difference quotient).
// Branches and clamps look at the value, so a clamp contributes a zero derivative where it binds
// and the identity where it does not (one-sided at the kink itself).
//
// The type and its functions live in their own namespace: calls on plain doubles elsewhere in
// the library keep the CUDA math functions, and calls on Dual find these by argument lookup.
#pragma once

#include <cmath>

namespace grace {
namespace ad {

struct Dual {
    double val, der;
    Dual() = default;
    __host__ __device__ Dual(double v) : val(v), der(0.0) {}
    __host__ __device__ Dual(double v, double d) : val(v), der(d) {}
    __host__ __device__ Dual &operator+=(const Dual &o)
    {
        val += o.val;
        der += o.der;
        return *this;
    }
    __host__ __device__ Dual &operator-=(const Dual &o)
    {
        val -= o.val;
        der -= o.der;
        return *this;
    }
};

__host__ __device__ inline double value_of(double x) { return x; }
__host__ __device__ inline double value_of(const Dual &x) { return x.val; }
__host__ __device__ inline double deriv_of(double) { return 0.0; }
__host__ __device__ inline double deriv_of(const Dual &x) { return x.der; }

__host__ __device__ inline Dual operator-(const Dual &a) { return Dual(-a.val, -a.der); }
__host__ __device__ inline Dual operator+(const Dual &a, const Dual &b) { return Dual(a.val + b.val, a.der + b.der); }
__host__ __device__ inline Dual operator-(const Dual &a, const Dual &b) { return Dual(a.val - b.val, a.der - b.der); }
__host__ __device__ inline Dual operator*(const Dual &a, const Dual &b)
{
    return Dual(a.val * b.val, a.der * b.val + a.val * b.der);
}
__host__ __device__ inline Dual operator/(const Dual &a, const Dual &b)
{
    const double q = a.val / b.val;
    return Dual(q, (a.der - q * b.der) / b.val);
}
__host__ __device__ inline Dual operator+(const Dual &a, double b) { return Dual(a.val + b, a.der); }
__host__ __device__ inline Dual operator+(double a, const Dual &b) { return Dual(a + b.val, b.der); }
__host__ __device__ inline Dual operator-(const Dual &a, double b) { return Dual(a.val - b, a.der); }
__host__ __device__ inline Dual operator-(double a, const Dual &b) { return Dual(a - b.val, -b.der); }
__host__ __device__ inline Dual operator*(const Dual &a, double b) { return Dual(a.val * b, a.der * b); }
__host__ __device__ inline Dual operator*(double a, const Dual &b) { return Dual(a * b.val, a * b.der); }
__host__ __device__ inline Dual operator/(const Dual &a, double b) { return Dual(a.val / b, a.der / b); }
__host__ __device__ inline Dual operator/(double a, const Dual &b)
{
    const double q = a / b.val;
    return Dual(q, -q * b.der / b.val);
}

// d sqrt(x) = dx / (2 sqrt x); d cbrt(x) = dx / (3 cbrt(x)^2); d exp(x) = exp(x) dx;
// d erf(x) = 2 / sqrt(pi) exp(-x^2) dx
__host__ __device__ inline Dual sqrt(const Dual &a)
{
    const double r = ::sqrt(a.val);
    return Dual(r, 0.5 * a.der / r);
}
__host__ __device__ inline Dual cbrt(const Dual &a)
{
    const double r = ::cbrt(a.val);
    return Dual(r, a.der / (3.0 * r * r));
}
__host__ __device__ inline Dual exp(const Dual &a)
{
    const double r = ::exp(a.val);
    return Dual(r, r * a.der);
}
__host__ __device__ inline Dual erf(const Dual &a)
{
    constexpr double two_over_sqrt_pi = 1.1283791670955126;
    return Dual(::erf(a.val), two_over_sqrt_pi * ::exp(-a.val * a.val) * a.der);
}
// x^y with a constant base: d = x^y log(x) dy
__host__ __device__ inline Dual pow(double x, const Dual &y)
{
    const double r = ::pow(x, y.val);
    return Dual(r, y.der != 0.0 ? r * ::log(x) * y.der : 0.0);
}
// clamps and extrema select by value
__host__ __device__ inline Dual fmax(const Dual &a, const Dual &b) { return a.val >= b.val ? a : b; }
__host__ __device__ inline Dual fmin(const Dual &a, const Dual &b) { return a.val <= b.val ? a : b; }
__host__ __device__ inline Dual fmax(const Dual &a, double b) { return a.val >= b ? a : Dual(b); }
__host__ __device__ inline Dual fmin(const Dual &a, double b) { return a.val <= b ? a : Dual(b); }

}  // namespace ad
using ad::Dual;
using ad::value_of;
using ad::deriv_of;
}  // namespace grace
