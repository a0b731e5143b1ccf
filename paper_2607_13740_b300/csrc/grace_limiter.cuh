// Scaling limiter of eqs. (recon) and (gamma): minimum of a bin's polynomial
// (closed form for k <= 3; for k = 4 the stationary points are bracketed between the
// roots of the second derivative and found by bisection), an FP32 positivity
// pre-test and the limiter itself.
#pragma once

#include "grace_convert.cuh"
#include "grace_physics.cuh"

namespace grace {

constexpr int kBinMax = kKMax + 1;

__device__ __forceinline__ double poly(const double *c, int k, double xi)
{
    double P[kBinMax];
    dev_legendre(k, xi, P, nullptr);
    double s = 0.0;
    for (int i = 0; i <= k; ++i) s += c[i] * P[i];
    return s;
}

// Minimum over [-1, 1] of p = sum_{i <= 4} c_i phi_i for degree 4, in the arithmetic of T.  The
// derivative p' = a0 + a1 x + a2 x^2 + a3 x^3 (a0 = c1 - 3/2 c3, a1 = 3 c2 - 15/2 c4, a2 = 15/2 c3,
// a3 = 35/2 c4) is monotone between consecutive roots of p'' = a1 + 2 a2 x + 3 a3 x^2, so each such
// piece of [-1, 1] holds at most one stationary point, located by bisection on the sign of p'
// (ITERS halvings); the minimum is taken over the end points and those points.
template <typename T, int ITERS, typename Eval>
__device__ __forceinline__ T quartic_minimum(const T *c, Eval p)
{
    const T a0 = c[1] - T(1.5) * c[3], a1 = T(3) * c[2] - T(7.5) * c[4], a2 = T(7.5) * c[3], a3 = T(17.5) * c[4];
    auto dp = [&](T x) { return a0 + x * (a1 + x * (a2 + x * a3)); };
    // roots of p'' (a quadratic, 3 a3 x^2 + 2 a2 x + a1) inside (-1, 1), sorted
    T br[4];
    int nb = 0;
    br[nb++] = T(-1);
    {
        const T A = T(3) * a3, B = T(2) * a2, C = a1;
        T r0 = T(2), r1 = T(2);
        if (A == T(0)) {
            if (B != T(0)) r0 = -C / B;
        } else {
            const T disc = B * B - T(4) * A * C;
            if (disc >= T(0)) {
                const T sq = sqrt(disc);
                const T qq = T(-0.5) * (B + copysign(sq, B));
                if (qq != T(0)) {
                    r0 = qq / A;
                    r1 = C / qq;
                } else {
                    r0 = T(0);
                }
            }
        }
        if (r1 < r0) {
            const T t = r0;
            r0 = r1;
            r1 = t;
        }
        if (r0 > T(-1) && r0 < T(1)) br[nb++] = r0;
        if (r1 > T(-1) && r1 < T(1)) br[nb++] = r1;
    }
    br[nb++] = T(1);
    T m = p(T(-1)) < p(T(1)) ? p(T(-1)) : p(T(1));
    for (int s = 0; s + 1 < nb; ++s) {
        T lo = br[s], hi = br[s + 1];
        const T dlo = dp(lo), dhi = dp(hi);
        if (!((dlo < T(0) && dhi > T(0)) || (dlo > T(0) && dhi < T(0)))) continue;
        const bool rising = dlo < T(0);
        for (int it = 0; it < ITERS; ++it) {
            const T mid = T(0.5) * (lo + hi);
            if ((dp(mid) < T(0)) == rising) lo = mid;
            else hi = mid;
        }
        const T v = p(T(0.5) * (lo + hi));
        if (v < m) m = v;
    }
    return m;
}

// minimum over [-1, 1] of sum_i c_i phi_i: endpoints and interior stationary points
__device__ __forceinline__ double bin_minimum(const double *c, int k)
{
    if (k == 4) return quartic_minimum<double, 64>(c, [&](double x) { return poly(c, k, x); });
    if (k == 0) return c[0];
    double m = fmin(poly(c, k, -1.0), poly(c, k, 1.0));
    if (k == 2 && c[2] != 0.0) {
        const double xs = -c[1] / (3.0 * c[2]);          // phi_1' = 1, phi_2' = 3 xi
        if (xs > -1.0 && xs < 1.0) m = fmin(m, poly(c, k, xs));
    } else if (k == 3) {
        // derivative 7.5 c3 xi^2 + 3 c2 xi + (c1 - 1.5 c3)
        const double A = 7.5 * c[3], B = 3.0 * c[2], C = c[1] - 1.5 * c[3];
        double r0 = 2.0, r1 = 2.0;
        if (A == 0.0) {
            if (B != 0.0) r0 = -C / B;
        } else {
            const double disc = B * B - 4.0 * A * C;
            if (disc >= 0.0) {
                const double sq = sqrt(disc);
                const double qq = -0.5 * (B + copysign(sq, B));
                if (qq != 0.0) {
                    r0 = qq / A;
                    r1 = C / qq;
                } else {
                    r0 = 0.0;
                }
            }
        }
        if (r0 > -1.0 && r0 < 1.0) m = fmin(m, poly(c, k, r0));
        if (r1 > -1.0 && r1 < 1.0) m = fmin(m, poly(c, k, r1));
    }
    return m;
}

// FP32 test that a bin's polynomial (coefficients cf, already in FP32) is
// clearly positive on [-1, 1]: then the FP64 scaling limiter would leave it
// untouched (gamma = 1) and can be skipped.  The margin covers FP32 rounding of
// the evaluation (coefficients summed in |.|).
__device__ __forceinline__ float bin_minimum_f(const float *c, int k);

__device__ __forceinline__ bool clearly_positive_f(const float *cf, int k)
{
    float s = 0.f;
    for (int i = 0; i <= k; ++i) s += fabsf(cf[i]);
    if (!(cf[0] > 0.f)) return false;
    float m = cf[0];
    if (k >= 1) {
        // end points: p(1) = sum c_i, p(-1) = sum (-1)^i c_i
        float p1 = 0.f, pm = 0.f;
        for (int i = 0; i <= k; ++i) {
            p1 += cf[i];
            pm += (i & 1) ? -cf[i] : cf[i];
        }
        m = fminf(p1, pm);
        if (k == 4) {
            m = bin_minimum_f(cf, k);
        } else if (k == 2 && cf[2] != 0.f) {
            const float xs = -cf[1] / (3.f * cf[2]);
            if (xs > -1.f && xs < 1.f) m = fminf(m, cf[0] + cf[1] * xs + cf[2] * (1.5f * xs * xs - 0.5f));
        } else if (k == 3) {
            const float A = 7.5f * cf[3], B = 3.f * cf[2], C = cf[1] - 1.5f * cf[3];
            const float disc = B * B - 4.f * A * C;
            if (A != 0.f && disc >= 0.f) {
                const float sq = sqrtf(disc);
                const float r[2] = {(-B - sq) / (2.f * A), (-B + sq) / (2.f * A)};
                for (int t = 0; t < 2; ++t)
                    if (r[t] > -1.f && r[t] < 1.f) {
                        const float x = r[t];
                        m = fminf(m, cf[0] + cf[1] * x + cf[2] * (1.5f * x * x - 0.5f) +
                                         cf[3] * (2.5f * x * x * x - 1.5f * x));
                    }
            } else {
                return false;   // let the exact path decide
            }
        }
    }
    return m > 1e-5f * s;
}

__device__ __forceinline__ bool clearly_positive(const double *c, int k)
{
    float cf[kBinMax];
    for (int i = 0; i <= k; ++i) cf[i] = (float)c[i];
    return clearly_positive_f(cf, k);
}

// The same test for a bin whose mean v0 is FP64 and whose higher modes are FP32:
// everything is rescaled by the power of two that brings v0 into [1, 2), so the
// test holds at any magnitude (integer operations only, no FP64 arithmetic).
__device__ __forceinline__ bool clearly_positive_mixed(double v0, const float *c, int k)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v0);
    const uint32_t hi = (uint32_t)(u >> 32);
    const int e0 = (int)((hi >> 20) & 0x7FFu);
    if ((hi >> 31) || e0 == 0 || e0 == 0x7FF) return false;   // v0 <= 0, subnormal, inf or nan
    float cf[kBinMax];
    cf[0] = __uint_as_float(0x3F800000u | ((hi & 0xFFFFFu) << 3));   // mantissa of v0, truncated
    for (int i = 1; i <= k; ++i) cf[i] = scale_pow2(c[i], 1023 - e0);
    return clearly_positive_f(cf, k);
}

// sum_i c_i phi_i(x) in FP32 (Legendre polynomials up to degree 4)
__device__ __forceinline__ float poly_f(const float *c, int k, float x)
{
    float s = c[0];
    if (k >= 1) s += c[1] * x;
    if (k >= 2) s += c[2] * (1.5f * x * x - 0.5f);
    if (k >= 3) s += c[3] * (2.5f * x * x * x - 1.5f * x);
    if (k >= 4) {
        const float x2 = x * x;
        s += c[4] * (4.375f * x2 * x2 - 3.75f * x2 + 0.375f);
    }
    return s;
}

// minimum over [-1, 1] in FP32: end points and interior stationary points
__device__ __forceinline__ float bin_minimum_f(const float *c, int k)
{
    if (k == 4) return quartic_minimum<float, 28>(c, [&](float x) { return poly_f(c, k, x); });
    float m = fminf(poly_f(c, k, 1.f), poly_f(c, k, -1.f));
    if (k == 2 && c[2] != 0.f) {
        const float xs = -c[1] / (3.f * c[2]);
        if (xs > -1.f && xs < 1.f) m = fminf(m, poly_f(c, k, xs));
    } else if (k == 3) {
        // derivative 7.5 c3 x^2 + 3 c2 x + (c1 - 1.5 c3)
        const float A = 7.5f * c[3], B = 3.f * c[2], C = c[1] - 1.5f * c[3];
        float r0 = 2.f, r1 = 2.f;
        if (A == 0.f) {
            if (B != 0.f) r0 = -C / B;
        } else {
            const float disc = B * B - 4.f * A * C;
            if (disc >= 0.f) {
                const float sq = sqrtf(disc);
                const float qq = -0.5f * (B + copysignf(sq, B));
                if (qq != 0.f) {
                    r0 = qq / A;
                    r1 = C / qq;
                } else {
                    r0 = 0.f;
                }
            }
        }
        if (r0 > -1.f && r0 < 1.f) m = fminf(m, poly_f(c, k, r0));
        if (r1 > -1.f && r1 < 1.f) m = fminf(m, poly_f(c, k, r1));
    }
    return m;
}

// Scaling limiter (eqs. (recon), (gamma)) evaluated in FP32 on a bin rescaled by
// the power of two that brings its FP64 mean v0 into [1, 2): cf[0] is set here
// from v0, the caller passes the rescaled higher modes in cf[1..k] (rescale by
// 2^(1023 - e0), e0 from scaled_exponent).  Returns gamma in (0, 1]; a bin whose
// FP32 minimum lies within the evaluation's rounding (1e-6 of sum |cf|) of zero
// or above is left alone (gamma = 1).
__device__ __forceinline__ int scaled_exponent(double v0)
{
    // biased exponent of v0 when v0 is positive, normal and finite, else -1
    const unsigned long long u = (unsigned long long)__double_as_longlong(v0);
    const int e0 = (int)((u >> 52) & 0x7FFull);
    return ((u >> 63) || e0 == 0 || e0 == 0x7FF) ? -1 : e0;
}

__device__ __forceinline__ float limiter_gamma_scaled(double v0, float *cf, int k)
{
    const uint32_t hi = (uint32_t)((unsigned long long)__double_as_longlong(v0) >> 32);
    cf[0] = __uint_as_float(0x3F800000u | ((hi & 0xFFFFFu) << 3));
    float s = 0.f;
    for (int i = 0; i <= k; ++i) s += fabsf(cf[i]);
    if (!(s < 3.0e38f)) return -1.f;   // a mode out of FP32 range relative to the mean: exact path
    const float m = bin_minimum_f(cf, k);
    if (!(m < -1e-6f * s)) return 1.f;
    return fminf(cf[0] / (cf[0] - m), 1.f);
}

// eq. (recon) with gamma from eq. (gamma); returns flag bits
__device__ __forceinline__ unsigned limit_bin(double *c, int k)
{
    if (k == 0) return 0u;
    if (clearly_positive(c, k)) return 0u;
    const double gbar = c[0];
    double gamma;
    unsigned f = 0u;
    if (gbar < 0.0) {
        gamma = 0.0;
        f |= GRACE_FLAG_NEGATIVE_MEAN;
    } else {
        const double den = gbar - bin_minimum(c, k);
        gamma = den > 0.0 ? fmin(gbar / den, 1.0) : 1.0;
    }
    if (gamma < 1.0) {
        f |= GRACE_FLAG_LIMITED;
        for (int i = 1; i <= k; ++i) c[i] *= gamma;
    }
    return f;
}

}  // namespace grace
