// Scaling limiter of eqs. (recon) and (gamma): minimum of a bin's polynomial
// (closed form for k <= 3), an FP32 positivity pre-test and the limiter itself.
#pragma once

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

// minimum over [-1, 1] of sum_i c_i phi_i: endpoints and interior stationary points
__device__ __forceinline__ double bin_minimum(const double *c, int k)
{
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

// FP32 test that a bin's polynomial is clearly positive on [-1, 1]: then the FP64
// scaling limiter would leave it untouched (gamma = 1) and can be skipped.  The
// margin covers FP32 rounding of the evaluation (coefficients summed in |.|).
__device__ __forceinline__ bool clearly_positive(const double *c, int k)
{
    float cf[kBinMax], s = 0.f;
    for (int i = 0; i <= k; ++i) {
        cf[i] = (float)c[i];
        s += fabsf(cf[i]);
    }
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
        if (k == 2 && cf[2] != 0.f) {
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
