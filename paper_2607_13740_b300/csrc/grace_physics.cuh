// Device-side physics and basis functions of the GRACE-DG hot path.
//
// The kernels and breakage functions are templates over a parameter view: ParPlain reads the
// group's parameters as doubles (the tables T); ParSeed reads them as dual numbers whose
// derivative part is 1 for one parameter (the exact tables dT/dtheta, same operations).
#pragma once

#include "grace_dual.cuh"
#include "grace_internal.h"

namespace grace {

struct ParPlain {
    const DevGroup &G;
    __device__ double coag(int i) const { return G.coag_p[i]; }
    __device__ double frag(int i) const { return G.frag_p[i]; }
    __device__ double brk(int i) const { return G.break_p[i]; }
    __device__ double beta_coag() const { return G.beta_coag; }
    __device__ double beta_frag() const { return G.beta_frag; }
};

// parameter id: 0..7 coag_p[i], 8..15 frag_p[i - 8], 16..23 break_p[i - 16]; dbeta_* the
// derivatives of the Maxwellian probabilities along that parameter (computed on the host)
struct ParSeed {
    const DevGroup &G;
    int id;
    double dbeta_coag, dbeta_frag;
    __device__ Dual coag(int i) const { return Dual(G.coag_p[i], id == i ? 1.0 : 0.0); }
    __device__ Dual frag(int i) const { return Dual(G.frag_p[i], id == 8 + i ? 1.0 : 0.0); }
    __device__ Dual brk(int i) const { return Dual(G.break_p[i], id == 16 + i ? 1.0 : 0.0); }
    __device__ Dual beta_coag() const { return Dual(G.beta_coag, dbeta_coag); }
    __device__ Dual beta_frag() const { return Dual(G.beta_frag, dbeta_frag); }
};

template <class PV> using par_t = decltype(((const PV *)nullptr)->coag(0));

// Legendre polynomials phi_i (eq. 2.4) and derivatives at xi, i = 0..k
__device__ __forceinline__ void dev_legendre(int k, double xi, double *P, double *dP)
{
    P[0] = 1.0;
    if (dP) dP[0] = 0.0;
    if (k >= 1) {
        P[1] = xi;
        if (dP) dP[1] = 1.0;
    }
    for (int n = 1; n < k; ++n) {
        double c = 2.0 * n + 1.0;
        P[n + 1] = (c * xi * P[n] - n * P[n - 1]) / (n + 1.0);
        if (dP) dP[n + 1] = dP[n - 1] + c * P[n];
    }
}

// geometric cross section of Sec. 4.5 in mass units
__device__ __forceinline__ double dev_sigma(double u, double v)
{
    double r = cbrt(u) + cbrt(v);
    return 3.141592653589793 * r * r;
}

// ballistic cross section with a turbulent relative velocity and a linear
// fragmentation ramp (library model for the large disk batches)
template <class S>
__device__ __forceinline__ void ballistic_t(const S *p, double u, double v, S *kc, S *kf)
{
    const double pi = 3.141592653589793;
    S rho = p[0], sig = p[1], cs = p[2], alpha = p[3], vf = p[4], wr = p[5];
    S au = cbrt(3.0 * u / (4.0 * pi * rho));
    S av = cbrt(3.0 * v / (4.0 * pi * rho));
    S st = pi * rho * fmax(au, av) / (2.0 * sig);
    S dv = cs * sqrt(3.0 * alpha * st / (1.0 + st * st));
    S pf = fmin(fmax((dv - (1.0 - wr) * vf) / (2.0 * wr * vf), 0.0), 1.0);
    S rate = p[6] * pi * (au + av) * (au + av) * dv;
    *kc = rate * (1.0 - pf);
    *kf = rate * pf;
}

__device__ __forceinline__ void dev_ballistic(const double *p, double u, double v, double *kc, double *kf)
{
    ballistic_t<double>(p, u, v, kc, kf);
}

// The ballistic-turbulent kernels factor through sqrt(alpha_turb):
//   K_coag = s S0(u, v) (1 - pf(s D0)),  K_frag = s S0(u, v) pf(s D0),  s = sqrt(alpha_turb),
// with D0 = c_s sqrt(3 St / (1 + St^2)) a function of the larger particle only (St
// from max(a_u, a_v)), S0 = p6 pi (a_u + a_v)^2 D0, and pf(z) = clamp((z - (1 - w) v_f)
// / (2 w v_f), 0, 1).  A per-cell alpha_turb then enters only through s and pf.
__device__ __forceinline__ void dev_ballistic_split(const double *p, double u, double v, double *S0, double *D0)
{
    const double pi = 3.141592653589793;
    double rho = p[0], sig = p[1], cs = p[2];
    double au = cbrt(3.0 * u / (4.0 * pi * rho));
    double av = cbrt(3.0 * v / (4.0 * pi * rho));
    double st = pi * rho * fmax(au, av) / (2.0 * sig);
    double d0 = cs * sqrt(3.0 * st / (1.0 + st * st));
    *D0 = d0;
    *S0 = p[6] * pi * (au + av) * (au + av) * d0;
}

// fragmentation probability of the ramp as a function of z = s D0
__device__ __forceinline__ double dev_pfrag(const double *p, double z)
{
    const double vf = p[4], wr = p[5];
    return fmin(fmax((z - (1.0 - wr) * vf) / (2.0 * wr * vf), 0.0), 1.0);
}

template <class PV>
__device__ __forceinline__ par_t<PV> kcoag_t(const DevGroup &G, const PV &pv, double u, double v)
{
    using S = par_t<PV>;
    switch (G.coag_kind) {
    case GRACE_COAG_CONST: return pv.coag(0);
    case GRACE_COAG_ADD: return pv.coag(0) * (u + v);
    case GRACE_COAG_MULT: return pv.coag(0) * u * v;
    case GRACE_COAG_MAXWELL: return dev_sigma(u, v) * pv.coag(0) * pv.beta_coag();
    case GRACE_COAG_BALLISTIC: {
        S p[7], kc, kf;
        for (int i = 0; i < 7; ++i) p[i] = pv.coag(i);
        ballistic_t<S>(p, u, v, &kc, &kf);
        return kc;
    }
    default: return S(0.0);
    }
}

template <class PV>
__device__ __forceinline__ par_t<PV> kfrag_t(const DevGroup &G, const PV &pv, double u, double v)
{
    using S = par_t<PV>;
    switch (G.frag_kind) {
    case GRACE_FRAG_MULT: return pv.frag(0) * u * v;
    case GRACE_FRAG_MAXWELL: return dev_sigma(u, v) * pv.frag(0) * pv.beta_frag();
    case GRACE_FRAG_BALLISTIC: {
        S p[7], kc, kf;
        for (int i = 0; i < 7; ++i) p[i] = pv.frag(i);
        ballistic_t<S>(p, u, v, &kc, &kf);
        return kf;
    }
    default: return S(0.0);
    }
}

__device__ __forceinline__ double dev_kcoag(const DevGroup &G, double u, double v) { return kcoag_t(G, ParPlain{G}, u, v); }
__device__ __forceinline__ double dev_kfrag(const DevGroup &G, double u, double v) { return kfrag_t(G, ParPlain{G}, u, v); }

// m_frag / (y + z) of eq. (mfrag) as a function of the mass ratio q >= 1
__device__ __forceinline__ double dev_mfrag_ratio(double q)
{
    const double pi = 3.141592653589793;
    if (q <= 10.0) return 1.0;
    if (q <= 12.0) return (6.5 + 4.5 * cos(0.5 * (q - 10.0) * pi)) / (1.0 + q);
    if (q <= 15.0) return 2.0 / (1.0 + q);
    if (q <= 50.0) return (1.45 + 0.55 * cos((q - 15.0) / 35.0 * pi)) / (1.0 + q);
    return 0.9 / (1.0 + q);
}

template <class S> struct FragOutcomeT { double mfrag, mleft, mcut; S alpha; };
using FragOutcome = FragOutcomeT<double>;

template <class PV>
__device__ __forceinline__ FragOutcomeT<par_t<PV>> outcome_t(const DevGroup &G, const PV &pv, double u, double v)
{
    FragOutcomeT<par_t<PV>> o;
    double hi = fmax(u, v), lo = fmin(u, v), tot = u + v;
    o.alpha = pv.brk(0);
    o.mfrag = G.mfrag_mode == 1 ? tot : tot * dev_mfrag_ratio(hi / lo);
    o.mleft = fmax(tot - o.mfrag, 0.0);
    o.mcut = G.cutoff_mode == 1 ? hi : o.mfrag;
    return o;
}

__device__ __forceinline__ FragOutcome dev_outcome(const DevGroup &G, double u, double v)
{
    return outcome_t(G, ParPlain{G}, u, v);
}

// share of the power-law fragment mass (eq. break, normalised on [x_min, m_cut]) at or below x
template <class S>
__device__ __forceinline__ S pl_fraction_t(double x, double xmin, double mcut, S alpha)
{
    if (!(mcut > xmin)) return S(x > xmin ? 1.0 : 0.0);
    S e = 2.0 + alpha;
    S f = (pow(x, e) - pow(xmin, e)) / (pow(mcut, e) - pow(xmin, e));
    return fmin(fmax(f, 0.0), 1.0);
}

// product mass strictly above x (eq. inte1)
template <class PV>
__device__ __forceinline__ par_t<PV> mass_above_t(const DevGroup &G, const PV &pv, double x, double u, double v)
{
    using S = par_t<PV>;
    switch (G.break_kind) {
    case GRACE_BREAK_UNIFORM_BINARY:
        return S((u > x ? (u * u - x * x) / u : 0.0) + (v > x ? (v * v - x * x) / v : 0.0));
    case GRACE_BREAK_POWERLAW_REMNANT: {
        const auto o = outcome_t(G, pv, u, v);
        S m = o.mfrag * (1.0 - pl_fraction_t(x, G.x_min, o.mcut, o.alpha));
        return m + (o.mleft > x ? o.mleft : 0.0);
    }
    case GRACE_BREAK_COAG_DELTA:
        return S(u + v > x ? u + v : 0.0);
    default: return S(0.0);
    }
}

// product mass in [x_min, x] (eq. inte2)
template <class PV>
__device__ __forceinline__ par_t<PV> mass_below_t(const DevGroup &G, const PV &pv, double x, double u, double v)
{
    using S = par_t<PV>;
    double xm = G.x_min;
    switch (G.break_kind) {
    case GRACE_BREAK_UNIFORM_BINARY: {
        double mu = fmin(x, u), mv = fmin(x, v), m = 0.0;
        if (mu > xm) m += (mu * mu - xm * xm) / u;
        if (mv > xm) m += (mv * mv - xm * xm) / v;
        return S(m);
    }
    case GRACE_BREAK_POWERLAW_REMNANT: {
        const auto o = outcome_t(G, pv, u, v);
        S m = o.mfrag * pl_fraction_t(x, xm, o.mcut, o.alpha);
        return m + ((o.mleft >= xm && o.mleft <= x) ? o.mleft : 0.0);
    }
    case GRACE_BREAK_COAG_DELTA:
        return S(u + v <= x ? u + v : 0.0);
    default: return S(0.0);
    }
}

__device__ __forceinline__ double dev_mass_above(const DevGroup &G, double x, double u, double v)
{
    return mass_above_t(G, ParPlain{G}, x, u, v);
}

__device__ __forceinline__ double dev_mass_below(const DevGroup &G, double x, double u, double v)
{
    return mass_below_t(G, ParPlain{G}, x, u, v);
}

__device__ __forceinline__ double dev_vmax(const DevGroup &G, double u)
{
    return G.flux_mode == GRACE_FLUX_CONSERVATIVE ? G.x_max - u + G.x_min : G.x_max;
}

}  // namespace grace
