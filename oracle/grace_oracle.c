/*
 * GRACE-DG oracle: a plain, slow, FP64 CPU implementation of the
 * discontinuous-Galerkin coagulation-fragmentation solver of
 *   Yang, Chen & Bai, "GRACE-DG: A Discontinuous Galerkin Method-Based Code
 *   for General Nonlinear Coagulation-Fragmentation Equations" (arXiv 2607.13740).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library: every grid,
 * Legendre value, Gauss node and flux is computed here from the paper's
 * definitions, in the order the paper states them:
 *
 *   - grid and modal basis ............ Sec. 3.1, eqs. (2.2)-(2.5), (evo)
 *   - Gauss-Legendre rule (Q = k+1) ... Sec. 3.3, eq. (quad)
 *   - truncated fluxes ................. Sec. 3.3, eqs. (Fcoagtrun), (Ffragtrun),
 *                                        nested quadrature with partial bins A..B
 *   - fragmentation w-integrals ........ App. B, eqs. (inte1), (inte2)
 *   - reordered fragmentation volume term App. B (five sub-interval terms)
 *   - projection ....................... Sec. 3.2.1, eq. (init)
 *   - scaling limiter .................. Sec. 3.2.2, eqs. (recon), (gamma)
 *   - SSP-RK3 .......................... Sec. 3.2.3, eq. (RK3)
 *   - physics models ................... Sec. 4.5 (Maxwellian kernels,
 *                                        eqs. (break), (mfrag)), Sec. 4.4
 *
 * Readings of points where the paper is silent or garbled (both sides of the
 * parity tests follow the same reading):
 *   R1  flux_mode selects Delta x = -u + x_min (conservative) or 0.
 *   R2  the lower v limit is x - u + x_min in both modes.
 *   R3  the limiter runs once per full step, before the three RK stages.
 *   R4  gamma = 1 when gbar - min <= 0; gamma = 0 (flag bit 0) when gbar < 0.
 *   R5  every Gauss rule of the flux uses Q = k+1 nodes (quad_q overrides).
 *   R6  at a volume point x_j^theta the outer u-integral covers bins 0..j-1
 *       in full plus the partial piece [x_{j-1/2}, x_j^theta].
 *   R7  the App. B sub-intervals are taken from the un-reordered flux:
 *       positive terms live on x in (u, u+v-x_min), negative on (x_min, u),
 *       and v always runs over [x_min, v_max(u)].
 *   R8  each App. B sub-interval is integrated with its own Q-point Gauss rule.
 *   R9  fragmentation without a Dirac remnant uses Gauss on F(x_j^theta).
 *   R10 m_cut <= x_min puts all power-law fragment mass at x_min; a remnant
 *       with m_left < x_min is not counted below any x (w runs from x_min).
 *   R11 "above x" is strict (w > x), "below x" is x_min <= w <= x.
 *
 * Parity pins: see tests/test_oracle_*.py (closed forms, analytic solutions,
 * exact-polynomial cases, conservation, brute-force quadrature, convergence).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_QMAX 40
#define ORC_KMAX 8

/* Scalar type of every quantity that depends on the state g or on the physics parameters.
   This file, compiled as C, is the oracle and uses double.  grace_oracle_tangent.cpp compiles
   the same file as C++ with `real` a forward-mode dual number (value, derivative) to take exact
   derivatives of this arithmetic with respect to the state or one parameter; RV(x) is the value
   part (branches, flags and the limiter's minimum location are decided on values).  Grids, Gauss
   nodes, collision masses u, v and evaluation points x never depend on either and stay double. */
#ifndef ORC_TANGENT
typedef double real;
#define RV(x) (x)
#define REAL_IS_ZERO(x) ((x) == 0.0)
#define ORC_API
#endif

/* ------------------------------------------------------------------ */
/* public parameter block (mirrored by a ctypes.Structure in Python)   */
/* ------------------------------------------------------------------ */
enum { ORC_COAG_NONE = 0, ORC_COAG_CONST = 1, ORC_COAG_ADD = 2, ORC_COAG_MULT = 3,
       ORC_COAG_MAXWELL = 4, ORC_COAG_BALLISTIC = 5 };
enum { ORC_FRAG_NONE = 0, ORC_FRAG_MULT = 1, ORC_FRAG_MAXWELL = 2, ORC_FRAG_BALLISTIC = 3 };
enum { ORC_BREAK_UNIFORM_BINARY = 0, ORC_BREAK_POWERLAW_REMNANT = 1, ORC_BREAK_COAG_DELTA = 2 };
enum { ORC_IC_EXP = 0, ORC_IC_POWERLAW = 1, ORC_IC_FIRST_BIN = 2 };

typedef struct {
    int n_bins;      /* N                                                   */
    int order_k;     /* k: Legendre degree                                  */
    int quad_q;      /* Q: Gauss points; 0 means k+1                        */
    int flux_mode;   /* 0: conservative (Delta x = -u + x_min), 1: Delta x = 0 */
    int coag_kind;
    int frag_kind;
    int break_kind;
    int cutoff_mode; /* 0: power law up to m_frag (eq. break); 1: up to max(u,v) */
    int limiter;     /* 1: scaling limiter once per step (default); 0: off  */
    int mfrag_mode;  /* 0: eq. (mfrag); 1: destructive only, m_frag = u+v   */
    double x_min, x_max;
    double coag_p[8];
    double frag_p[8];
    double break_p[8];
    const double *edges;  /* n_bins + 1 bin edges from x_min to x_max, or NULL: the log grid */
} orc_params;

typedef struct {
    orc_params p;
    int N, k, Q, P;
    double *e;              /* N+1 bin edges x_{j-1/2}                    */
    double s[ORC_QMAX], w[ORC_QMAX];
    /* the physics parameters as read by the kernels and breakage functions */
    real coag_p[8], frag_p[8], break_p[8];
    /* Maxwellian collision probabilities (constant when dv_rms is constant) */
    real beta_coag, beta_frag;
} octx;

/* ------------------------------------------------------------------ */
/* Legendre basis (eq. 2.4) and its derivative                          */
/* ------------------------------------------------------------------ */
static void legendre(int k, double xi, double *P, double *dP)
{
    /* Bonnet recurrence (n+1) P_{n+1} = (2n+1) xi P_n - n P_{n-1};
       derivative P'_{n+1} = P'_{n-1} + (2n+1) P_n. */
    P[0] = 1.0;
    if (dP) dP[0] = 0.0;
    if (k >= 1) { P[1] = xi; if (dP) dP[1] = 1.0; }
    for (int n = 1; n < k; ++n) {
        P[n + 1] = ((2.0 * n + 1.0) * xi * P[n] - n * P[n - 1]) / (n + 1.0);
        if (dP) dP[n + 1] = dP[n - 1] + (2.0 * n + 1.0) * P[n];
    }
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights (eq. quad), by Newton on P_Q        */
/* ------------------------------------------------------------------ */
ORC_API int orc_gauss(int Q, double *s, double *w)
{
    if (Q < 1 || Q > ORC_QMAX) return -1;
    for (int i = 0; i < Q; ++i) {
        double x = cos(M_PI * (i + 0.75) / (Q + 0.5));
        double p0 = 1.0, p1 = x, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            p0 = 1.0; p1 = x;
            for (int n = 1; n < Q; ++n) {
                double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
                p0 = p1; p1 = p2;
            }
            dp = Q * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        /* final derivative at the converged root */
        p0 = 1.0; p1 = x;
        for (int n = 1; n < Q; ++n) {
            double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
            p0 = p1; p1 = p2;
        }
        dp = Q * (x * p1 - p0) / ((x - 1.0) * (x + 1.0));
        s[Q - 1 - i] = x;
        w[Q - 1 - i] = 2.0 / ((1.0 - x) * (1.0 + x) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* context                                                             */
/* ------------------------------------------------------------------ */
static real maxwell_below(real vth, real dv)
{
    /* beta_coag = int_0^{v_b} f_v dv (Sec. 4.5) */
    real a = sqrt(3.0 / (2.0 * dv * dv));
    return erf(a * vth) - vth * sqrt(6.0 / (M_PI * dv * dv)) * exp(-3.0 * vth * vth / (2.0 * dv * dv));
}

static real maxwell_above(real vth, real dv)
{
    /* beta_frag = int_{v_f}^inf f_v dv (Sec. 4.5) */
    real a = sqrt(3.0 / (2.0 * dv * dv));
    return 1.0 - erf(a * vth) + vth * sqrt(6.0 / (M_PI * dv * dv)) * exp(-3.0 * vth * vth / (2.0 * dv * dv));
}

static void ctx_betas(octx *c)
{
    if (c->p.coag_kind == ORC_COAG_MAXWELL)
        c->beta_coag = maxwell_below(c->coag_p[1], c->coag_p[0]);
    if (c->p.frag_kind == ORC_FRAG_MAXWELL)
        c->beta_frag = maxwell_above(c->frag_p[1], c->frag_p[0]);
}

static void ctx_free(octx *c) { free(c->e); c->e = NULL; }

static int ctx_init(octx *c, const orc_params *p)
{
    memset(c, 0, sizeof(*c));
    c->p = *p;
    c->N = p->n_bins;
    c->k = p->order_k;
    c->Q = p->quad_q > 0 ? p->quad_q : p->order_k + 1;
    if (c->N < 1 || c->k < 0 || c->k > ORC_KMAX || c->Q > ORC_QMAX) return -1;
    if (!(p->x_min > 0.0) || !(p->x_max > p->x_min)) return -1;
    c->P = c->N * (c->k + 1);
    c->e = (double *)malloc(sizeof(double) * (c->N + 1));
    if (!c->e) return -2;
    if (p->edges) {
        /* caller's grid: strictly increasing from x_min to x_max */
        for (int j = 0; j <= c->N; ++j) c->e[j] = p->edges[j];
        if (c->e[0] != p->x_min || c->e[c->N] != p->x_max) { ctx_free(c); return -1; }
        for (int j = 0; j < c->N; ++j)
            if (!(c->e[j + 1] > c->e[j])) { ctx_free(c); return -1; }
    } else {
        /* logarithmic grid (Sec. 3.1) */
        for (int j = 0; j <= c->N; ++j)
            c->e[j] = p->x_min * pow(p->x_max / p->x_min, (double)j / c->N);
        c->e[0] = p->x_min;
        c->e[c->N] = p->x_max;
    }
    orc_gauss(c->Q, c->s, c->w);
    for (int i = 0; i < 8; ++i) {
        c->coag_p[i] = p->coag_p[i];
        c->frag_p[i] = p->frag_p[i];
        c->break_p[i] = p->break_p[i];
    }
    ctx_betas(c);
    return 0;
}


/* ------------------------------------------------------------------ */
/* physics: kernels (Secs. 4.2-4.5) and breakage mass functions         */
/* ------------------------------------------------------------------ */
static double cross_section(double u, double v)
{
    /* sigma(x, y) = pi (x^{1/3} + y^{1/3})^2 (Sec. 4.5) */
    double r = cbrt(u) + cbrt(v);
    return M_PI * r * r;
}

/* ballistic kernel with a turbulent relative velocity: the project's own model
   for the large disk workloads (the paper gives no formula; parameters in p).
   The formula is pinned in the tests by what its definition fixes (symmetry, power
   laws in alpha, c_s, the rate scale and, for St << 1 and St >> 1, the grain mass;
   the larger grain setting St; St <-> 1/St invariance and the maximum at St = 1; the
   ramp's end and mid points); the flux quadrature with it is pinned against
   brute-force adaptive integration.  Parameters:
   p[0] = rho_s, p[1] = Sigma_g, p[2] = c_s, p[3] = alpha_turb, p[4] = v_frag,
   p[5] = ramp half-width fraction, p[6] = overall rate scale. */
static void ballistic(const real *p, double u, double v, real *kc, real *kf)
{
    real rho = p[0], sig = p[1], cs = p[2], alpha = p[3], vf = p[4], wr = p[5];
    real au = cbrt(3.0 * u / (4.0 * M_PI * rho));
    real av = cbrt(3.0 * v / (4.0 * M_PI * rho));
    real st = M_PI * rho * fmax(au, av) / (2.0 * sig);
    real dv = cs * sqrt(3.0 * alpha * st / (1.0 + st * st));
    real pf = (dv - (1.0 - wr) * vf) / (2.0 * wr * vf);
    if (pf < 0.0) pf = 0.0;
    if (pf > 1.0) pf = 1.0;
    real rate = p[6] * M_PI * (au + av) * (au + av) * dv;
    *kc = rate * (1.0 - pf);
    *kf = rate * pf;
}

static real kcoag(const octx *c, double u, double v)
{
    const real *p = c->coag_p;
    switch (c->p.coag_kind) {
    case ORC_COAG_CONST: return p[0];
    case ORC_COAG_ADD: return p[0] * (u + v);
    case ORC_COAG_MULT: return p[0] * u * v;
    case ORC_COAG_MAXWELL: return cross_section(u, v) * p[0] * c->beta_coag;
    case ORC_COAG_BALLISTIC: { real kc, kf; ballistic(p, u, v, &kc, &kf); return kc; }
    default: return 0.0;
    }
}

static real kfrag(const octx *c, double u, double v)
{
    const real *p = c->frag_p;
    switch (c->p.frag_kind) {
    case ORC_FRAG_MULT: return p[0] * u * v;
    case ORC_FRAG_MAXWELL: return cross_section(u, v) * p[0] * c->beta_frag;
    case ORC_FRAG_BALLISTIC: { real kc, kf; ballistic(p, u, v, &kc, &kf); return kf; }
    default: return 0.0;
    }
}

/* fragment mass fraction m_frag / (y+z), eq. (mfrag) */
ORC_API double orc_mfrag_ratio(double q)
{
    if (q <= 10.0) return 1.0;
    if (q <= 12.0) return (6.5 + 4.5 * cos((q - 10.0) / (12.0 - 10.0) * M_PI)) / (1.0 + q);
    if (q <= 15.0) return 2.0 / (1.0 + q);
    if (q <= 50.0) return (1.45 + 0.55 * cos((q - 15.0) / (50.0 - 15.0) * M_PI)) / (1.0 + q);
    return 0.9 / (1.0 + q);
}

typedef struct { double mfrag, mleft, mcut; real alpha; } frag_out;

static frag_out frag_outcome(const octx *c, double u, double v)
{
    frag_out o;
    double big = u > v ? u : v, small = u > v ? v : u;
    double tot = u + v;
    o.alpha = c->break_p[0];
    o.mfrag = c->p.mfrag_mode == 1 ? tot : tot * orc_mfrag_ratio(big / small);
    o.mleft = tot - o.mfrag;
    if (o.mleft < 0.0) o.mleft = 0.0;
    o.mcut = c->p.cutoff_mode == 1 ? big : o.mfrag;
    return o;
}

/* fraction of power-law fragment mass in [x_min, x] (eq. break with the
   normalisation A of Sec. 4.5); R10 for a cutoff at or below x_min */
static real pl_fraction(double x, double xmin, double mcut, real alpha)
{
    if (!(mcut > xmin)) return x > xmin ? 1.0 : 0.0;
    real a2 = 2.0 + alpha;
    real f = (pow(x, a2) - pow(xmin, a2)) / (pow(mcut, a2) - pow(xmin, a2));
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    return f;
}

/* mass of collision products with w > x:  int_x^{u+v} w b(w,u,v) dw  (eq. inte1) */
static real mass_above(const octx *c, double x, double u, double v)
{
    switch (c->p.break_kind) {
    case ORC_BREAK_UNIFORM_BINARY: {
        /* b = btilde(w,u;v) + btilde(w,v;u), btilde = 2/y on (0, y] (Sec. 4.4) */
        double m = 0.0;
        if (u > x) m += (u * u - x * x) / u;
        if (v > x) m += (v * v - x * x) / v;
        return m;
    }
    case ORC_BREAK_POWERLAW_REMNANT: {
        frag_out o = frag_outcome(c, u, v);
        real m = o.mfrag * (1.0 - pl_fraction(x, c->p.x_min, o.mcut, o.alpha));
        if (o.mleft > x) m += o.mleft;
        return m;
    }
    case ORC_BREAK_COAG_DELTA:
        return (u + v > x) ? u + v : 0.0;
    default: return 0.0;
    }
}

/* mass of collision products with x_min <= w <= x:  int_{x_min}^x w b dw  (eq. inte2) */
static real mass_below(const octx *c, double x, double u, double v)
{
    double xmin = c->p.x_min;
    switch (c->p.break_kind) {
    case ORC_BREAK_UNIFORM_BINARY: {
        double mu = x < u ? x : u, mv = x < v ? x : v;
        double m = 0.0;
        if (mu > xmin) m += (mu * mu - xmin * xmin) / u;
        if (mv > xmin) m += (mv * mv - xmin * xmin) / v;
        return m;
    }
    case ORC_BREAK_POWERLAW_REMNANT: {
        frag_out o = frag_outcome(c, u, v);
        real m = o.mfrag * pl_fraction(x, xmin, o.mcut, o.alpha);
        if (o.mleft >= xmin && o.mleft <= x) m += o.mleft;
        return m;
    }
    case ORC_BREAK_COAG_DELTA:
        return (u + v <= x) ? u + v : 0.0;
    default: return 0.0;
    }
}

static int has_remnant_delta(const octx *c)
{
    return c->p.frag_kind != ORC_FRAG_NONE && c->p.break_kind == ORC_BREAK_POWERLAW_REMNANT;
}

/* ------------------------------------------------------------------ */
/* DG representation helpers                                           */
/* ------------------------------------------------------------------ */
static int bin_of(const octx *c, double y)
{
    /* j with x_{j-1/2} <= y < x_{j+1/2}; clamps to [0, N-1] */
    int lo = 0, hi = c->N - 1;
    if (y <= c->e[0]) return 0;
    if (y >= c->e[c->N]) return c->N - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (c->e[mid] <= y) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* g_l(u) = sum_i g_l^i phi_i(xi_l(u)) (eq. 2.3); *gabs = sum_i |g_l^i phi_i| */
static real gval(const octx *c, const real *g, int l, double u, real *gabs)
{
    double P[ORC_KMAX + 1];
    double h = c->e[l + 1] - c->e[l];
    double xc = 0.5 * (c->e[l] + c->e[l + 1]);
    double xi = 2.0 / h * (u - xc);
    legendre(c->k, xi, P, NULL);
    const real *gl = g + (size_t)l * (c->k + 1);
    real s = 0.0, a = 0.0;
    for (int i = 0; i <= c->k; ++i) { s += gl[i] * P[i]; a += fabs(gl[i] * P[i]); }
    if (gabs) *gabs = a;
    return s;
}

static double vmax_of(const octx *c, double u)
{
    /* upper v limit x_max + Delta x (eqs. Fcoagtrun, Ffragtrun) */
    return c->p.flux_mode == 0 ? c->p.x_max - u + c->p.x_min : c->p.x_max;
}

/* ------------------------------------------------------------------ */
/* pointwise truncated flux F(x) (eqs. Fcoagtrun, Ffragtrun) evaluated by
   the nested Gauss quadrature of Sec. 3.3: the outer u-integral bin by
   bin (a partial last piece when x lies inside a bin, R6), and for every
   outer node the inner v-integral split at the bin edges, with the end
   bins A and B reduced to the sub-intervals [a_m, b_m] and Q remapped
   nodes each.                                                         */
/* ------------------------------------------------------------------ */
static void flux_point(const octx *c, const real *go, const real *g, double x, int want_coag,
                       int want_frag, real *F, real *Fabs)
{
    const int Q = c->Q;
    const double xmin = c->p.x_min;
    int do_coag = want_coag && c->p.coag_kind != ORC_COAG_NONE;
    int do_frag = want_frag && c->p.frag_kind != ORC_FRAG_NONE;
    real Fs = 0.0, Fa = 0.0;

    /* positive flux: u in [x_min, x], v in [x - u + x_min, v_max(u)] */
    if (do_coag || do_frag) {
        for (int l = 0; l < c->N && c->e[l] < x; ++l) {
            double a = c->e[l], b = c->e[l + 1] < x ? c->e[l + 1] : x;
            if (!(b > a)) continue;
            for (int al = 0; al < Q; ++al) {
                double u = 0.5 * (a + b) + 0.5 * (b - a) * c->s[al];
                double Wu = 0.5 * (b - a) * c->w[al];
                real gua, gu = gval(c, go, l, u, &gua);
                double lo = x - u + xmin, hi = vmax_of(c, u);
                if (!(hi > lo)) continue;
                for (int m = bin_of(c, lo); m < c->N && c->e[m] < hi; ++m) {
                    double va = lo > c->e[m] ? lo : c->e[m];
                    double vb = hi < c->e[m + 1] ? hi : c->e[m + 1];
                    if (!(vb > va)) continue;
                    for (int be = 0; be < Q; ++be) {
                        double v = 0.5 * (va + vb) + 0.5 * (vb - va) * c->s[be];
                        double Wv = 0.5 * (vb - va) * c->w[be];
                        real gva, gv = gval(c, g, m, v, &gva);
                        real t = 0.0;
                        if (do_coag) t += kcoag(c, u, v) / v;
                        if (do_frag) t += kfrag(c, u, v) * mass_above(c, x, u, v) / (v * (u + v));
                        Fs += Wu * Wv * t * gu * gv;
                        Fa += fabs(Wu * Wv * t) * gua * gva;
                    }
                }
            }
        }
    }
    /* negative flux: u in [x, x_max], v in [x_min, v_max(u)] (eq. Ffragtrun) */
    if (do_frag) {
        for (int l = bin_of(c, x); l < c->N; ++l) {
            double a = c->e[l] > x ? c->e[l] : x, b = c->e[l + 1];
            if (!(b > a)) continue;
            for (int al = 0; al < Q; ++al) {
                double u = 0.5 * (a + b) + 0.5 * (b - a) * c->s[al];
                double Wu = 0.5 * (b - a) * c->w[al];
                real gua, gu = gval(c, go, l, u, &gua);
                double lo = xmin, hi = vmax_of(c, u);
                if (!(hi > lo)) continue;
                for (int m = 0; m < c->N && c->e[m] < hi; ++m) {
                    double va = lo > c->e[m] ? lo : c->e[m];
                    double vb = hi < c->e[m + 1] ? hi : c->e[m + 1];
                    if (!(vb > va)) continue;
                    for (int be = 0; be < Q; ++be) {
                        double v = 0.5 * (va + vb) + 0.5 * (vb - va) * c->s[be];
                        double Wv = 0.5 * (vb - va) * c->w[be];
                        real gva, gv = gval(c, g, m, v, &gva);
                        real t = kfrag(c, u, v) * mass_below(c, x, u, v) / (v * (u + v));
                        Fs -= Wu * Wv * t * gu * gv;
                        Fa += fabs(Wu * Wv * t) * gua * gva;
                    }
                }
            }
        }
    }
    *F = Fs;
    if (Fabs) *Fabs = Fa;
}

/* Gauss integral of f(x) * d/dx phi_i(xi_j(x)), i = 1..k, over [a, b] inside
   bin j, for f = c0 + c1 * x^{2+alpha} (pw = 1) or f = c0 (pw = 0).
   Adds into J[i] and |.| into Jabs[i]. */
static void sub_integral(const octx *c, int j, double a, double b, real c0, real c1,
                         real alpha, int pw, double sign, real *J, real *Jabs)
{
    if (!(b > a)) return;
    double P[ORC_KMAX + 1], dP[ORC_KMAX + 1];
    double h = c->e[j + 1] - c->e[j];
    double xc = 0.5 * (c->e[j] + c->e[j + 1]);
    for (int t = 0; t < c->Q; ++t) {
        double x = 0.5 * (a + b) + 0.5 * (b - a) * c->s[t];
        double W = 0.5 * (b - a) * c->w[t];
        real f = pw ? c0 + c1 * pow(x, 2.0 + alpha) : c0;
        legendre(c->k, 2.0 / h * (x - xc), P, dP);
        for (int i = 1; i <= c->k; ++i) {
            real d = W * f * (2.0 / h) * dP[i];
            J[i] += sign * d;
            Jabs[i] += fabs(d);
        }
    }
}

static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

/* App. B for one collision pair (u, v): J[i] = int_{I_j} f_uv(x) d_x phi_i dx, i = 1..k, where
   f_uv(x) is the pair's share of the fragmentation flux at x per unit K_frag g(u) g(v) / (v (u+v)):
   the products heavier than x (eq. inte1) while u < x <= u + v - x_min, minus the products in
   [x_min, x] (eq. inte2) while x_min < x < u.  The x-integral is split into the five
   sub-interval terms of App. B (R7, R8); Ja[i] collects their absolute values. */
static void appB_pair(const octx *c, int j, double u, double v, real *J, real *Ja)
{
    const double xmin = c->p.x_min;
    const double ja = c->e[j], jb = c->e[j + 1];
    frag_out o = frag_outcome(c, u, v);
    double top = u + v - xmin;  /* x <= u + v - x_min (R7) */
    real a2 = 2.0 + o.alpha;
    if (o.mcut > xmin) {
        real cA = o.mfrag / (pow(o.mcut, a2) - pow(xmin, a2)); /* A/(2+alpha) */
        real mc2 = pow(o.mcut, a2), xm2 = pow(xmin, a2);
        /* term 1: +int_{I_j cap (u, min(top, m_cut))} A/(2+a) (m_cut^{2+a} - x^{2+a}) */
        sub_integral(c, j, dmax(ja, u), dmin(jb, dmin(top, o.mcut)),
                     cA * mc2, -cA, o.alpha, 1, +1.0, J, Ja);
        /* term 2: -int_{I_j cap (x_min, u)} A/(2+a) (x^{2+a} - x_min^{2+a}) */
        sub_integral(c, j, dmax(ja, xmin), dmin(jb, u),
                     -cA * xm2, cA, o.alpha, 1, -1.0, J, Ja);
        /* term 3: +int_{I_j cap (m_cut, u)} A/(2+a) (x^{2+a} - m_cut^{2+a}) */
        sub_integral(c, j, dmax(ja, o.mcut), dmin(jb, u),
                     -cA * mc2, cA, o.alpha, 1, +1.0, J, Ja);
    } else {
        /* R10: all fragment mass sits at x_min, i.e. below every x > x_min */
        sub_integral(c, j, dmax(ja, xmin), dmin(jb, u), o.mfrag, 0.0, 0.0, 0, -1.0, J, Ja);
    }
    if (o.mleft > 0.0) {
        /* term 4: +int_{I_j cap (u, min(top, m_left))} m_left */
        sub_integral(c, j, dmax(ja, u), dmin(jb, dmin(top, o.mleft)),
                     o.mleft, 0.0, 0.0, 0, +1.0, J, Ja);
        /* term 5: -int_{I_j cap (m_left, u)} m_left, remnant inside the domain (R10) */
        if (o.mleft >= xmin)
            sub_integral(c, j, dmax(ja, o.mleft), dmin(jb, u),
                         o.mleft, 0.0, 0.0, 0, -1.0, J, Ja);
    }
}

/* App. B: the fragmentation volume term int_{I_j} F_frag d_x phi_i dx for a
   breakage with a Dirac remnant, with the x-integral moved inside the
   (u, v) quadrature (appB_pair).  The outer (u, v) quadrature runs over full
   bins in u and over the bins of [x_min, v_max(u)] in v.  V[i], Vabs[i] for
   i = 1..k. */
static void vol_frag_appB(const octx *c, const real *go, const real *g, int j, real *V, real *Vabs)
{
    const int Q = c->Q, k = c->k;
    const double xmin = c->p.x_min;
    for (int i = 0; i <= k; ++i) { V[i] = 0.0; Vabs[i] = 0.0; }
    for (int l = 0; l < c->N; ++l) {
        double a = c->e[l], b = c->e[l + 1];
        for (int al = 0; al < Q; ++al) {
            double u = 0.5 * (a + b) + 0.5 * (b - a) * c->s[al];
            double Wu = 0.5 * (b - a) * c->w[al];
            real gua, gu = gval(c, go, l, u, &gua);
            double hi = vmax_of(c, u);
            for (int m = 0; m < c->N && c->e[m] < hi; ++m) {
                double va = c->e[m] > xmin ? c->e[m] : xmin;
                double vb = hi < c->e[m + 1] ? hi : c->e[m + 1];
                if (!(vb > va)) continue;
                for (int be = 0; be < Q; ++be) {
                    double v = 0.5 * (va + vb) + 0.5 * (vb - va) * c->s[be];
                    double Wv = 0.5 * (vb - va) * c->w[be];
                    real base = Wu * Wv * kfrag(c, u, v) / (v * (u + v));
                    if (REAL_IS_ZERO(base)) continue;
                    real J[ORC_KMAX + 1] = {0}, Ja[ORC_KMAX + 1] = {0};
                    appB_pair(c, j, u, v, J, Ja);
                    real gva, gv = gval(c, g, m, v, &gva);
                    for (int i = 1; i <= k; ++i) {
                        V[i] += base * gu * gv * J[i];
                        Vabs[i] += fabs(base) * gua * gva * Ja[i];
                    }
                }
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* the operator L[g] (eq. evo)                                         */
/* ------------------------------------------------------------------ */
/* Fif[j+1] = F(x_{j+1/2}) for j = -1..N-1 (Fif[0] = F(x_{-1/2}) = 0).
   go is the distribution of the outer collider of every flux integral (the particle of mass u
   whose share of the products crosses x), g that of its partner v: go = g gives L[g]; go = g_s,
   the partial mass density of a species s of grains that are mixtures of species (Sec. 5.3, with
   g = sum_s g_s), gives the rate of that species' partial mass (reading R24). */
static void rhs_one_outer(const octx *c, const real *go, const real *g, real *L, real *S)
{
    const int N = c->N, k = c->k, Q = c->Q;
    real *Fif = (real *)calloc((size_t)(N + 1) * 2, sizeof(real));
    real *Fab = Fif + (N + 1);
    /* interface fluxes; F(x_min) = 0 in both modes and F(x_max) = 0 in the
       conservative mode (Sec. 3.3), so those two are not evaluated */
    int jmax = c->p.flux_mode == 0 ? N - 2 : N - 1;
    for (int j = 0; j <= jmax; ++j)
        flux_point(c, go, g, c->e[j + 1], 1, 1, &Fif[j + 1], &Fab[j + 1]);

    double P[ORC_KMAX + 1], dP[ORC_KMAX + 1];
    int delta = has_remnant_delta(c);
    for (int j = 0; j < N; ++j) {
        double h = c->e[j + 1] - c->e[j];
        double xc = 0.5 * (c->e[j] + c->e[j + 1]);
        real V[ORC_KMAX + 1] = {0}, Va[ORC_KMAX + 1] = {0};
        if (k >= 1) {
            /* volume term int_{I_j} F d_x phi_i = sum_theta w_theta phi_i'(s_theta) F(x_j^theta) */
            for (int th = 0; th < Q; ++th) {
                double xt = xc + 0.5 * h * c->s[th];
                real Ft, Fta;
                flux_point(c, go, g, xt, 1, !delta, &Ft, &Fta);
                legendre(k, c->s[th], P, dP);
                for (int i = 1; i <= k; ++i) {
                    V[i] += c->w[th] * dP[i] * Ft;
                    Va[i] += fabs(c->w[th] * dP[i]) * Fta;
                }
            }
            if (delta) {
                real Vf[ORC_KMAX + 1], Vfa[ORC_KMAX + 1];
                vol_frag_appB(c, go, g, j, Vf, Vfa);
                for (int i = 1; i <= k; ++i) { V[i] += Vf[i]; Va[i] += Vfa[i]; }
            }
        }
        for (int i = 0; i <= k; ++i) {
            double di = 2.0 / (2.0 * i + 1.0);
            double sgn = (i % 2 == 0) ? 1.0 : -1.0;   /* phi_i(-1) = (-1)^i, phi_i(1) = 1 */
            real val = V[i] - Fif[j + 1] + sgn * Fif[j];
            real sc = Va[i] + Fab[j + 1] + Fab[j];
            L[(size_t)j * (k + 1) + i] = 2.0 / h / di * val;
            if (S) S[(size_t)j * (k + 1) + i] = 2.0 / h / di * sc;
        }
    }
    free(Fif);
}

/* the operator L[g] (eq. evo) */
static void rhs_one(const octx *c, const real *g, real *L, real *S) { rhs_one_outer(c, g, g, L, S); }

/* ------------------------------------------------------------------ */
/* scaling limiter (eqs. recon, gamma), minimum computed analytically   */
/* ------------------------------------------------------------------ */
static double poly_at(const double *gj, int k, double xi)
{
    double P[ORC_KMAX + 1];
    legendre(k, xi, P, NULL);
    double s = 0.0;
    for (int i = 0; i <= k; ++i) s += gj[i] * P[i];
    return s;
}

static double dpoly_at(const double *gj, int k, double xi)
{
    double P[ORC_KMAX + 1], dP[ORC_KMAX + 1];
    legendre(k, xi, P, dP);
    double s = 0.0;
    for (int i = 0; i <= k; ++i) s += gj[i] * dP[i];
    return s;
}

/* xi in [-1, 1] where sum_i g^i phi_i takes its minimum: the endpoints and the interior critical
   points are the candidates.  k <= 3 in closed form; k >= 4 by bracketing the derivative on a
   uniform grid of 256 intervals followed by bisection. */
static double bin_argmin(const double *gj, int k)
{
    double xm = -1.0, m = poly_at(gj, k, -1.0), t = poly_at(gj, k, 1.0);
    if (t < m) { m = t; xm = 1.0; }
    if (k <= 1) return xm;
    if (k == 2) {
        if (gj[2] != 0.0) {
            double xs = -gj[1] / (3.0 * gj[2]);
            if (xs > -1.0 && xs < 1.0) { t = poly_at(gj, k, xs); if (t < m) { m = t; xm = xs; } }
        }
        return xm;
    }
    if (k == 3) {
        /* p'(xi) = (15/2) g3 xi^2 + 3 g2 xi + (g1 - 3 g3 / 2) */
        double A = 7.5 * gj[3], B = 3.0 * gj[2], C = gj[1] - 1.5 * gj[3];
        double r[2]; int nr = 0;
        if (A == 0.0) {
            if (B != 0.0) r[nr++] = -C / B;
        } else {
            double disc = B * B - 4.0 * A * C;
            if (disc >= 0.0) {
                double sq = sqrt(disc);
                double qq = -0.5 * (B + (B >= 0.0 ? sq : -sq));
                if (qq != 0.0) { r[nr++] = qq / A; r[nr++] = C / qq; }
                else r[nr++] = 0.0;
            }
        }
        for (int i = 0; i < nr; ++i)
            if (r[i] > -1.0 && r[i] < 1.0) { t = poly_at(gj, k, r[i]); if (t < m) { m = t; xm = r[i]; } }
        return xm;
    }
    const int M = 256;
    double x0 = -1.0, d0 = dpoly_at(gj, k, x0);
    for (int s = 1; s <= M; ++s) {
        double x1 = -1.0 + 2.0 * s / M, d1 = dpoly_at(gj, k, x1);
        if ((d0 < 0.0 && d1 >= 0.0) || (d0 > 0.0 && d1 <= 0.0)) {
            double lo = x0, hi = x1, dlo = d0;
            for (int it = 0; it < 80; ++it) {
                double mid = 0.5 * (lo + hi), dm = dpoly_at(gj, k, mid);
                if ((dlo < 0.0) == (dm < 0.0)) { lo = mid; dlo = dm; } else hi = mid;
            }
            t = poly_at(gj, k, 0.5 * (lo + hi));
            if (t < m) { m = t; xm = 0.5 * (lo + hi); }
        }
        x0 = x1; d0 = d1;
    }
    return xm;
}

/* min over [-1, 1] of sum_i g^i phi_i (the value at bin_argmin) */
ORC_API double orc_bin_min(const double *gj, int k)
{
    return k == 0 ? gj[0] : poly_at(gj, k, bin_argmin(gj, k));
}

/* applies eq. (recon) with gamma from eq. (gamma) to every bin; returns flag bits.  The bin
   minimum is the polynomial at its argmin (found on the values), so in a derivative build the
   minimum's derivative is the derivative of the polynomial at that fixed point (the envelope
   theorem: the polynomial's xi-derivative vanishes at an interior minimum). */
static unsigned limit_one(const octx *c, real *g)
{
    unsigned flags = 0;
    const int k = c->k;
    if (k == 0) return 0;
    for (int j = 0; j < c->N; ++j) {
        real *gj = g + (size_t)j * (k + 1);
        real gbar = gj[0];
        real gamma;
        if (gbar < 0.0) { gamma = 0.0; flags |= 1u; }
        else {
            double gv[ORC_KMAX + 1], P[ORC_KMAX + 1];
            for (int i = 0; i <= k; ++i) gv[i] = RV(gj[i]);
            legendre(k, bin_argmin(gv, k), P, NULL);
            real mn = 0.0;
            for (int i = 0; i <= k; ++i) mn += gj[i] * P[i];
            real den = gbar - mn;
            gamma = den > 0.0 ? gbar / den : (real)1.0;
            if (gamma > 1.0) gamma = 1.0;
        }
        if (gamma < 1.0) {
            flags |= 2u;
            for (int i = 1; i <= k; ++i) gj[i] *= gamma;
        }
    }
    return flags;
}

static real mass_one(const octx *c, const real *g)
{
    /* M_1 = sum_j h_j g_j^0 (Sec. 4.1) */
    real m = 0.0;
    for (int j = 0; j < c->N; ++j) m += (c->e[j + 1] - c->e[j]) * g[(size_t)j * (c->k + 1)];
    return m;
}

static unsigned stage_flags(const octx *c, const real *g)
{
    unsigned f = 0;
    for (int j = 0; j < c->N; ++j) {
        if (g[(size_t)j * (c->k + 1)] < 0.0) f |= 1u;
        for (int i = 0; i <= c->k; ++i)
            if (!isfinite(RV(g[(size_t)j * (c->k + 1) + i]))) f |= 4u;
    }
    return f;
}

/* eq. (dt): the forward-Euler update of stage input gs with rhs L keeps the mean of
   bin j positive when dt |F_{j-1/2} - F_{j+1/2}| < h_j g_j^0, i.e. dt |L_j^0| < g_j^0.
   The bound protects positivity, so it is tested where the bin loses mass
   (L_j^0 < 0); a bin with influx or no flux cannot turn negative and is not flagged.
   For L_j^0 < 0 the bound fails exactly when g_j^0 + dt L_j^0 <= 0, evaluated with
   one rounding (fma), which keeps its sign exact.  Flag bit 3. */
static unsigned cfl_flags(const octx *c, const real *gs, const real *L, double dt)
{
    unsigned f = 0;
    for (int j = 0; j < c->N; ++j) {
        const double L0 = RV(L[(size_t)j * (c->k + 1)]);
        if (L0 < 0.0 && fma(dt, L0, RV(gs[(size_t)j * (c->k + 1)])) <= 0.0) f |= 8u;
    }
    return f;
}

/* A planted mistake for the tests of the mass-drift bit, 0 in every other use: when non-zero,
   every step_one adds planted_leak * M_1 to the mass of bin 0 (a non-conservative update). */
static double planted_leak = 0.0;

/* one SSP-RK3 step (eq. RK3) preceded by the reconstruction (Sec. 3.2) */
static unsigned step_one(const octx *c, real *g, double dt, real *work)
{
    const int P = c->P;
    real *L = work, *g1 = work + P, *g2 = work + 2 * P;
    unsigned f = 0;
    if (c->p.limiter) f |= limit_one(c, g);
    rhs_one(c, g, L, NULL);
    f |= cfl_flags(c, g, L, dt);
    for (int i = 0; i < P; ++i) g1[i] = g[i] + dt * L[i];
    f |= stage_flags(c, g1);
    rhs_one(c, g1, L, NULL);
    f |= cfl_flags(c, g1, L, dt);
    for (int i = 0; i < P; ++i) g2[i] = 0.75 * g[i] + 0.25 * (g1[i] + dt * L[i]);
    f |= stage_flags(c, g2);
    rhs_one(c, g2, L, NULL);
    f |= cfl_flags(c, g2, L, dt);
    for (int i = 0; i < P; ++i) g[i] = g[i] / 3.0 + 2.0 / 3.0 * (g2[i] + dt * L[i]);
    if (planted_leak != 0.0) g[0] += planted_leak * mass_one(c, g) / (c->e[1] - c->e[0]);
    f |= stage_flags(c, g);
    return f;
}

/* Relative tolerance of the mass-drift bit for a call of n steps.  With conservative fluxes
   (eq. g0) the flux differences telescope exactly, so M_1 moves only by the rounding of the
   stage updates.  A stage g' = a g^n + b (g^s + dt L) with non-negative means and eq. (dt)
   kept has sum_j h_j dt |L_j^0| <= 2 M_1, and its roundings (five in dt L_j^0, three in the
   b term, two in the a term) move M_1 by at most u (13 b + 2 a) M_1, u = 2^-53; the three
   stages of eq. (RK3) add up to 27.1 u M_1 per step, the two sums that form M_1 add 2 N u.
   The tolerance is 32 u per step, with a floor of 1e-10 for short calls. */
static double drift_tol(int n_steps)
{
    double t = 32.0 * ldexp(1.0, -53) * n_steps;
    return t > 1e-10 ? t : 1e-10;
}

/* ------------------------------------------------------------------ */
/* projection of an initial condition (eq. init) with a 16-point rule  */
/* ------------------------------------------------------------------ */
static double ic_value(int kind, const double *q, double x, const octx *c)
{
    switch (kind) {
    case ORC_IC_EXP:        /* g0 = A x exp(-x / x0) */
        return q[0] * x * exp(-x / q[1]);
    case ORC_IC_POWERLAW:   /* g0 = A x^beta on [lo, hi] */
        return (x >= q[2] && x <= q[3]) ? q[0] * pow(x, q[1]) : 0.0;
    case ORC_IC_FIRST_BIN:  /* g0 = A on the first bin */
        return x < c->e[1] ? q[0] : 0.0;
    default: return 0.0;
    }
}

static void project_one(const octx *c, int kind, const double *q, double *g)
{
    double s16[16], w16[16], P[ORC_KMAX + 1];
    orc_gauss(16, s16, w16);
    for (int j = 0; j < c->N; ++j) {
        double h = c->e[j + 1] - c->e[j], xc = 0.5 * (c->e[j] + c->e[j + 1]);
        for (int i = 0; i <= c->k; ++i) g[(size_t)j * (c->k + 1) + i] = 0.0;
        for (int a = 0; a < 16; ++a) {
            double x = xc + 0.5 * h * s16[a];
            double v = ic_value(kind, q, x, c);
            legendre(c->k, s16[a], P, NULL);
            for (int i = 0; i <= c->k; ++i)
                g[(size_t)j * (c->k + 1) + i] += w16[a] * v * P[i] * (2.0 * i + 1.0) / 2.0;
        }
    }
}

#ifndef ORC_TANGENT
/* ------------------------------------------------------------------ */
/* exported entry points (ctypes)                                      */
/* ------------------------------------------------------------------ */
static int set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_max_threads(void) { return set_threads(0); }

int orc_edges(const orc_params *p, double *edges)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    memcpy(edges, c.e, sizeof(double) * (c.N + 1));
    ctx_free(&c);
    return 0;
}

int orc_legendre(int k, double xi, double *P, double *dP)
{
    if (k < 0 || k > ORC_KMAX) return -1;
    legendre(k, xi, P, dP);
    return 0;
}

int orc_kernels(const orc_params *p, int n, const double *u, const double *v, double *kc, double *kf)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    for (int i = 0; i < n; ++i) { kc[i] = kcoag(&c, u[i], v[i]); kf[i] = kfrag(&c, u[i], v[i]); }
    ctx_free(&c);
    return 0;
}

int orc_mass_split(const orc_params *p, int n, const double *x, const double *u, const double *v,
                   double *above, double *below)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    for (int i = 0; i < n; ++i) {
        above[i] = mass_above(&c, x[i], u[i], v[i]);
        below[i] = mass_below(&c, x[i], u[i], v[i]);
    }
    ctx_free(&c);
    return 0;
}

/* pointwise flux F(x) for one cell; parts: bit0 coagulation, bit1 fragmentation */
int orc_flux_point(const orc_params *p, const double *g, int n, const double *x, int parts,
                   double *F, double *Fabs)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    for (int i = 0; i < n; ++i)
        flux_point(&c, g, g, x[i], parts & 1, (parts >> 1) & 1, &F[i], Fabs ? &Fabs[i] : NULL);
    ctx_free(&c);
    return 0;
}

/* App. B fragmentation volume term of bin j: V[i], i = 0..k (V[0] = 0) */
int orc_vol_frag(const orc_params *p, const double *g, int j, double *V, double *Vabs)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    if (j < 0 || j >= c.N) { ctx_free(&c); return -1; }
    vol_frag_appB(&c, g, g, j, V, Vabs);
    ctx_free(&c);
    return 0;
}

/* App. B sub-interval integrals of one collision pair (u, v) in bin j: J[i], i = 0..k (J[0] = 0) */
int orc_appB_pair(const orc_params *p, int j, double u, double v, double *J)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    if (j < 0 || j >= c.N) { ctx_free(&c); return -1; }
    double Jl[ORC_KMAX + 1] = {0}, Ja[ORC_KMAX + 1] = {0};
    appB_pair(&c, j, u, v, Jl, Ja);
    for (int i = 0; i <= c.k; ++i) J[i] = Jl[i];
    ctx_free(&c);
    return 0;
}

int orc_rhs_batch(const orc_params *p, int n_cells, const double *g, double *L, double *S, int n_threads)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    set_threads(n_threads);
    const int P = c.P;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int cell = 0; cell < n_cells; ++cell)
        rhs_one(&c, g + (size_t)cell * P, L + (size_t)cell * P, S ? S + (size_t)cell * P : NULL);
    ctx_free(&c);
    return 0;
}

int orc_limit_batch(const orc_params *p, int n_cells, double *g, unsigned char *flags)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    for (int cell = 0; cell < n_cells; ++cell) {
        unsigned f = limit_one(&c, g + (size_t)cell * c.P);
        if (flags) flags[cell] = (unsigned char)f;
    }
    ctx_free(&c);
    return 0;
}

int orc_step_batch(const orc_params *p, int n_cells, double *g, const double *dt, int n_steps,
                   double *mass, unsigned char *flags, int n_threads)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    set_threads(n_threads);
    const int P = c.P;
    int bad = 0;
    #pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 3 * (size_t)P);
        if (!work) {
            #pragma omp atomic write
            bad = 1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int cell = 0; cell < n_cells; ++cell) {
                double *gc = g + (size_t)cell * P;
                unsigned f = 0;
                const double m0 = mass_one(&c, gc);
                for (int s = 0; s < n_steps; ++s) f |= step_one(&c, gc, dt[cell], work);
                const double m1 = mass_one(&c, gc);
                /* eq. (g0): conservative fluxes keep M_1 to round-off while every stage keeps
                   eq. (dt) (each bin's update below the bin's mass); bit 4 marks a change above
                   drift_tol(n_steps) of M_1 over the call (or a NaN) in a cell with no
                   negative-mean, non-finite or eq. (dt) bit */
                if (c.p.flux_mode == 0 && !(f & (1u | 4u | 8u)) &&
                    !(fabs(m1 - m0) <= drift_tol(n_steps) * fabs(m0)))
                    f |= 16u;
                if (mass) mass[cell] = m1;
                if (flags) flags[cell] = (unsigned char)f;
            }
            free(work);
        }
    }
    ctx_free(&c);
    return bad ? -2 : 0;
}

/* Sub-step counts of the operator-split coupling (Sec. 5.2, the library's sub-cycling): for each
   cell the eq. (dt) bound B = min over bins losing mass (L_j^0 < 0) of g_j^0 / |L_j^0| of its state,
   and n = ceil(dt_hydro / (cfl B)), at least 1 (1 when no bin loses mass); counts[cell] = n. */
int orc_substep_counts(const orc_params *p, int n_cells, const double *g, const double *dt_hydro, double cfl,
                       int *counts)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    const int P = c.P, K1 = c.k + 1;
    double *L = (double *)malloc(sizeof(double) * (size_t)P);
    if (!L) { ctx_free(&c); return -2; }
    for (int cell = 0; cell < n_cells; ++cell) {
        const double *gc = g + (size_t)cell * P;
        rhs_one(&c, gc, L, NULL);
        double B = INFINITY;
        for (int j = 0; j < c.N; ++j)
            if (L[(size_t)j * K1] < 0.0) {
                const double r = gc[(size_t)j * K1] / -L[(size_t)j * K1];
                if (r < B) B = r;
            }
        const double want = dt_hydro[cell] / (cfl * B);
        int n = 1;
        if (want > 1.0) n = want < 1073741824.0 ? (int)ceil(want) : 1073741824;
        else if (!(want >= 0.0)) n = 1073741824;
        counts[cell] = n;
    }
    free(L);
    ctx_free(&c);
    return 0;
}

/* Species of grains that are mixtures (Sec. 5.3, reading R24): gs holds S partial mass densities in
   the layout [S][n_cells][P]; per cell g = sum_s g_s and L_s = L[g_s; g] (rhs_one_outer), written to
   Ls in the same layout, Ss the rounding scales (or NULL). */
int orc_rhs_species_batch(const orc_params *p, int n_cells, int n_species, const double *gs, double *Ls,
                          double *Ss)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    const int P = c.P;
    int bad = 0;
    #pragma omp parallel
    {
        double *g = (double *)malloc(sizeof(double) * (size_t)P);
        if (!g) {
            #pragma omp atomic write
            bad = 1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int cell = 0; cell < n_cells; ++cell) {
                for (int i = 0; i < P; ++i) g[i] = 0.0;
                for (int sp = 0; sp < n_species; ++sp)
                    for (int i = 0; i < P; ++i) g[i] += gs[((size_t)sp * n_cells + cell) * P + i];
                for (int sp = 0; sp < n_species; ++sp) {
                    const size_t o = ((size_t)sp * n_cells + cell) * P;
                    rhs_one_outer(&c, gs + o, g, Ls + o, Ss ? Ss + o : NULL);
                }
            }
            free(g);
        }
    }
    ctx_free(&c);
    return bad ? -2 : 0;
}

/* n_steps SSP-RK3 steps (eq. RK3) of the S species of every cell: each stage forms g = sum_s g_s of
   the stage input, L_s = L[g_s; g] and the stage combination per species; the scaling limiter
   (eqs. recon, gamma) acts on each species before each step.  mass[S][n_cells] receives M_1 of each
   species after the last step, flags[n_cells] the OR of the status bits of the cell's species
   (as orc_step_batch, the eq. dt bit from each species' forward-Euler mean update; the drift bit
   from the cell's total M_1). */
int orc_step_species_batch(const orc_params *p, int n_cells, int n_species, double *gs, const double *dt,
                           int n_steps, double *mass, unsigned char *flags)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    const int P = c.P, S = n_species;
    int bad = 0;
    #pragma omp parallel
    {
        /* g^n, g^(1), g^(2) of every species, L of every species, the total */
        double *w = (double *)malloc(sizeof(double) * (size_t)P * (4 * (size_t)S + 1));
        if (!w) {
            #pragma omp atomic write
            bad = 1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int cell = 0; cell < n_cells; ++cell) {
                double *gn = w, *g1 = w + (size_t)S * P, *g2 = w + 2 * (size_t)S * P, *L = w + 3 * (size_t)S * P;
                double *gt = w + 4 * (size_t)S * P;
                unsigned f = 0;
                double m0 = 0.0;
                for (int sp = 0; sp < S; ++sp) {
                    memcpy(gn + (size_t)sp * P, gs + ((size_t)sp * n_cells + cell) * P, sizeof(double) * P);
                    m0 += mass_one(&c, gn + (size_t)sp * P);
                }
                const double d = dt[cell];
                for (int st = 0; st < n_steps; ++st) {
                    if (c.p.limiter)
                        for (int sp = 0; sp < S; ++sp) f |= limit_one(&c, gn + (size_t)sp * P);
                    for (int stage = 0; stage < 3; ++stage) {
                        double *in = stage == 0 ? gn : (stage == 1 ? g1 : g2);
                        double *out = stage == 0 ? g1 : (stage == 1 ? g2 : gn);
                        for (int i = 0; i < P; ++i) gt[i] = 0.0;
                        for (int sp = 0; sp < S; ++sp)
                            for (int i = 0; i < P; ++i) gt[i] += in[(size_t)sp * P + i];
                        for (int sp = 0; sp < S; ++sp)
                            rhs_one_outer(&c, in + (size_t)sp * P, gt, L + (size_t)sp * P, NULL);
                        for (int sp = 0; sp < S; ++sp) {
                            const double *a = gn + (size_t)sp * P, *b = in + (size_t)sp * P, *l = L + (size_t)sp * P;
                            double *o = out + (size_t)sp * P;
                            f |= cfl_flags(&c, b, l, d);
                            /* the stage combinations written as in step_one */
                            if (stage == 0)
                                for (int i = 0; i < P; ++i) o[i] = b[i] + d * l[i];
                            else if (stage == 1)
                                for (int i = 0; i < P; ++i) o[i] = 0.75 * a[i] + 0.25 * (b[i] + d * l[i]);
                            else
                                for (int i = 0; i < P; ++i) o[i] = a[i] / 3.0 + 2.0 / 3.0 * (b[i] + d * l[i]);
                            f |= stage_flags(&c, o);
                        }
                    }
                }
                double m1 = 0.0;
                for (int sp = 0; sp < S; ++sp) {
                    const double ms = mass_one(&c, gn + (size_t)sp * P);
                    m1 += ms;
                    if (mass) mass[(size_t)sp * n_cells + cell] = ms;
                    memcpy(gs + ((size_t)sp * n_cells + cell) * P, gn + (size_t)sp * P, sizeof(double) * P);
                }
                if (c.p.flux_mode == 0 && !(f & (1u | 4u | 8u)) && !(fabs(m1 - m0) <= drift_tol(n_steps) * fabs(m0)))
                    f |= 16u;
                if (flags) flags[cell] = (unsigned char)f;
            }
            free(w);
        }
    }
    ctx_free(&c);
    return bad ? -2 : 0;
}

/* Plants a non-conservative update in every later step (tests of the mass-drift bit only);
   0 removes it. */
void orc_plant_mass_leak(double leak) { planted_leak = leak; }

double orc_drift_tol(int n_steps) { return drift_tol(n_steps); }

int orc_mass_batch(const orc_params *p, int n_cells, const double *g, double *mass)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    for (int cell = 0; cell < n_cells; ++cell) mass[cell] = mass_one(&c, g + (size_t)cell * c.P);
    ctx_free(&c);
    return 0;
}

/* ic_params: [n_cells][4] per-cell initial-condition parameters */
int orc_project_batch(const orc_params *p, int n_cells, int kind, const double *ic_params, double *g)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    for (int cell = 0; cell < n_cells; ++cell)
        project_one(&c, kind, ic_params + (size_t)cell * 4, g + (size_t)cell * c.P);
    ctx_free(&c);
    return 0;
}
#endif /* ORC_TANGENT */
