/*
 * Oracle of the two-dimensional (mass x, volume v) DG of Sec. 5.3 ("Toward a Multidimensional
 * Treatment"): the multidimensional Smoluchowski coagulation equation (the Sec. 5.3 equation that
 * extends eq. (fcoag)) discretised on cells I_{j,m} = I_j x I_m with the tensor-product Legendre
 * basis phi_p(xi_j(x)) phi_q(eta_m(v)), p, q <= k (the Sec. 5.3 expansion of g).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg may load this code.  It shares nothing with the CUDA library.
 *
 * What it computes, for the unknown g = x f (mass density), written out as the plain definition:
 * the Galerkin weak form of the equation tested with x phi_{j,m}^{p,q}(X),
 *
 *   h_j h_m / ((2p+1)(2q+1)) d g_{j,m}^{p,q} / dt
 *     = 1/2 int int K(X1, X2) f(X1) f(X2) (x1 + x2) phi_{j,m}^{p,q}(X1 + X2) dX1 dX2
 *       -   int int K(X1, X2) f(X1) f(X2) x1 phi_{j,m}^{p,q}(X1) dX1 dX2,
 *
 * with f = g / x, merging additive in both coordinates (X_{I+II} = X_I + X_II; readings R29, R31),
 * pairs whose merger leaves the domain lost (R30), and K a sum of separable power laws
 * K = sum_t c_t x1^ax_t x2^bx_t v1^av_t v2^bv_t (R32).  Every integral is a product Gauss rule
 * with Q nodes per coordinate (the rule of Sec. 3.3 per dimension), split exactly where the
 * merger crosses a cell edge: for a source pair (j1, j2) and a target bin j the outer x1-range I_j1
 * is cut at the points where the inner x2-range I_j2 n (I_j - x1) changes its end points, each
 * piece gets Q nodes in x1 and the inner range Q nodes in x2; the same in v.  The kernel and the
 * state are evaluated at every four-dimensional node (no factorisation of K is used here).
 *
 * State layout (per spatial cell): g_{j,m}^{p,q} at ((j (k+1) + p) Nv + m)(k+1) + q, i.e. a
 * row-major matrix G[(j,p)][(m,q)].  Grids are logarithmic: x_{j-1/2} = x_min (x_max/x_min)^(j/Nx).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MV_QMAX 24
#define MV_KMAX 4
#define MV_TMAX 8

typedef struct {
    int Nx, Nv, k, Q;
    double x_min, x_max, v_min, v_max;
    int n_terms;
    double coef[MV_TMAX], ax[MV_TMAX], bx[MV_TMAX], av[MV_TMAX], bv[MV_TMAX];
} orc_mv_desc;

/* Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_Q) */
static void mv_gauss(int Q, double *z, double *w)
{
    for (int i = 0; i < Q; ++i) {
        double t = cos(M_PI * (i + 0.75) / (Q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int n = 2; n <= Q; ++n) {
                const double p2 = ((2.0 * n - 1.0) * t * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            const double dp = Q * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int n = 2; n <= Q; ++n) {
            const double p2 = ((2.0 * n - 1.0) * t * p1 - (n - 1.0) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        const double dp = Q * (t * p1 - p0) / (t * t - 1.0);
        z[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* Legendre P_0..P_k at t */
static void mv_legendre(int k, double t, double *P)
{
    P[0] = 1.0;
    if (k >= 1) P[1] = t;
    for (int n = 2; n <= k; ++n) P[n] = ((2.0 * n - 1.0) * t * P[n - 1] - (n - 1.0) * P[n - 2]) / n;
}

static void mv_edges(int N, double lo, double hi, double *e)
{
    for (int i = 0; i <= N; ++i) e[i] = lo * pow(hi / lo, (double)i / N);
    e[0] = lo;
    e[N] = hi;
}

/* the bin of y (-1 outside [e0, eN)) */
static int mv_bin(const double *e, int N, double y)
{
    if (!(y >= e[0]) || !(y < e[N])) return -1;
    int lo = 0, hi = N;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (y >= e[mid]) lo = mid;
        else hi = mid;
    }
    return lo;
}

/* Nodes of the split rule over {y1 in B1, y2 in B2, y1 + y2 in T} for one coordinate: triples
   (y1, y2, weight).  The inner range is non-empty only for y1 in (tl - b2r, tr - b2l), and its end
   points switch at tl - b2l and tr - b2r, so at most three pieces carry nodes: at most 3 Q^2 of them.
   Returns the count. */
static int mv_pair_nodes(double b1l, double b1r, double b2l, double b2r, double tl, double tr, int Q,
                         const double *z, const double *w, double *y1o, double *y2o, double *wo)
{
    double cut[8];
    int nc = 0;
    cut[nc++] = b1l;
    const double cand[4] = {tl - b2l, tr - b2r, tl - b2r, tr - b2l};
    for (int i = 0; i < 4; ++i)
        if (cand[i] > b1l && cand[i] < b1r) cut[nc++] = cand[i];
    cut[nc++] = b1r;
    for (int i = 1; i < nc; ++i)   /* insertion sort */
        for (int j = i; j > 0 && cut[j] < cut[j - 1]; --j) {
            const double t = cut[j];
            cut[j] = cut[j - 1];
            cut[j - 1] = t;
        }
    int n = 0;
    for (int s = 0; s + 1 < nc; ++s) {
        const double a = cut[s], b = cut[s + 1];
        if (!(b > a)) continue;
        for (int i = 0; i < Q; ++i) {
            const double y1 = 0.5 * (a + b) + 0.5 * (b - a) * z[i], w1 = 0.5 * (b - a) * w[i];
            const double lo = fmax(b2l, tl - y1), hi = fmin(b2r, tr - y1);
            if (!(hi > lo)) continue;
            for (int l = 0; l < Q; ++l) {
                y1o[n] = y1;
                y2o[n] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * z[l];
                wo[n] = w1 * 0.5 * (hi - lo) * w[l];
                ++n;
            }
        }
    }
    return n;
}

static double mv_kernel(const orc_mv_desc *d, double x1, double x2, double v1, double v2)
{
    double K = 0.0;
    for (int t = 0; t < d->n_terms; ++t)
        K += d->coef[t] * pow(x1, d->ax[t]) * pow(x2, d->bx[t]) * pow(v1, d->av[t]) * pow(v2, d->bv[t]);
    return K;
}

/* g of one spatial cell at (x, v) inside cell (j, m) */
static double mv_eval(const orc_mv_desc *d, const double *G, const double *ex, const double *ev, int j, int m,
                      double x, double v)
{
    const int K1 = d->k + 1;
    double Px[MV_KMAX + 1], Pv[MV_KMAX + 1];
    mv_legendre(d->k, (2.0 * x - ex[j] - ex[j + 1]) / (ex[j + 1] - ex[j]), Px);
    mv_legendre(d->k, (2.0 * v - ev[m] - ev[m + 1]) / (ev[m + 1] - ev[m]), Pv);
    double s = 0.0;
    for (int p = 0; p < K1; ++p)
        for (int q = 0; q < K1; ++q) s += G[((j * K1 + p) * d->Nv + m) * K1 + q] * Px[p] * Pv[q];
    return s;
}

static int mv_check(const orc_mv_desc *d)
{
    if (!d || d->Nx < 1 || d->Nv < 1 || d->k < 0 || d->k > MV_KMAX || d->Q < 1 || d->Q > MV_QMAX) return -1;
    if (!(d->x_min > 0) || !(d->x_max > d->x_min) || !(d->v_min > 0) || !(d->v_max > d->v_min)) return -1;
    if (d->n_terms < 1 || d->n_terms > MV_TMAX) return -1;
    return 0;
}

/* L = dg/dt of the weak form above for n_cells independent cells */
int orc_mv_rhs(const orc_mv_desc *d, int n_cells, const double *g, double *L)
{
    if (mv_check(d) || n_cells < 0) return -1;
    const int Nx = d->Nx, Nv = d->Nv, K1 = d->k + 1, Q = d->Q;
    const int P = Nx * Nv * K1 * K1;
    double *ex = malloc(sizeof(double) * (Nx + 1)), *ev = malloc(sizeof(double) * (Nv + 1));
    double z[MV_QMAX], w[MV_QMAX];
    mv_edges(Nx, d->x_min, d->x_max, ex);
    mv_edges(Nv, d->v_min, d->v_max, ev);
    mv_gauss(Q, z, w);
    const int cap = 5 * Q * Q;   /* at most 3 Q^2 are used */
    double *xa = malloc(sizeof(double) * cap), *xb = malloc(sizeof(double) * cap), *xw = malloc(sizeof(double) * cap);
    double *va = malloc(sizeof(double) * cap), *vb = malloc(sizeof(double) * cap), *vw = malloc(sizeof(double) * cap);
    for (int c = 0; c < n_cells; ++c) {
        const double *G = g + (size_t)c * P;
        double *Lc = L + (size_t)c * P;
        double *acc = calloc((size_t)P, sizeof(double));
        /* gain: 1/2 sum over ordered source pairs, targets (j, m) where the merger can land */
        for (int j1 = 0; j1 < Nx; ++j1)
            for (int j2 = 0; j2 < Nx; ++j2)
                for (int j = 0; j < Nx; ++j) {
                    if (!(ex[j1] + ex[j2] < ex[j + 1]) || !(ex[j1 + 1] + ex[j2 + 1] > ex[j])) continue;
                    const int nx = mv_pair_nodes(ex[j1], ex[j1 + 1], ex[j2], ex[j2 + 1], ex[j], ex[j + 1], Q, z, w, xa, xb, xw);
                    for (int m1 = 0; m1 < Nv; ++m1)
                        for (int m2 = 0; m2 < Nv; ++m2)
                            for (int m = 0; m < Nv; ++m) {
                                if (!(ev[m1] + ev[m2] < ev[m + 1]) || !(ev[m1 + 1] + ev[m2 + 1] > ev[m])) continue;
                                const int nv = mv_pair_nodes(ev[m1], ev[m1 + 1], ev[m2], ev[m2 + 1], ev[m], ev[m + 1], Q, z, w,
                                                             va, vb, vw);
                                for (int a = 0; a < nx; ++a)
                                    for (int b = 0; b < nv; ++b) {
                                        const double x1 = xa[a], x2 = xb[a], v1 = va[b], v2 = vb[b];
                                        const double f1 = mv_eval(d, G, ex, ev, j1, m1, x1, v1) / x1;
                                        const double f2 = mv_eval(d, G, ex, ev, j2, m2, x2, v2) / x2;
                                        const double s = 0.5 * mv_kernel(d, x1, x2, v1, v2) * f1 * f2 * (x1 + x2) * xw[a] * vw[b];
                                        double Px[MV_KMAX + 1], Pv[MV_KMAX + 1];
                                        mv_legendre(d->k, (2.0 * (x1 + x2) - ex[j] - ex[j + 1]) / (ex[j + 1] - ex[j]), Px);
                                        mv_legendre(d->k, (2.0 * (v1 + v2) - ev[m] - ev[m + 1]) / (ev[m + 1] - ev[m]), Pv);
                                        for (int p = 0; p < K1; ++p)
                                            for (int q = 0; q < K1; ++q) acc[((j * K1 + p) * Nv + m) * K1 + q] += s * Px[p] * Pv[q];
                                    }
                            }
                }
        /* loss: every source pair, the first particle's cell is the target */
        for (int j = 0; j < Nx; ++j)
            for (int m = 0; m < Nv; ++m)
                for (int a = 0; a < Q; ++a)
                    for (int b = 0; b < Q; ++b) {
                        const double x1 = 0.5 * (ex[j] + ex[j + 1]) + 0.5 * (ex[j + 1] - ex[j]) * z[a];
                        const double v1 = 0.5 * (ev[m] + ev[m + 1]) + 0.5 * (ev[m + 1] - ev[m]) * z[b];
                        const double w1 = 0.25 * (ex[j + 1] - ex[j]) * (ev[m + 1] - ev[m]) * w[a] * w[b];
                        const double f1 = mv_eval(d, G, ex, ev, j, m, x1, v1) / x1;
                        double sum = 0.0;
                        for (int j2 = 0; j2 < Nx; ++j2)
                            for (int m2 = 0; m2 < Nv; ++m2)
                                for (int a2 = 0; a2 < Q; ++a2)
                                    for (int b2 = 0; b2 < Q; ++b2) {
                                        const double x2 = 0.5 * (ex[j2] + ex[j2 + 1]) + 0.5 * (ex[j2 + 1] - ex[j2]) * z[a2];
                                        const double v2 = 0.5 * (ev[m2] + ev[m2 + 1]) + 0.5 * (ev[m2 + 1] - ev[m2]) * z[b2];
                                        const double w2 = 0.25 * (ex[j2 + 1] - ex[j2]) * (ev[m2 + 1] - ev[m2]) * w[a2] * w[b2];
                                        sum += mv_kernel(d, x1, x2, v1, v2) * mv_eval(d, G, ex, ev, j2, m2, x2, v2) / x2 * w2;
                                    }
                        const double s = sum * f1 * x1 * w1;
                        double Px[MV_KMAX + 1], Pv[MV_KMAX + 1];
                        mv_legendre(d->k, z[a], Px);
                        mv_legendre(d->k, z[b], Pv);
                        for (int p = 0; p < K1; ++p)
                            for (int q = 0; q < K1; ++q) acc[((j * K1 + p) * Nv + m) * K1 + q] -= s * Px[p] * Pv[q];
                    }
        /* divide by the norm of the basis function, h_j h_m / ((2p+1)(2q+1)) */
        for (int j = 0; j < Nx; ++j)
            for (int p = 0; p < K1; ++p)
                for (int m = 0; m < Nv; ++m)
                    for (int q = 0; q < K1; ++q) {
                        const int i = ((j * K1 + p) * Nv + m) * K1 + q;
                        Lc[i] = acc[i] * (2.0 * p + 1.0) * (2.0 * q + 1.0) / ((ex[j + 1] - ex[j]) * (ev[m + 1] - ev[m]));
                    }
        free(acc);
    }
    free(xa); free(xb); free(xw); free(va); free(vb); free(vw); free(ex); free(ev);
    return 0;
}

/* n_steps SSP-RK3 steps (eq. (RK3)) of the weak form, dt per cell, no limiter (R33) */
int orc_mv_step(const orc_mv_desc *d, int n_cells, double *g, const double *dt, int n_steps)
{
    if (mv_check(d) || n_cells < 0 || n_steps < 0) return -1;
    const int K1 = d->k + 1, P = d->Nx * d->Nv * K1 * K1;
    double *g1 = malloc(sizeof(double) * P), *g2 = malloc(sizeof(double) * P), *Lb = malloc(sizeof(double) * P);
    for (int c = 0; c < n_cells; ++c) {
        double *gc = g + (size_t)c * P;
        const double h = dt[c];
        for (int s = 0; s < n_steps; ++s) {
            orc_mv_rhs(d, 1, gc, Lb);
            for (int i = 0; i < P; ++i) g1[i] = gc[i] + h * Lb[i];
            orc_mv_rhs(d, 1, g1, Lb);
            for (int i = 0; i < P; ++i) g2[i] = 0.75 * gc[i] + 0.25 * (g1[i] + h * Lb[i]);
            orc_mv_rhs(d, 1, g2, Lb);
            for (int i = 0; i < P; ++i) gc[i] = gc[i] / 3.0 + 2.0 / 3.0 * (g2[i] + h * Lb[i]);
        }
    }
    free(g1); free(g2); free(Lb);
    return 0;
}

/* total mass sum_{j,m} h_j h_m g_{j,m}^{0,0} of each cell */
int orc_mv_mass(const orc_mv_desc *d, int n_cells, const double *g, double *mass)
{
    if (mv_check(d) || n_cells < 0) return -1;
    const int Nx = d->Nx, Nv = d->Nv, K1 = d->k + 1, P = Nx * Nv * K1 * K1;
    double *ex = malloc(sizeof(double) * (Nx + 1)), *ev = malloc(sizeof(double) * (Nv + 1));
    mv_edges(Nx, d->x_min, d->x_max, ex);
    mv_edges(Nv, d->v_min, d->v_max, ev);
    for (int c = 0; c < n_cells; ++c) {
        double s = 0.0;
        for (int j = 0; j < Nx; ++j)
            for (int m = 0; m < Nv; ++m)
                s += (ex[j + 1] - ex[j]) * (ev[m + 1] - ev[m]) * g[(size_t)c * P + ((j * K1) * Nv + m) * K1];
        mass[c] = s;
    }
    free(ex); free(ev);
    return 0;
}

/* x-bin and v-bin edges of the grids (Nx + 1 and Nv + 1 values) */
int orc_mv_edges(const orc_mv_desc *d, double *ex, double *ev)
{
    if (mv_check(d)) return -1;
    mv_edges(d->Nx, d->x_min, d->x_max, ex);
    mv_edges(d->Nv, d->v_min, d->v_max, ev);
    return 0;
}

/* the bin containing y on an Nx-bin grid (for the brute-force pin), -1 outside */
int orc_mv_bin(const double *e, int N, double y) { return mv_bin(e, N, y); }
