// K-a1: FP64 precompute of the coefficient tensors T_r of every flux functional.
//
// For a group with N bins, degree k (K1 = k+1 coefficients per bin) and
// P = N K1 coefficients per cell, every flux functional r is a quadratic
// form of the coefficients, functional_r = sum_{p,q} T_r[p,q] g_p g_q, because
// the flux integrands of eqs. (Fcoagtrun) and (Ffragtrun) are products
// g(u) g(v) and g at any quadrature node is linear in the coefficients of the
// node's bin (eq. 2.3).  The functionals are
//   r <  n_if : the interface fluxes F(x_{j+1/2}), j = r (Sec. 3.3);
//   r >= n_if : the volume terms int_{I_j} F d_x phi_i dx of eq. (evo),
//               i = 1..k, r = n_if + j k + (i-1).
// The interface fluxes use the nested Gauss rule of Sec. 3.3 (partial end
// bins A..B, Q nodes per piece); the volume terms use Gauss on F(x_j^theta)
// for coagulation and for breakage without a Dirac remnant, and the
// reordered five-term form of App. B for the power-law + remnant breakage.
//
// One thread builds the K1 x K1 block T_r[(l,.),(m,.)] for one (r, l, m): it
// visits the outer nodes in bin l and the inner nodes in bin m.  Blocks are
// independent, so the build is deterministic and needs no atomics.
#include "grace_physics.cuh"

namespace grace {

namespace {

constexpr int kB = kKMax + 1;   // max coefficients per bin

// what a table entry stores: the value of a plain sum, the derivative part of a dual one
__device__ __forceinline__ double deriv_or_value(double x) { return x; }
__device__ __forceinline__ double deriv_or_value(const Dual &x) { return x.der; }

// Accumulates c * (contribution of outer bin l and inner bin m to F(x)).  PV: the parameter view
// (ParPlain for T, ParSeed for the exact dT/dtheta on dual numbers).
template <class PV>
__device__ void point_block(const DevGroup &G, const PV &pv, double x, int l, int m, double c, bool coag,
                            bool frag, par_t<PV> *acc)
{
    using S = par_t<PV>;
    const double *e = G.edges;
    const int k = G.k, K1 = G.K1, Q = G.Q;
    const bool do_coag = coag && G.coag_kind != GRACE_COAG_NONE;
    const bool do_frag = frag && G.frag_kind != GRACE_FRAG_NONE;
    const double hl = e[l + 1] - e[l], xl = 0.5 * (e[l] + e[l + 1]);
    const double hm = e[m + 1] - e[m], xm = 0.5 * (e[m] + e[m + 1]);
    double pu[kB], pw[kB];

    // positive flux: u in [x_min, x] (outer bin l, partial when x is inside it),
    // v in [x - u + x_min, v_max(u)] restricted to bin m (end bins A, B partial)
    if ((do_coag || do_frag) && e[l] < x) {
        const double a = e[l], b = fmin(e[l + 1], x);
        if (b > a) {
            for (int al = 0; al < Q; ++al) {
                const double u = 0.5 * (a + b) + 0.5 * (b - a) * G.gs[al];
                const double Wu = 0.5 * (b - a) * G.gw[al];
                const double lo = x - u + G.x_min, hi = dev_vmax(G, u);
                if (!(hi > lo)) continue;
                const double va = fmax(lo, e[m]), vb = fmin(hi, e[m + 1]);
                if (!(vb > va)) continue;
                dev_legendre(k, 2.0 / hl * (u - xl), pu, nullptr);
                for (int be = 0; be < Q; ++be) {
                    const double v = 0.5 * (va + vb) + 0.5 * (vb - va) * G.gs[be];
                    const double Wv = 0.5 * (vb - va) * G.gw[be];
                    S t = 0.0;
                    if (do_coag) t += kcoag_t(G, pv, u, v) / v;
                    if (do_frag) t += kfrag_t(G, pv, u, v) * mass_above_t(G, pv, x, u, v) / (v * (u + v));
                    const S wt = c * Wu * Wv * t;
                    dev_legendre(k, 2.0 / hm * (v - xm), pw, nullptr);
                    for (int ia = 0; ia < K1; ++ia)
                        for (int ib = 0; ib < K1; ++ib) acc[ia * K1 + ib] += wt * pu[ia] * pw[ib];
                }
            }
        }
    }
    // negative fragmentation flux: u in [x, x_max], v in [x_min, v_max(u)]
    if (do_frag && e[l + 1] > x) {
        const double a = fmax(e[l], x), b = e[l + 1];
        if (b > a) {
            for (int al = 0; al < Q; ++al) {
                const double u = 0.5 * (a + b) + 0.5 * (b - a) * G.gs[al];
                const double Wu = 0.5 * (b - a) * G.gw[al];
                const double hi = dev_vmax(G, u);
                const double va = fmax(G.x_min, e[m]), vb = fmin(hi, e[m + 1]);
                if (!(vb > va)) continue;
                dev_legendre(k, 2.0 / hl * (u - xl), pu, nullptr);
                for (int be = 0; be < Q; ++be) {
                    const double v = 0.5 * (va + vb) + 0.5 * (vb - va) * G.gs[be];
                    const double Wv = 0.5 * (vb - va) * G.gw[be];
                    const S t = kfrag_t(G, pv, u, v) * mass_below_t(G, pv, x, u, v) / (v * (u + v));
                    const S wt = c * Wu * Wv * t;
                    dev_legendre(k, 2.0 / hm * (v - xm), pw, nullptr);
                    for (int ia = 0; ia < K1; ++ia)
                        for (int ib = 0; ib < K1; ++ib) acc[ia * K1 + ib] -= wt * pu[ia] * pw[ib];
                }
            }
        }
    }
}

// Gauss rule on [a, b] (inside bin j) of (c0 + c1 x^{2+alpha}) d_x phi_i(xi_j(x))
template <class S>
__device__ S sub_interval(const DevGroup &G, int j, int i, double a, double b, S c0, S c1, S alpha, bool pw)
{
    if (!(b > a)) return S(0.0);
    const double *e = G.edges;
    const double h = e[j + 1] - e[j], xc = 0.5 * (e[j] + e[j + 1]);
    double P[kB], dP[kB];
    S s = 0.0;
    for (int t = 0; t < G.Q; ++t) {
        const double x = 0.5 * (a + b) + 0.5 * (b - a) * G.gs[t];
        const double W = 0.5 * (b - a) * G.gw[t];
        const S f = pw ? c0 + c1 * pow(x, 2.0 + alpha) : c0;
        dev_legendre(G.k, 2.0 / h * (x - xc), P, dP);
        s += W * f * (2.0 / h) * dP[i];
    }
    return s;
}

// App. B: int_{I_j} [above(x) 1{u < x < u+v-x_min} - below(x) 1{x_min < x < u}] d_x phi_i dx
// for one collision (u, v), as the paper's five sub-interval terms.
template <class PV>
__device__ par_t<PV> appB_J(const DevGroup &G, const PV &pv, int j, int i, double u, double v)
{
    using S = par_t<PV>;
    const double ja = G.edges[j], jb = G.edges[j + 1], xmin = G.x_min;
    const auto o = outcome_t(G, pv, u, v);
    const double top = u + v - xmin;
    const S zero = 0.0;
    S J = 0.0;
    if (o.mcut > xmin) {
        const S a2 = 2.0 + o.alpha;
        const S mc2 = pow(o.mcut, a2), xm2 = pow(xmin, a2);
        const S cA = o.mfrag / (mc2 - xm2);   // A / (2 + alpha)
        J += sub_interval<S>(G, j, i, fmax(ja, u), fmin(jb, fmin(top, o.mcut)), cA * mc2, -cA, o.alpha, true);
        J -= sub_interval<S>(G, j, i, fmax(ja, xmin), fmin(jb, u), -cA * xm2, cA, o.alpha, true);
        J += sub_interval<S>(G, j, i, fmax(ja, o.mcut), fmin(jb, u), -cA * mc2, cA, o.alpha, true);
    } else {
        J -= sub_interval<S>(G, j, i, fmax(ja, xmin), fmin(jb, u), S(o.mfrag), zero, zero, false);
    }
    if (o.mleft > 0.0) {
        J += sub_interval<S>(G, j, i, fmax(ja, u), fmin(jb, fmin(top, o.mleft)), S(o.mleft), zero, zero, false);
        if (o.mleft >= xmin)
            J -= sub_interval<S>(G, j, i, fmax(ja, o.mleft), fmin(jb, u), S(o.mleft), zero, zero, false);
    }
    return J;
}

__device__ __forceinline__ bool is_zero(double x) { return x == 0.0; }
__device__ __forceinline__ bool is_zero(const Dual &x) { return x.val == 0.0 && x.der == 0.0; }

template <class PV>
__device__ void appB_block(const DevGroup &G, const PV &pv, int j, int i, int l, int m, par_t<PV> *acc)
{
    using S = par_t<PV>;
    const double *e = G.edges;
    const int k = G.k, K1 = G.K1, Q = G.Q;
    const double hl = e[l + 1] - e[l], xl = 0.5 * (e[l] + e[l + 1]);
    const double hm = e[m + 1] - e[m], xm = 0.5 * (e[m] + e[m + 1]);
    double pu[kB], pw[kB];
    for (int al = 0; al < Q; ++al) {
        const double u = xl + 0.5 * hl * G.gs[al];
        const double Wu = 0.5 * hl * G.gw[al];
        const double hi = dev_vmax(G, u);
        const double va = fmax(G.x_min, e[m]), vb = fmin(hi, e[m + 1]);
        if (!(vb > va)) continue;
        dev_legendre(k, 2.0 / hl * (u - xl), pu, nullptr);
        for (int be = 0; be < Q; ++be) {
            const double v = 0.5 * (va + vb) + 0.5 * (vb - va) * G.gs[be];
            const double Wv = 0.5 * (vb - va) * G.gw[be];
            const S base = Wu * Wv * kfrag_t(G, pv, u, v) / (v * (u + v));
            if (is_zero(base)) continue;
            const S wt = base * appB_J(G, pv, j, i, u, v);
            dev_legendre(k, 2.0 / hm * (v - xm), pw, nullptr);
            for (int ia = 0; ia < K1; ++ia)
                for (int ib = 0; ib < K1; ++ib) acc[ia * K1 + ib] += wt * pu[ia] * pw[ib];
        }
    }
}

// one thread per (functional r, outer bin l, inner bin m): the K1 x K1 block of T_r, or with a
// seeded parameter view the block of dT_r/dtheta (the derivative parts of the same sums)
template <class PV>
__device__ void build_block(const DevGroup &G, const PV &pv, double *__restrict__ out)
{
    using S = par_t<PV>;
    const int r = blockIdx.y;
    const int lm = blockIdx.x * blockDim.x + threadIdx.x;
    if (lm >= G.N * G.N || r >= G.R) return;
    const int l = lm / G.N, m = lm % G.N;
    const int K1 = G.K1, P = G.P;
    S acc[kB * kB];
    for (int t = 0; t < kB * kB; ++t) acc[t] = 0.0;

    if (r < G.n_if) {
        point_block(G, pv, G.edges[r + 1], l, m, 1.0, true, true, acc);
    } else {
        const int q = r - G.n_if, j = q / G.k, i = q % G.k + 1;
        const double h = G.edges[j + 1] - G.edges[j], xc = 0.5 * (G.edges[j] + G.edges[j + 1]);
        double P_[kB], dP[kB];
        for (int th = 0; th < G.Q; ++th) {
            dev_legendre(G.k, G.gs[th], P_, dP);
            const double c = G.gw[th] * dP[i];
            point_block(G, pv, xc + 0.5 * h * G.gs[th], l, m, c, true, !G.has_delta, acc);
        }
        if (G.has_delta) appB_block(G, pv, j, i, l, m, acc);
    }
    for (int a = 0; a < K1; ++a)
        for (int b = 0; b < K1; ++b)
            out[((size_t)r * P + l * K1 + a) * P + m * K1 + b] = deriv_or_value(acc[a * K1 + b]);
}

__global__ void __launch_bounds__(128) build_T_kernel(DevGroup G, double *__restrict__ T)
{
    build_block(G, ParPlain{G}, T);
}

__global__ void __launch_bounds__(128) build_dT_kernel(DevGroup G, int id, double dbeta_coag, double dbeta_frag,
                                                       double *__restrict__ dT)
{
    build_block(G, ParSeed{G, id, dbeta_coag, dbeta_frag}, dT);
}

// first / one-past-last non-zero q of every row (r, p)
__global__ void row_extent_kernel(int R, int P, const double *__restrict__ T, int *qlo, int *qhi)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= R * P) return;
    const double *t = T + (size_t)row * P;
    int lo = P, hi = 0;
    for (int q = 0; q < P; ++q)
        if (t[q] != 0.0) {
            if (lo == P) lo = q;
            hi = q + 1;
        }
    qlo[row] = lo;
    qhi[row] = hi;
}

__global__ void p_range_kernel(int R, int P, const int *qlo, const int *qhi, int *prange)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int lo = P, hi = 0;
    for (int p = 0; p < P; ++p)
        if (qlo[r * P + p] < qhi[r * P + p]) {
            if (lo == P) lo = p;
            hi = p + 1;
        }
    prange[2 * r] = lo < hi ? lo : 0;
    prange[2 * r + 1] = hi;
}

}  // namespace

cudaError_t launch_build_T(const DevGroup &g, double *d_T, cudaStream_t st)
{
    dim3 grid((g.N * g.N + 127) / 128, g.R);
    build_T_kernel<<<grid, 128, 0, st>>>(g, d_T);
    return cudaGetLastError();
}

cudaError_t launch_build_dT(const DevGroup &g, int param_id, double dbeta_coag, double dbeta_frag, double *d_dT,
                            cudaStream_t st)
{
    dim3 grid((g.N * g.N + 127) / 128, g.R);
    build_dT_kernel<<<grid, 128, 0, st>>>(g, param_id, dbeta_coag, dbeta_frag, d_dT);
    return cudaGetLastError();
}

cudaError_t launch_row_extents(const DevGroup &g, const double *d_T, int *d_qlo, int *d_qhi, int *d_prange,
                               cudaStream_t st)
{
    const int rows = g.R * g.P;
    row_extent_kernel<<<(rows + 127) / 128, 128, 0, st>>>(g.R, g.P, d_T, d_qlo, d_qhi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    p_range_kernel<<<(g.R + 127) / 128, 128, 0, st>>>(g.R, g.P, d_qlo, d_qhi, d_prange);
    return cudaGetLastError();
}

}  // namespace grace
