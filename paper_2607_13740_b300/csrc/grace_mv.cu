// Two-dimensional (mass x, volume v) DG of Sec. 5.3 ("Toward a Multidimensional Treatment").
//
// Cells I_{j,m} = I_j x I_m of logarithmic grids in x and v, the tensor-product Legendre basis
// phi_p(xi_j(x)) phi_q(eta_m(v)) (p, q <= k), and the unknown g = x f.  The right-hand side is the
// Galerkin weak form of the multidimensional Smoluchowski equation of Sec. 5.3 with additive merging
// (x = x1 + x2, v = v1 + v2) and pairs whose merger leaves the grid lost:
//
//   h_j h_m / ((2p+1)(2q+1)) dg_{j,m}^{p,q}/dt = 1/2 int int K f1 f2 (x1 + x2) phi_{j,m}^{p,q}(X1 + X2)
//                                                 -   int int K f1 f2 x1 phi_{j,m}^{p,q}(X1).
//
// For a kernel that is a sum of separable power laws, K = sum_t c_t x1^ax x2^bx v1^av v2^bv, and
// since f1 f2 = sum G[a1][b1] G[a2][b2] (phi_a1(x1) / x1) phi_b1(v1) (phi_a2(x2) / x2) phi_b2(v2) with
// G[(j,p)][(m,q)] = g_{j,m}^{p,q}, the Gauss product rule of every four-dimensional integral (Q nodes
// per coordinate, split exactly where a merger crosses a cell edge) factorises into rules over
// (x1, x2) and over (v1, v2):
//
//   L[a][b] = sum_t sum_{a1 a2 b1 b2} Xg_t[a][a1][a2] Vg_t[b][b1][b2] G[a1][b1] G[a2][b2]   (gain)
//           - sum_t (sum_{p1 q1} XL1_t[j][p][p1] VL1_t[m][q][q1] G[(j,p1)][(m,q1)])
//                   (sum_{a2 b2} XL2_t[a2] VL2_t[b2] G[a2][b2])                          (loss)
//
// with a = (j, p), b = (m, q).  The 1-D factor forms are built once on the GPU in FP64 (setup); the
// contraction of every cell runs on the CUDA cores in FP64 (one CTA per cell, G staged in shared
// memory): per term and target row a, H = Xg_t[a] G (only source bins j1, j2 <= j can land in
// bin j), W = G^T H, then L[a][b] += <Vg_t[b], W> over source bins m1, m2 <= m.  O(N^{2d}) per cell
// as the paper notes; the cost is P_x^3 P_v + P_x^2 P_v^2 + P_x P_v^3 per term.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "grace_internal.h"

struct grace_mv {
    int device = 0;
    cudaStream_t stream = nullptr;
    grace_mv_desc d;
    int K1 = 1, Px = 0, Pv = 0, P = 0, T = 0;
    double *ex = nullptr, *ev = nullptr, *gz = nullptr, *gw = nullptr;
    double *Xg = nullptr, *Vg = nullptr, *XL1 = nullptr, *XL2 = nullptr, *VL1 = nullptr, *VL2 = nullptr;
    float *f32 = nullptr;    // FP32 copies of the six factor-form arrays, back to back (arithmetic 1)
    double *ws = nullptr;   // step workspace: g1, g2, L (3 x n_cap x P doubles)
    long long ws_cells = 0;
    size_t smem = 0;
};

namespace grace {
namespace {

constexpr int kMvThreads = 256;
constexpr int kMvF32Threads = 128;   // the FP32 kernel: more, smaller CTAs per SM
constexpr int kMvQMax = 24, kMvKMax = 4, kMvTMax = 8;

__device__ __forceinline__ double leg(int p, double t)
{
    double p0 = 1.0, p1 = t;
    if (p == 0) return p0;
    for (int n = 2; n <= p; ++n) {
        const double p2 = ((2.0 * n - 1.0) * t * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// logarithmic edges e[i] = lo (hi / lo)^(i / N), e[0] = lo and e[N] = hi exactly
__global__ void mv_edges_kernel(int N, double lo, double hi, double *e)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    e[i] = i == 0 ? lo : (i == N ? hi : lo * pow(hi / lo, (double)i / N));
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_Q), one thread per node
__global__ void mv_gauss_kernel(int Q, double *z, double *w)
{
    const int i = threadIdx.x;
    if (i >= Q) return;
    double t = cos(M_PI * (i + 0.75) / (Q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = t;
        for (int n = 2; n <= Q; ++n) {
            const double p2 = ((2.0 * n - 1.0) * t * p1 - (n - 1.0) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        dp = Q * (t * p1 - p0) / (t * t - 1.0);
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
    dp = Q * (t * p1 - p0) / (t * t - 1.0);
    z[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
}

// Split product rule over {y1 in [b1l, b1r], y2 in [b2l, b2r], y1 + y2 in [tl, tr]}: the y1-range is
// cut where the y2-range [max(b2l, tl - y1), min(b2r, tr - y1)] changes its end points; Q nodes on
// each piece of y1 and Q on the y2-range.  Calls f(y1, y2, weight) for every node.
template <class F>
__device__ void pair_rule(double b1l, double b1r, double b2l, double b2r, double tl, double tr, int Q,
                          const double *z, const double *w, F f)
{
    double cut[6];
    int nc = 0;
    cut[nc++] = b1l;
    const double cand[4] = {tl - b2l, tr - b2r, tl - b2r, tr - b2l};
    for (int i = 0; i < 4; ++i)
        if (cand[i] > b1l && cand[i] < b1r) cut[nc++] = cand[i];
    cut[nc++] = b1r;
    for (int i = 1; i < nc; ++i)
        for (int jj = i; jj > 0 && cut[jj] < cut[jj - 1]; --jj) {
            const double tmp = cut[jj];
            cut[jj] = cut[jj - 1];
            cut[jj - 1] = tmp;
        }
    for (int s = 0; s + 1 < nc; ++s) {
        const double a = cut[s], b = cut[s + 1];
        if (!(b > a)) continue;
        for (int i = 0; i < Q; ++i) {
            const double y1 = 0.5 * (a + b) + 0.5 * (b - a) * z[i], w1 = 0.5 * (b - a) * w[i];
            const double lo = fmax(b2l, tl - y1), hi = fmin(b2r, tr - y1);
            if (!(hi > lo)) continue;
            for (int l = 0; l < Q; ++l) f(y1, 0.5 * (lo + hi) + 0.5 * (hi - lo) * z[l], w1 * 0.5 * (hi - lo) * w[l]);
        }
    }
}

struct MvTerms {
    double c[kMvTMax], ax[kMvTMax], bx[kMvTMax], av[kMvTMax], bv[kMvTMax];
};

// gain factor forms: Xg_t[a][a1][a2] (x: mass-weighted, with 1/2 c_t (2p+1)/h_j) and Vg_t[b][b1][b2]
// (v: (2q+1)/h_m), one thread per entry; `dim` 0 builds X, 1 builds V
__global__ void mv_gain_forms_kernel(int dim, int N, int K1, int T, int Q, const double *e, const double *z,
                                     const double *w, MvTerms tm, double *out)
{
    const long long P = (long long)N * K1;
    const long long total = (long long)T * P * P * P;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int a2 = (int)(idx % P), a1 = (int)((idx / P) % P), a = (int)((idx / (P * P)) % P), t = (int)(idx / (P * P * P));
    const int j = a / K1, p = a % K1, j1 = a1 / K1, p1 = a1 % K1, j2 = a2 / K1, p2 = a2 % K1;
    double s = 0.0;
    if (e[j1] + e[j2] < e[j + 1] && e[j1 + 1] + e[j2 + 1] > e[j]) {
        const double ea = dim == 0 ? tm.ax[t] : tm.av[t], eb = dim == 0 ? tm.bx[t] : tm.bv[t];
        pair_rule(e[j1], e[j1 + 1], e[j2], e[j2 + 1], e[j], e[j + 1], Q, z, w, [&](double y1, double y2, double wt) {
            const double t1 = (2.0 * y1 - e[j1] - e[j1 + 1]) / (e[j1 + 1] - e[j1]);
            const double t2 = (2.0 * y2 - e[j2] - e[j2 + 1]) / (e[j2 + 1] - e[j2]);
            const double ts = (2.0 * (y1 + y2) - e[j] - e[j + 1]) / (e[j + 1] - e[j]);
            double v = wt * pow(y1, ea) * pow(y2, eb) * leg(p1, t1) * leg(p2, t2) * leg(p, ts);
            if (dim == 0) v *= (y1 + y2) / (y1 * y2);
            s += v;
        });
        s *= (2.0 * p + 1.0) / (e[j + 1] - e[j]);
        if (dim == 0) s *= 0.5 * tm.c[t];
    }
    out[idx] = s;
}

// loss factors: L1_t[j][p][p1] = (2p+1)/h_j int_{I_j} y^ea phi_p1 phi_p (x: times c_t; the x1 of the
// weak form cancels the 1/x1 of f1) and L2_t[(j2,p2)] = int_{I_j2} y^eb phi_p2 (/ y for x)
__global__ void mv_loss_forms_kernel(int dim, int N, int K1, int T, int Q, const double *e, const double *z,
                                     const double *w, MvTerms tm, double *L1, double *L2)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int n1 = T * N * K1 * K1, n2 = T * N * K1;
    if (idx < n1) {
        const int p1 = idx % K1, p = (idx / K1) % K1, j = (idx / (K1 * K1)) % N, t = idx / (K1 * K1 * N);
        const double ea = dim == 0 ? tm.ax[t] : tm.av[t];
        double s = 0.0;
        for (int i = 0; i < Q; ++i) {
            const double y = 0.5 * (e[j] + e[j + 1]) + 0.5 * (e[j + 1] - e[j]) * z[i];
            s += 0.5 * (e[j + 1] - e[j]) * w[i] * pow(y, ea) * leg(p1, z[i]) * leg(p, z[i]);
        }
        s *= (2.0 * p + 1.0) / (e[j + 1] - e[j]);
        if (dim == 0) s *= tm.c[t];
        L1[idx] = s;
    } else if (idx < n1 + n2) {
        const int i2 = idx - n1;
        const int p2 = i2 % K1, j2 = (i2 / K1) % N, t = i2 / (K1 * N);
        const double eb = dim == 0 ? tm.bx[t] : tm.bv[t];
        double s = 0.0;
        for (int i = 0; i < Q; ++i) {
            const double y = 0.5 * (e[j2] + e[j2 + 1]) + 0.5 * (e[j2 + 1] - e[j2]) * z[i];
            double v = 0.5 * (e[j2 + 1] - e[j2]) * w[i] * pow(y, eb) * leg(p2, z[i]);
            if (dim == 0) v /= y;
            s += v;
        }
        L2[i2] = s;
    }
}

template <class R>
struct MvArgs {
    int Nx, Nv, K1, Px, Pv, T;
    const R *Xg, *Vg, *XL1, *XL2, *VL1, *VL2;
};

template <class R>
__device__ __forceinline__ R block_sum(R v, R *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    R s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// L = dg/dt of one cell per CTA, in the arithmetic R (instantiated for double; the FP32 form is
// mv_rhs_f32_kernel below); the state is read and L written in FP64
template <class R>
__global__ void __launch_bounds__(kMvThreads) mv_rhs_kernel(MvArgs<R> A, int n_cells, const double *__restrict__ g,
                                                           double *__restrict__ Lout)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    R *sm = reinterpret_cast<R *>(sm_raw);
    const int Px = A.Px, Pv = A.Pv, K1 = A.K1, P = Px * Pv;
    R *G = sm, *Lc = G + P, *H = Lc + P, *Wm = H + P, *Xa = Wm + (size_t)Pv * Pv, *red = Xa + (size_t)Px * Px;
    const long long cell = blockIdx.x;
    if (cell >= n_cells) return;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int i = tid; i < P; i += nt) {
        G[i] = (R)g[cell * P + i];
        Lc[i] = 0;
    }
    __syncthreads();
    for (int t = 0; t < A.T; ++t) {
        // ---- loss: the bilinear scalar, then the cell-local operator
        const R *XL2 = A.XL2 + (size_t)t * Px, *VL2 = A.VL2 + (size_t)t * Pv;
        R part = 0;
        for (int i = tid; i < P; i += nt) part += XL2[i / Pv] * VL2[i % Pv] * G[i];
        const R S = block_sum(part, red);
        const R *XL1 = A.XL1 + (size_t)t * A.Nx * K1 * K1, *VL1 = A.VL1 + (size_t)t * A.Nv * K1 * K1;
        for (int i = tid; i < P; i += nt) {
            const int a = i / Pv, b = i % Pv, j = a / K1, p = a % K1, m = b / K1, q = b % K1;
            R s = 0;
            for (int p1 = 0; p1 < K1; ++p1) {
                const R xl = XL1[(j * K1 + p) * K1 + p1];
                if (xl == (R)0) continue;
                for (int q1 = 0; q1 < K1; ++q1) s += xl * VL1[(m * K1 + q) * K1 + q1] * G[(j * K1 + p1) * Pv + m * K1 + q1];
            }
            Lc[i] -= S * s;
        }
        __syncthreads();
        // ---- gain, one target row a at a time
        const R *Xt = A.Xg + (size_t)t * Px * Px * Px, *Vt = A.Vg + (size_t)t * Pv * Pv * Pv;
        for (int a = 0; a < Px; ++a) {
            const int amax = (a / K1 + 1) * K1;             // source bins j1, j2 <= j
            for (int i = tid; i < amax * amax; i += nt) Xa[i] = Xt[((size_t)a * Px + i / amax) * Px + i % amax];
            __syncthreads();
            // H[a1][b2] = sum_{a2} Xa[a1][a2] G[a2][b2]
            for (int i = tid; i < amax * Pv; i += nt) {
                const int a1 = i / Pv, b2 = i % Pv;
                R s = 0;
                for (int a2 = 0; a2 < amax; ++a2) s += Xa[a1 * amax + a2] * G[a2 * Pv + b2];
                H[i] = s;
            }
            __syncthreads();
            // W[b1][b2] = sum_{a1} G[a1][b1] H[a1][b2]
            for (int i = tid; i < Pv * Pv; i += nt) {
                const int b1 = i / Pv, b2 = i % Pv;
                R s = 0;
                for (int a1 = 0; a1 < amax; ++a1) s += G[a1 * Pv + b1] * H[a1 * Pv + b2];
                Wm[i] = s;
            }
            __syncthreads();
            // L[a][b] += sum_{b1, b2 <= (m+1) K1} Vg[b][b1][b2] W[b1][b2], one warp per b
            for (int b = warp; b < Pv; b += nw) {
                const int bmax = (b / K1 + 1) * K1;
                const R *Vb = Vt + (size_t)b * Pv * Pv;
                R s = 0;
                for (int i = lane; i < bmax * bmax; i += 32) {
                    const int b1 = i / bmax, b2 = i % bmax;
                    s += Vb[b1 * Pv + b2] * Wm[b1 * Pv + b2];
                }
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) Lc[a * Pv + b] += s;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < P; i += nt) Lout[cell * P + i] = (double)Lc[i];
}

// Shared-memory layout of the FP32 kernel, in floats, each array starting on a 16-byte boundary:
// G and L (P each), the K1 rows of one mass bin of X_t (K1 Px^2), their H (K1 Px Pv) and W
// (K1 Pv^2), the block-sum scratch
struct MvF32Smem {
    size_t G, L, X, H, W, red, total;
};

__host__ __device__ inline size_t mv_round4(size_t n) { return (n + 3) & ~(size_t)3; }

__host__ __device__ inline MvF32Smem mv_f32_layout(int Px, int Pv, int K1)
{
    MvF32Smem o;
    const size_t P = (size_t)Px * Pv;
    o.G = 0;
    o.L = mv_round4(P);
    o.X = o.L + mv_round4(P);
    o.H = o.X + mv_round4((size_t)K1 * Px * Px);
    o.W = o.H + mv_round4((size_t)K1 * Px * Pv);
    o.red = o.W + mv_round4((size_t)K1 * Pv * Pv);
    o.total = o.red + kMvF32Threads / 32;
    return o;
}

// The FP32 contraction, one cell per CTA.  The same sums as mv_rhs_kernel, with the K1 target rows
// a = j K1 + p of a mass bin j taken together (they share the source range a1, a2 < (j+1) K1):
// per bin, H_p = X_t[a] G over that range, W_p = G^T H_p, and L[a][b] += <V_t[b], W_p>, so each
// bin needs three barriers and each V_t element loaded serves K1 products.  With VEC (P_v a
// multiple of 4) a thread computes four adjacent columns of H or W from one float4 load.  The
// degree is a template parameter (K1 = k + 1 = A.K1), so the loops over the K1 rows carry no
// predicates and the index divisions by K1 are by a constant.
template <int K1, bool VEC>
__global__ void __launch_bounds__(kMvF32Threads) mv_rhs_f32_kernel(MvArgs<float> A, int n_cells, const double *__restrict__ g,
                                                               double *__restrict__ Lout)
{
    extern __shared__ __align__(16) float smf[];
    const int Px = A.Px, Pv = A.Pv, P = Px * Pv;
    const MvF32Smem o = mv_f32_layout(Px, Pv, K1);
    float *G = smf + o.G, *Lc = smf + o.L, *Xs = smf + o.X, *H = smf + o.H, *Wm = smf + o.W, *red = smf + o.red;
    const long long cell = blockIdx.x;
    if (cell >= n_cells) return;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const int Pv4 = Pv / 4;
    for (int i = tid; i < P; i += nt) {
        G[i] = (float)g[cell * P + i];
        Lc[i] = 0.f;
    }
    __syncthreads();
    for (int t = 0; t < A.T; ++t) {
        // ---- loss, as in the FP64 kernel
        const float *XL2 = A.XL2 + (size_t)t * Px, *VL2 = A.VL2 + (size_t)t * Pv;
        float part = 0.f;
        for (int i = tid; i < P; i += nt) part += XL2[i / Pv] * VL2[i % Pv] * G[i];
        const float S = block_sum(part, red);
        const float *XL1 = A.XL1 + (size_t)t * A.Nx * K1 * K1, *VL1 = A.VL1 + (size_t)t * A.Nv * K1 * K1;
        for (int i = tid; i < P; i += nt) {
            const int a = i / Pv, b = i % Pv, j = a / K1, p = a % K1, m = b / K1, q = b % K1;
            float s = 0.f;
            for (int p1 = 0; p1 < K1; ++p1) {
                const float xl = XL1[(j * K1 + p) * K1 + p1];
                if (xl == 0.f) continue;
                for (int q1 = 0; q1 < K1; ++q1) s += xl * VL1[(m * K1 + q) * K1 + q1] * G[(j * K1 + p1) * Pv + m * K1 + q1];
            }
            Lc[i] -= S * s;
        }
        __syncthreads();
        // ---- gain, one mass bin (K1 target rows) at a time
        const float *Xt = A.Xg + (size_t)t * Px * Px * Px, *Vt = A.Vg + (size_t)t * Pv * Pv * Pv;
        for (int j = 0; j < A.Nx; ++j) {
            const int amax = (j + 1) * K1, aa = amax * amax;
            // Xs[p][a1][a2] = X_t[j K1 + p][a1][a2], a1, a2 < amax
            for (int i = tid; i < K1 * aa; i += nt) {
                const int p = i / aa, r = i % aa;
                Xs[i] = Xt[((size_t)(j * K1 + p) * Px + r / amax) * Px + r % amax];
            }
            __syncthreads();
            // H[p][a1][b2] = sum_{a2 < amax} Xs[p][a1][a2] G[a2][b2]
            if (VEC) {
                // a thread: four columns of row a1 for all K1 rows p (one G load serves K1 x 4 FMAs)
                const float4 *G4 = reinterpret_cast<const float4 *>(G);
                float4 *H4 = reinterpret_cast<float4 *>(H);
                for (int i = tid; i < amax * Pv4; i += nt) {
                    const int a1 = i / Pv4, c = i % Pv4;
                    float4 s[K1];
#pragma unroll
                    for (int p = 0; p < K1; ++p) s[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int a2 = 0; a2 < amax; ++a2) {
                        const float4 v = G4[a2 * Pv4 + c];
#pragma unroll
                        for (int p = 0; p < K1; ++p) {
                            const float x = Xs[(p * amax + a1) * amax + a2];
                            s[p].x = fmaf(x, v.x, s[p].x);
                            s[p].y = fmaf(x, v.y, s[p].y);
                            s[p].z = fmaf(x, v.z, s[p].z);
                            s[p].w = fmaf(x, v.w, s[p].w);
                        }
                    }
#pragma unroll
                    for (int p = 0; p < K1; ++p) H4[(p * amax + a1) * Pv4 + c] = s[p];
                }
            } else {
                for (int i = tid; i < K1 * amax * Pv; i += nt) {
                    const int pa = i / Pv, b2 = i % Pv;
                    const float *xr = Xs + (size_t)pa * amax;
                    float s = 0.f;
                    for (int a2 = 0; a2 < amax; ++a2) s = fmaf(xr[a2], G[a2 * Pv + b2], s);
                    H[i] = s;
                }
            }
            __syncthreads();
            // W[p][b1][b2] = sum_{a1 < amax} G[a1][b1] H[p][a1][b2]
            if (VEC) {
                // a thread: four columns of row b1 for all K1 rows p (one G load serves K1 x 4 FMAs)
                const float4 *H4 = reinterpret_cast<const float4 *>(H);
                float4 *W4 = reinterpret_cast<float4 *>(Wm);
                for (int i = tid; i < Pv * Pv4; i += nt) {
                    const int b1 = i / Pv4, c = i % Pv4;
                    float4 s[K1];
#pragma unroll
                    for (int p = 0; p < K1; ++p) s[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int a1 = 0; a1 < amax; ++a1) {
                        const float x = G[a1 * Pv + b1];
#pragma unroll
                        for (int p = 0; p < K1; ++p) {
                            const float4 v = H4[(p * amax + a1) * Pv4 + c];
                            s[p].x = fmaf(x, v.x, s[p].x);
                            s[p].y = fmaf(x, v.y, s[p].y);
                            s[p].z = fmaf(x, v.z, s[p].z);
                            s[p].w = fmaf(x, v.w, s[p].w);
                        }
                    }
#pragma unroll
                    for (int p = 0; p < K1; ++p) W4[(p * Pv + b1) * Pv4 + c] = s[p];
                }
            } else {
                for (int i = tid; i < K1 * Pv * Pv; i += nt) {
                    const int p = i / (Pv * Pv), r = i % (Pv * Pv), b1 = r / Pv, b2 = r % Pv;
                    const float *hp = H + (size_t)p * amax * Pv + b2;
                    float s = 0.f;
                    for (int a1 = 0; a1 < amax; ++a1) s = fmaf(G[a1 * Pv + b1], hp[a1 * Pv], s);
                    Wm[i] = s;
                }
            }
            __syncthreads();
            // L[j K1 + p][b] += sum_{b1, b2 < bmax} V_t[b][b1][b2] W[p][b1][b2], one warp per b; the
            // lanes walk the (b1, column group) pairs of the range, the index advanced without a
            // division; with VEC a group is four columns, those at or beyond bmax masked
            for (int b = warp; b < Pv; b += nw) {
                const int bmax = (b / K1 + 1) * K1;
                const float *Vb = Vt + (size_t)b * Pv * Pv;
                float s[K1];
#pragma unroll
                for (int p = 0; p < K1; ++p) s[p] = 0.f;
                const int cw = VEC ? (bmax + 3) / 4 : bmax, db1 = 32 / cw, dc = 32 % cw;
                int b1 = lane / cw, c = lane % cw;
                while (b1 < bmax) {
                    if (VEC) {
                        float4 v = *reinterpret_cast<const float4 *>(Vb + b1 * Pv + 4 * c);
                        if (4 * c + 1 >= bmax) v.y = 0.f;
                        if (4 * c + 2 >= bmax) v.z = 0.f;
                        if (4 * c + 3 >= bmax) v.w = 0.f;
#pragma unroll
                        for (int p = 0; p < K1; ++p) {
                            const float4 w = *reinterpret_cast<const float4 *>(Wm + (size_t)p * Pv * Pv + b1 * Pv + 4 * c);
                            s[p] = fmaf(v.x, w.x, fmaf(v.y, w.y, fmaf(v.z, w.z, fmaf(v.w, w.w, s[p]))));
                        }
                    } else {
                        const int e = b1 * Pv + c;
                        const float v = Vb[e];
#pragma unroll
                        for (int p = 0; p < K1; ++p) s[p] = fmaf(v, Wm[(size_t)p * Pv * Pv + e], s[p]);
                    }
                    c += dc;
                    b1 += db1;
                    if (c >= cw) {
                        c -= cw;
                        ++b1;
                    }
                }
#pragma unroll
                for (int p = 0; p < K1; ++p) {
                    float r = s[p];
                    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
                    if (lane == 0) Lc[(j * K1 + p) * Pv + b] += r;
                }
            }
            // the next bin writes Xs, H and W only after two more barriers
        }
        __syncthreads();
    }
    for (int i = tid; i < P; i += nt) Lout[cell * P + i] = (double)Lc[i];
}

using MvF32Kernel = void (*)(MvArgs<float>, int, const double *, double *);

template <int K1>
MvF32Kernel mv_f32_pick(bool vec)
{
    return vec ? mv_rhs_f32_kernel<K1, true> : mv_rhs_f32_kernel<K1, false>;
}

// the FP32 kernel for degree k = K1 - 1 (0 .. 4) and the column form VEC
MvF32Kernel mv_f32_kernel_for(int K1, bool vec)
{
    switch (K1) {
    case 1: return mv_f32_pick<1>(vec);
    case 2: return mv_f32_pick<2>(vec);
    case 3: return mv_f32_pick<3>(vec);
    case 4: return mv_f32_pick<4>(vec);
    case 5: return mv_f32_pick<5>(vec);
    default: return nullptr;
    }
}

__global__ void mv_to_f32_kernel(long long n, const double *src, float *dst)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

// out = a gn + b (gs + dt_cell L), elementwise over n_cells x P
__global__ void mv_combine_kernel(long long n, int P, double a, double b, const double *gn, const double *gs,
                                  const double *dt, const double *L, double *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = dt[i / P];
    out[i] = (a == 0.0 ? 0.0 : a * gn[i]) + b * (gs[i] + h * L[i]);
}

size_t mv_smem(int Px, int Pv, size_t elem)
{
    return elem * ((size_t)4 * Px * Pv + (size_t)Pv * Pv + (size_t)Px * Px + kMvThreads / 32);
}

}  // namespace
}  // namespace grace

using namespace grace;

extern "C" {

grace_status grace_mv_setup(grace_mv **out, const grace_mv_desc *d, int device)
{
    if (!out || !d) {
        set_error("grace_mv_setup: null argument");
        return GRACE_ERR_ARG;
    }
    *out = nullptr;
    if (d->n_x < 1 || d->n_v < 1 || d->n_x > 256 || d->n_v > 256 || d->order_k < 0 || d->order_k > kMvKMax ||
        d->quad_q < 1 || d->quad_q > kMvQMax || d->n_terms < 1 || d->n_terms > kMvTMax || !(d->x_min > 0) ||
        !(d->x_max > d->x_min) || !(d->v_min > 0) || !(d->v_max > d->v_min) || !std::isfinite(d->x_max) ||
        !std::isfinite(d->v_max) || device < 0 || (d->arithmetic != 0 && d->arithmetic != 1)) {
        set_error("grace_mv_setup: invalid grid, order, rule, kernel terms, arithmetic or device");
        return GRACE_ERR_ARG;
    }
    for (int t = 0; t < d->n_terms; ++t)
        if (!std::isfinite(d->coef[t]) || !std::isfinite(d->ax[t]) || !std::isfinite(d->bx[t]) ||
            !std::isfinite(d->av[t]) || !std::isfinite(d->bv[t])) {
            set_error("grace_mv_setup: kernel terms must be finite");
            return GRACE_ERR_ARG;
        }
    const int K1 = d->order_k + 1, Px = d->n_x * K1, Pv = d->n_v * K1;
    const size_t smem = d->arithmetic ? sizeof(float) * mv_f32_layout(Px, Pv, K1).total : mv_smem(Px, Pv, sizeof(double));
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || device >= dev_count) {
        set_error("grace_mv_setup: no such CUDA device");
        return GRACE_ERR_ARG;
    }
    Guard guard(device);
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (smem > (size_t)smem_max) {
        set_error("grace_mv_setup: the grid's coefficient matrix does not fit the per-cell shared-memory stage");
        return GRACE_ERR_UNSUPPORTED;
    }
    grace_mv *m = new grace_mv();
    m->device = device;
    m->d = *d;
    m->K1 = K1;
    m->Px = Px;
    m->Pv = Pv;
    m->P = Px * Pv;
    m->T = d->n_terms;
    m->smem = smem;
    const int T = m->T, Q = d->quad_q;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](double **p, size_t n) {
        if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(double));
    };
    alloc(&m->ex, d->n_x + 1);
    alloc(&m->ev, d->n_v + 1);
    alloc(&m->gz, Q);
    alloc(&m->gw, Q);
    alloc(&m->Xg, (size_t)T * Px * Px * Px);
    alloc(&m->Vg, (size_t)T * Pv * Pv * Pv);
    alloc(&m->XL1, (size_t)T * d->n_x * K1 * K1);
    alloc(&m->XL2, (size_t)T * Px);
    alloc(&m->VL1, (size_t)T * d->n_v * K1 * K1);
    alloc(&m->VL2, (size_t)T * Pv);
    if (e != cudaSuccess) {
        grace_mv_destroy(m);
        return cuda_fail(e, "grace_mv_setup: allocation");
    }
    MvTerms tm;
    std::memset(&tm, 0, sizeof(tm));
    for (int t = 0; t < T; ++t) {
        tm.c[t] = d->coef[t];
        tm.ax[t] = d->ax[t];
        tm.bx[t] = d->bx[t];
        tm.av[t] = d->av[t];
        tm.bv[t] = d->bv[t];
    }
    mv_edges_kernel<<<1, 512>>>(d->n_x, d->x_min, d->x_max, m->ex);
    mv_edges_kernel<<<1, 512>>>(d->n_v, d->v_min, d->v_max, m->ev);
    mv_gauss_kernel<<<1, 32>>>(Q, m->gz, m->gw);
    const long long nx3 = (long long)T * Px * Px * Px, nv3 = (long long)T * Pv * Pv * Pv;
    mv_gain_forms_kernel<<<(unsigned)((nx3 + 127) / 128), 128>>>(0, d->n_x, K1, T, Q, m->ex, m->gz, m->gw, tm, m->Xg);
    mv_gain_forms_kernel<<<(unsigned)((nv3 + 127) / 128), 128>>>(1, d->n_v, K1, T, Q, m->ev, m->gz, m->gw, tm, m->Vg);
    const int nlx = T * d->n_x * K1 * (K1 + 1), nlv = T * d->n_v * K1 * (K1 + 1);
    mv_loss_forms_kernel<<<(nlx + 127) / 128, 128>>>(0, d->n_x, K1, T, Q, m->ex, m->gz, m->gw, tm, m->XL1, m->XL2);
    mv_loss_forms_kernel<<<(nlv + 127) / 128, 128>>>(1, d->n_v, K1, T, Q, m->ev, m->gz, m->gw, tm, m->VL1, m->VL2);
    e = cudaGetLastError();
    if (e == cudaSuccess && d->arithmetic == 1) {
        // FP32 copies of the forms, in the order Xg, Vg, XL1, XL2, VL1, VL2
        const size_t n[6] = {(size_t)nx3, (size_t)nv3, (size_t)T * d->n_x * K1 * K1, (size_t)T * Px,
                             (size_t)T * d->n_v * K1 * K1, (size_t)T * Pv};
        const double *src[6] = {m->Xg, m->Vg, m->XL1, m->XL2, m->VL1, m->VL2};
        size_t tot = 0;
        for (int i = 0; i < 6; ++i) tot += mv_round4(n[i]);   // each copy 16-byte aligned
        e = cudaMalloc(&m->f32, tot * sizeof(float));
        size_t off = 0;
        for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
            mv_to_f32_kernel<<<(unsigned)((n[i] + 255) / 256), 256>>>((long long)n[i], src[i], m->f32 + off);
            off += mv_round4(n[i]);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = d->arithmetic == 0 ? cudaFuncSetAttribute(mv_rhs_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                               : cudaFuncSetAttribute(mv_f32_kernel_for(K1, Pv % 4 == 0), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        grace_mv_destroy(m);
        return cuda_fail(e, "grace_mv_setup: factor forms");
    }
    *out = m;
    return GRACE_OK;
}

grace_status grace_mv_set_stream(grace_mv *m, void *stream)
{
    if (!m) {
        set_error("grace_mv_set_stream: null handle");
        return GRACE_ERR_ARG;
    }
    m->stream = (cudaStream_t)stream;
    return GRACE_OK;
}

}  // extern "C"

template <class R>
static MvArgs<R> mv_args(const grace_mv *m)
{
    MvArgs<R> A;
    A.Nx = m->d.n_x;
    A.Nv = m->d.n_v;
    A.K1 = m->K1;
    A.Px = m->Px;
    A.Pv = m->Pv;
    A.T = m->T;
    if (sizeof(R) == sizeof(double)) {
        A.Xg = (const R *)m->Xg;
        A.Vg = (const R *)m->Vg;
        A.XL1 = (const R *)m->XL1;
        A.XL2 = (const R *)m->XL2;
        A.VL1 = (const R *)m->VL1;
        A.VL2 = (const R *)m->VL2;
    } else {
        const size_t nx3 = mv_round4((size_t)A.T * A.Px * A.Px * A.Px), nv3 = mv_round4((size_t)A.T * A.Pv * A.Pv * A.Pv);
        const size_t nl1x = mv_round4((size_t)A.T * A.Nx * A.K1 * A.K1), nl2x = mv_round4((size_t)A.T * A.Px);
        const size_t nl1v = mv_round4((size_t)A.T * A.Nv * A.K1 * A.K1);
        const R *f = (const R *)m->f32;
        A.Xg = f;
        A.Vg = f + nx3;
        A.XL1 = f + nx3 + nv3;
        A.XL2 = f + nx3 + nv3 + nl1x;
        A.VL1 = f + nx3 + nv3 + nl1x + nl2x;
        A.VL2 = f + nx3 + nv3 + nl1x + nl2x + nl1v;
    }
    return A;
}

static void mv_launch_rhs(const grace_mv *m, int n_cells, const double *g, double *L)
{
    if (m->d.arithmetic)
        mv_f32_kernel_for(m->K1, m->Pv % 4 == 0)<<<n_cells, kMvF32Threads, m->smem, m->stream>>>(mv_args<float>(m), n_cells, g, L);
    else
        mv_rhs_kernel<double><<<n_cells, kMvThreads, m->smem, m->stream>>>(mv_args<double>(m), n_cells, g, L);
}

extern "C" {

grace_status grace_mv_rhs(grace_mv *m, int n_cells, const double *g, double *L)
{
    if (!m || n_cells < 0 || (n_cells > 0 && (!g || !L))) {
        set_error("grace_mv_rhs: bad argument");
        return GRACE_ERR_ARG;
    }
    if (n_cells == 0) return GRACE_OK;
    Guard guard(m->device);
    mv_launch_rhs(m, n_cells, g, L);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_mv_rhs");
}

grace_status grace_mv_step(grace_mv *m, int n_cells, double *g, const double *dt, int n_steps)
{
    if (!m || n_cells < 0 || n_steps < 0 || (n_cells > 0 && (!g || !dt))) {
        set_error("grace_mv_step: bad argument");
        return GRACE_ERR_ARG;
    }
    if (n_cells == 0 || n_steps == 0) return GRACE_OK;
    Guard guard(m->device);
    const long long n = (long long)n_cells * m->P;
    if (m->ws_cells < n_cells) {
        cudaFree(m->ws);
        m->ws = nullptr;
        m->ws_cells = 0;
        const cudaError_t e = cudaMalloc(&m->ws, sizeof(double) * 3 * (size_t)n);
        if (e != cudaSuccess) return cuda_fail(e, "grace_mv_step: workspace");
        m->ws_cells = n_cells;
    }
    double *g1 = m->ws, *g2 = g1 + n, *Lb = g2 + n;
    const unsigned cb = (unsigned)((n + 255) / 256);
    for (int s = 0; s < n_steps; ++s) {
        // SSP-RK3, eq. (RK3); the state and the stage combinations stay FP64
        mv_launch_rhs(m, n_cells, g, Lb);
        mv_combine_kernel<<<cb, 256, 0, m->stream>>>(n, m->P, 0.0, 1.0, g, g, dt, Lb, g1);
        mv_launch_rhs(m, n_cells, g1, Lb);
        mv_combine_kernel<<<cb, 256, 0, m->stream>>>(n, m->P, 0.75, 0.25, g, g1, dt, Lb, g2);
        mv_launch_rhs(m, n_cells, g2, Lb);
        mv_combine_kernel<<<cb, 256, 0, m->stream>>>(n, m->P, 1.0 / 3.0, 2.0 / 3.0, g, g2, dt, Lb, g);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_mv_step");
}

void grace_mv_destroy(grace_mv *m)
{
    if (!m) return;
    Guard guard(m->device);
    cudaFree(m->ex);
    cudaFree(m->ev);
    cudaFree(m->gz);
    cudaFree(m->gw);
    cudaFree(m->Xg);
    cudaFree(m->Vg);
    cudaFree(m->XL1);
    cudaFree(m->XL2);
    cudaFree(m->VL1);
    cudaFree(m->VL2);
    cudaFree(m->f32);
    cudaFree(m->ws);
    delete m;
}

}  // extern "C"
