// K-c: fused flux difference, SSP-RK3 stage update, scaling limiter, mass and flags.
//
// One warp per cell, one lane per bin.  Lane j reads the cell's flux
// functionals F(x_{j-1/2}), F(x_{j+1/2}) and the volume terms of bin j,
// forms L_j^i of eq. (evo), combines it with the stage inputs as in eq.
// (RK3), optionally applies the scaling limiter of eqs. (recon)/(gamma) to the
// result (the reconstruction that opens the next step), writes the bin, and
// adds h_j g_j^0 to the cell's mass (warp-shuffle reduction, FP64).  The
// i = 0 row only ever sees F(x_{j-1/2}) - F(x_{j+1/2}), so the sum of h_j L_j^0
// telescopes and the mass is conserved to round-off whatever precision the
// functionals came from.
#include "grace_physics.cuh"
#include "grace_tc_layout.cuh"

namespace grace {

namespace {

constexpr int kB = kKMax + 1;

__device__ __forceinline__ double poly(const double *c, int k, double xi)
{
    double P[kB];
    dev_legendre(k, xi, P, nullptr);
    double s = 0.0;
    for (int i = 0; i <= k; ++i) s += c[i] * P[i];
    return s;
}

// minimum over [-1, 1] of sum_i c_i phi_i: endpoints and interior stationary points
__device__ double bin_minimum(const double *c, int k)
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

// eq. (recon) with gamma from eq. (gamma); returns flag bits
__device__ __forceinline__ unsigned limit_bin(double *c, int k)
{
    if (k == 0) return 0u;
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

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned warp_or(unsigned v)
{
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) update_kernel(DevGroup G, UpdateArgs A, int n_cells)
{
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const int N = G.N, k = G.k, K1 = G.K1, R = G.R, P = G.P;
    const double *Fd = A.F ? A.F + cell * R : nullptr;
    const float *Ff = A.F32 ? A.F32 + cell * R : nullptr;
    const double dt = A.dt ? A.dt[cell] : 0.0;
    double msum = 0.0;
    unsigned fl = 0u;
    for (int j = lane; j < N; j += 32) {
        auto Fr = [&](int r) -> double { return Fd ? Fd[r] : (double)Ff[r]; };
        const double Fm = j == 0 ? 0.0 : Fr(j - 1);            // F(x_{j-1/2}), F(x_min) = 0
        const double Fp = j < G.n_if ? Fr(j) : 0.0;            // F(x_{j+1/2}), 0 at x_max (cons.)
        const double h = G.edges[j + 1] - G.edges[j];
        const size_t base = (size_t)cell * P + (size_t)j * K1;
        double v[kB];
        for (int i = 0; i <= k; ++i) {
            const double V = i == 0 ? 0.0 : Fr(G.n_if + j * k + i - 1);
            const double L = (2.0 * i + 1.0) / h * (V - Fp + ((i & 1) ? -Fm : Fm));
            if (A.dt)
                v[i] = A.a * A.gn[base + i] + A.b * (A.gs[base + i] + dt * L);
            else
                v[i] = L;
        }
        if (A.dt) {
            if (v[0] < 0.0) fl |= GRACE_FLAG_NEGATIVE_MEAN;
            for (int i = 0; i <= k; ++i)
                if (!isfinite(v[i])) fl |= GRACE_FLAG_NONFINITE;
            if (A.apply_limiter) fl |= limit_bin(v, k);
        }
        for (int i = 0; i <= k; ++i) A.gout[base + i] = v[i];
        if (A.opA)
            for (int i = 0; i <= k; ++i) opA_store(A.opA, A.opA_prec, A.opA_kpad, cell, j * K1 + i, v[i] * h);
        msum += h * v[0];
    }
    if (A.mass) {
        msum = warp_sum(msum);
        if (lane == 0) A.mass[cell] = msum;
    }
    if (A.flags) {
        fl = warp_or(fl);
        if (lane == 0) A.flags[cell] |= (unsigned char)fl;
    }
}

__global__ void __launch_bounds__(256) limit_kernel(DevGroup G, double *g, int n_cells, unsigned char *flags,
                                                     void *opA, int prec, int kpad)
{
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const int k = G.k, K1 = G.K1;
    unsigned fl = 0u;
    for (int j = lane; j < G.N; j += 32) {
        const size_t base = (size_t)cell * G.P + (size_t)j * K1;
        double v[kB];
        for (int i = 0; i <= k; ++i) v[i] = g[base + i];
        if (G.limiter) {
            const unsigned f = limit_bin(v, k);
            if (f & GRACE_FLAG_LIMITED)
                for (int i = 1; i <= k; ++i) g[base + i] = v[i];
            fl |= f;
        }
        if (opA) {
            const double h = G.edges[j + 1] - G.edges[j];
            for (int i = 0; i <= k; ++i) opA_store(opA, prec, kpad, cell, j * K1 + i, v[i] * h);
        }
    }
    if (flags) {
        fl = warp_or(fl);
        if (lane == 0) flags[cell] |= (unsigned char)fl;
    }
}

__global__ void __launch_bounds__(256) mass_kernel(DevGroup G, const double *g, int n_cells, double *mass)
{
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    double s = 0.0;
    for (int j = lane; j < G.N; j += 32)
        s += (G.edges[j + 1] - G.edges[j]) * g[(size_t)cell * G.P + (size_t)j * G.K1];
    s = warp_sum(s);
    if (lane == 0) mass[cell] = s;
}

struct Rule16 {
    double s[16], w[16];
};

// eq. (init) with a 16-point Gauss rule per bin; one thread per (cell, bin)
__global__ void project_kernel(DevGroup G, Rule16 rule, int kind, const double *ic, int n_cells, double *g)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_cells * G.N) return;
    const long long cell = t / G.N;
    const int j = (int)(t - cell * G.N);
    const double *q = ic + cell * 4;
    const double lo = G.edges[j], hi = G.edges[j + 1];
    const double h = hi - lo, xc = 0.5 * (lo + hi);
    double acc[kB] = {0.0, 0.0, 0.0, 0.0}, P[kB];
    for (int a = 0; a < 16; ++a) {
        const double x = xc + 0.5 * h * rule.s[a];
        double val = 0.0;
        if (kind == GRACE_IC_EXP) val = q[0] * x * exp(-x / q[1]);
        else if (kind == GRACE_IC_POWERLAW) val = (x >= q[2] && x <= q[3]) ? q[0] * pow(x, q[1]) : 0.0;
        else if (kind == GRACE_IC_FIRST_BIN) val = x < G.edges[1] ? q[0] : 0.0;
        dev_legendre(G.k, rule.s[a], P, nullptr);
        for (int i = 0; i <= G.k; ++i) acc[i] += rule.w[a] * val * P[i];
    }
    for (int i = 0; i <= G.k; ++i) g[(size_t)cell * G.P + (size_t)j * G.K1 + i] = acc[i] * (2.0 * i + 1.0) * 0.5;
}

inline int warp_blocks(int n_cells) { return (int)(((long long)n_cells * 32 + 255) / 256); }

}  // namespace

cudaError_t launch_update(const DevGroup &g, const UpdateArgs &a, int n_cells, cudaStream_t st)
{
    update_kernel<<<warp_blocks(n_cells), 256, 0, st>>>(g, a, n_cells);
    return cudaGetLastError();
}

cudaError_t launch_limit(const DevGroup &g, double *d_g, int n_cells, unsigned char *flags, void *opA,
                         int opA_prec, int opA_kpad, cudaStream_t st)
{
    limit_kernel<<<warp_blocks(n_cells), 256, 0, st>>>(g, d_g, n_cells, flags, opA, opA_prec, opA_kpad);
    return cudaGetLastError();
}

cudaError_t launch_mass(const DevGroup &g, const double *d_g, int n_cells, double *mass, cudaStream_t st)
{
    mass_kernel<<<warp_blocks(n_cells), 256, 0, st>>>(g, d_g, n_cells, mass);
    return cudaGetLastError();
}

cudaError_t launch_project(const DevGroup &g, int ic_kind, const double *ic, int n_cells, double *d_g,
                           cudaStream_t st)
{
    Rule16 rule;
    gauss_rule(16, rule.s, rule.w);
    const long long n = (long long)n_cells * g.N;
    project_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, rule, ic_kind, ic, n_cells, d_g);
    return cudaGetLastError();
}

cudaError_t launch_pack_A(const DevGroup &g, const double *d_g, int n_cells, void *opA, int prec, int kpad,
                          cudaStream_t st)
{
    DevGroup g0 = g;
    g0.limiter = 0;
    limit_kernel<<<warp_blocks(n_cells), 256, 0, st>>>(g0, const_cast<double *>(d_g), n_cells, nullptr, opA,
                                                       prec, kpad);
    return cudaGetLastError();
}

}  // namespace grace
