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
#include "grace_limiter.cuh"
#include "grace_tc_layout.cuh"

namespace grace {

namespace {

constexpr int kB = kKMax + 1;

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

// Writes one cell's new coefficients, staged in shared memory, to the FP64 state
// (coalesced) and, if requested, to the cell's row of the tensor-core A operand
// as whole 16-byte chunks (TF32: 4 values, BF16: 8 hi + 8 lo values per chunk).
__device__ __forceinline__ void write_row(const DevGroup &G, const double *row, long long cell, double *gout,
                                          void *opA, int prec, int kpad, int lane)
{
    const int P = G.P;
    if (gout)
        for (int i = lane; i < P; i += 32) gout[(size_t)cell * P + i] = row[i];
    if (!opA) return;
    const long long tile = cell / kTileM;
    const int r = (int)(cell - tile * kTileM);
    char *t = (char *)opA + (size_t)tile * opA_tile_bytes(prec, kpad);
    if (prec == GRACE_TF32) {
        for (int c = lane; c * 4 < P; c += 32) {
            uint32_t w[4];
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * c + e;
                w[e] = k < P ? f32_to_tf32_rna((float)(row[k] * G.hbin[k / G.K1])) : 0u;
            }
            *reinterpret_cast<uint4 *>(t + swz_offset(kTileM, r, 4 * c, 4)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        const size_t plane = (size_t)kTileM * kpad * 2;
        for (int c = lane; c * 8 < P; c += 32) {
            uint32_t hi[4], lo[4];
            for (int e = 0; e < 4; ++e) {
                uint32_t h2[2], l2[2];
                for (int u = 0; u < 2; ++u) {
                    const int k = 8 * c + 2 * e + u;
                    const double v = k < P ? row[k] * G.hbin[k / G.K1] : 0.0;
                    const __nv_bfloat16 h = __double2bfloat16(v);
                    const __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
                    h2[u] = (uint32_t)__bfloat16_as_ushort(h);
                    l2[u] = (uint32_t)__bfloat16_as_ushort(l);
                }
                hi[e] = h2[0] | (h2[1] << 16);
                lo[e] = l2[0] | (l2[1] << 16);
            }
            const size_t off = swz_offset(kTileM, r, 8 * c, 2);
            *reinterpret_cast<uint4 *>(t + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(t + plane + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

// FT = double: FP64 functionals, everything in FP64 (the plain path).
// FT = float: functionals from the tensor path; the i = 0 row (flux difference,
// stage combination, mass) stays FP64 so the telescoping sum conserves mass to
// FP64 round-off, the i >= 1 rows are formed in FP32 (their error is far below
// that of the reduced-precision contraction they come from).
// One warp per cell; the new row is staged in shared memory and written out
// coalesced.
template <typename FT>
__global__ void __launch_bounds__(256) update_kernel(DevGroup G, UpdateArgs A, int n_cells)
{
    extern __shared__ double rows[];
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const int N = G.N, k = G.k, K1 = G.K1, R = G.R, P = G.P;
    double *row = rows + (size_t)(threadIdx.x >> 5) * P;
    const FT *F = (const FT *)(sizeof(FT) == 8 ? (const void *)A.F : (const void *)A.F32) + cell * R;
    const bool step = A.dt != nullptr;
    const double dt = step ? A.dt[cell] : 0.0;
    double msum = 0.0;
    unsigned fl = 0u;
    for (int j = lane; j < N; j += 32) {
        const FT Fm = j == 0 ? FT(0) : F[j - 1];             // F(x_{j-1/2}), F(x_min) = 0
        const FT Fp = j < G.n_if ? F[j] : FT(0);             // F(x_{j+1/2}), 0 at x_max (cons.)
        const size_t base = (size_t)cell * P + (size_t)j * K1;
        double v[kB];
        const double L0 = ((double)Fm - (double)Fp) * G.inv_h[j];
        v[0] = step ? A.a * A.gn[base] + A.b * (A.gs[base] + dt * L0) : L0;
        if (sizeof(FT) == 8) {
            const double ih = G.inv_h[j];
            for (int i = 1; i <= k; ++i) {
                const double V = (double)F[G.n_if + j * k + i - 1];
                const double L = (2.0 * i + 1.0) * ih * (V - (double)Fp + ((i & 1) ? -(double)Fm : (double)Fm));
                v[i] = step ? A.a * A.gn[base + i] + A.b * (A.gs[base + i] + dt * L) : L;
            }
        } else {
            const float ih = G.inv_h32[j];
            const float a = (float)A.a, b = (float)A.b, dtf = (float)dt;
            const float fp = (float)Fp, fm = (float)Fm;
            for (int i = 1; i <= k; ++i) {
                const float V = (float)F[G.n_if + j * k + i - 1];
                const float L = (2.f * i + 1.f) * ih * (V - fp + ((i & 1) ? -fm : fm));
                v[i] = step ? (double)(a * (float)A.gn[base + i] + b * ((float)A.gs[base + i] + dtf * L)) : (double)L;
            }
        }
        if (step) {
            if (v[0] < 0.0) fl |= GRACE_FLAG_NEGATIVE_MEAN;
            for (int i = 0; i <= k; ++i)
                if (!isfinite(v[i])) fl |= GRACE_FLAG_NONFINITE;
            if (A.apply_limiter) fl |= limit_bin(v, k);
        }
        for (int i = 0; i <= k; ++i) row[j * K1 + i] = v[i];
        if (A.mass) msum += G.hbin[j] * v[0];
    }
    __syncwarp();
    write_row(G, row, cell, A.gout, A.opA, A.opA_prec, A.opA_kpad, lane);
    if (A.mass) {
        msum = warp_sum(msum);
        if (lane == 0) A.mass[cell] = msum;
    }
    if (A.flags) {
        fl = warp_or(fl);
        if (lane == 0 && fl) A.flags[cell] |= (unsigned char)fl;
    }
}

__global__ void __launch_bounds__(256) limit_kernel(DevGroup G, double *g, int n_cells, unsigned char *flags,
                                                     void *opA, int prec, int kpad)
{
    extern __shared__ double rows[];
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const int k = G.k, K1 = G.K1, P = G.P;
    double *row = rows + (size_t)(threadIdx.x >> 5) * P;
    for (int i = lane; i < P; i += 32) row[i] = g[(size_t)cell * P + i];
    __syncwarp();
    unsigned fl = 0u, changed = 0u;
    for (int j = lane; j < G.N; j += 32) {
        double *v = row + j * K1;
        if (G.limiter) {
            const unsigned f = limit_bin(v, k);
            if (f & GRACE_FLAG_LIMITED) changed = 1u;
            fl |= f;
        }
    }
    __syncwarp();
    changed = warp_or(changed);
    write_row(G, row, cell, changed ? g : nullptr, opA, prec, kpad, lane);
    if (flags) {
        fl = warp_or(fl);
        if (lane == 0 && fl) flags[cell] |= (unsigned char)fl;
    }
}

__global__ void __launch_bounds__(256) mass_kernel(DevGroup G, const double *g, int n_cells, double *mass)
{
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    double s = 0.0;
    for (int j = lane; j < G.N; j += 32) s += G.hbin[j] * g[(size_t)cell * G.P + (size_t)j * G.K1];
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
    const size_t smem = (size_t)8 * g.P * sizeof(double);
    if (a.F)
        update_kernel<double><<<warp_blocks(n_cells), 256, smem, st>>>(g, a, n_cells);
    else
        update_kernel<float><<<warp_blocks(n_cells), 256, smem, st>>>(g, a, n_cells);
    return cudaGetLastError();
}

cudaError_t launch_limit(const DevGroup &g, double *d_g, int n_cells, unsigned char *flags, void *opA,
                         int opA_prec, int opA_kpad, cudaStream_t st)
{
    limit_kernel<<<warp_blocks(n_cells), 256, (size_t)8 * g.P * sizeof(double), st>>>(g, d_g, n_cells, flags, opA,
                                                                                       opA_prec, opA_kpad);
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
    limit_kernel<<<warp_blocks(n_cells), 256, (size_t)8 * g.P * sizeof(double), st>>>(
        g0, const_cast<double *>(d_g), n_cells, nullptr, opA, prec, kpad);
    return cudaGetLastError();
}

}  // namespace grace
