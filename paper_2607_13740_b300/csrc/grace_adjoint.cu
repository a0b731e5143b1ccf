// Tangent-linear and adjoint of the DG right-hand side and of the SSP-RK3 step.
//
// With F_r = g^T T_r g (every flux functional is a quadratic form of the cell's
// coefficients) and L = D F (D: the flux-difference / volume assembly of eq.
// (evo), linear), the derivatives are
//     J v        = D ( g^T (T_r + T_r^T) v )_r                 (JVP)
//     J^T lambda = sum_r mu_r (T_r + T_r^T) g,  mu = D^T lambda  (VJP)
// The scaling limiter (eqs. recon, gamma) is differentiated with the envelope
// theorem: the derivative of the bin minimum with respect to g^i is phi_i at
// the minimiser.  The SSP-RK3 stages (eq. RK3) are reversed exactly, with the
// stage states recomputed from checkpoints.  Parameter gradients contract
// mu with g^T (dT_r / dtheta) g, where dT/dtheta is a central difference of the
// FP64 precompute.
//
// Forms: FP64 on the CUDA cores, and TF32 / BF16x3 on the tensor cores.  The
// tensor-form JVP uses polarization, exact for a quadratic form:
//     J(g) v = [L(g + eps v) - L(g - eps v)] / (2 eps)
// with eps a power of two per cell that brings v to the size of g (so the two
// contractions do not cancel), i.e. two forward contractions of grace_tc.cu.  The
// tensor-form VJP contracts the window-major tiles of S_r = T_r + T_r^T (one MMA
// per tile, Y = Shat ghat) and sums mu_r Y in the epilogue; mu is scaled per cell
// by a power of two into FP32.  The adjoint's own forward sweep then runs the
// tensor form too, so that the reverse sweep differentiates the trajectory it
// recomputes.
#include <string>
#include <vector>

#include "grace_physics.cuh"
#include "grace_tc_layout.cuh"

namespace grace {

namespace {

constexpr int kB = kKMax + 1;

// ------------------------------------------------------------------ JVP contraction
// F_r = sum_{p,q} T_r[p,q] (a_p b_q + b_p a_q), one warp per 32 cells
__global__ void __launch_bounds__(128) contract_pair_kernel(
    const double *__restrict__ T, const int *__restrict__ qlo, const int *__restrict__ qhi,
    const int *__restrict__ prange, int R, int P, const double *__restrict__ a, const double *__restrict__ b,
    int n_cells, double *__restrict__ F)
{
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const long long cell0 = ((long long)blockIdx.x * nw + warp) * 32;
    double *aw = sm + (size_t)warp * 2 * P * 32;
    double *bw = aw + (size_t)P * 32;
    for (int idx = lane; idx < 32 * P; idx += 32) {
        const int c = idx / P, q = idx - c * P;
        const long long cell = cell0 + c;
        aw[q * 32 + c] = cell < n_cells ? a[cell * P + q] : 0.0;
        bw[q * 32 + c] = cell < n_cells ? b[cell * P + q] : 0.0;
    }
    __syncwarp();
    const long long cell = cell0 + lane;
    const int r_per = (R + gridDim.y - 1) / gridDim.y;
    const int r_begin = blockIdx.y * r_per, r_end = min(R, r_begin + r_per);
    for (int r = r_begin; r < r_end; ++r) {
        double Fr = 0.0;
        for (int p = prange[2 * r]; p < prange[2 * r + 1]; ++p) {
            const int q0 = qlo[r * P + p], q1 = qhi[r * P + p];
            if (q0 >= q1) continue;
            const double *Trow = T + ((size_t)r * P + p) * P;
            double ya = 0.0, yb = 0.0;
            for (int q = q0; q < q1; ++q) {
                const double t = __ldg(Trow + q);
                ya = fma(t, aw[q * 32 + lane], ya);
                yb = fma(t, bw[q * 32 + lane], yb);
            }
            Fr = fma(aw[p * 32 + lane], yb, fma(bw[p * 32 + lane], ya, Fr));
        }
        if (cell < n_cells) F[cell * R + r] = Fr;
    }
}

// ------------------------------------------------------------------ mu = D^T lambda
// L_j^i = (2i+1)/h_j [ V_j^i - F_{j+1/2} + (-1)^i F_{j-1/2} ]  (eq. evo)
__global__ void dT_lambda_kernel(DevGroup G, const double *lambda, int n_cells, double *mu)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_cells * G.R) return;
    const long long cell = t / G.R;
    const int r = (int)(t - cell * G.R);
    const double *lam = lambda + cell * G.P;
    double m = 0.0;
    if (r < G.n_if) {
        const int j = r;   // F_{j+1/2}: -(2i+1)/h_j in bin j, +(-1)^i (2i+1)/h_{j+1} in bin j+1
        for (int i = 0; i <= G.k; ++i) {
            m -= (2.0 * i + 1.0) * G.inv_h[j] * lam[j * G.K1 + i];
            if (j + 1 < G.N) m += ((i & 1) ? -1.0 : 1.0) * (2.0 * i + 1.0) * G.inv_h[j + 1] * lam[(j + 1) * G.K1 + i];
        }
    } else {
        const int q = r - G.n_if, j = q / G.k, i = q % G.k + 1;
        m = (2.0 * i + 1.0) * G.inv_h[j] * lam[j * G.K1 + i];
    }
    mu[cell * G.R + r] = m;
}

// ------------------------------------------------------------------ VJP contraction
// w = sum_r mu_r (T_r + T_r^T) g, one warp per 32 cells
__global__ void __launch_bounds__(128) vjp_kernel(const double *__restrict__ T, const int *__restrict__ qlo,
                                                   const int *__restrict__ qhi, const int *__restrict__ prange,
                                                   int R, int P, const double *__restrict__ g,
                                                   const double *__restrict__ mu, int n_cells, double *__restrict__ w)
{
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const long long cell0 = ((long long)blockIdx.x * nw + warp) * 32;
    double *gw = sm + (size_t)warp * 2 * P * 32;
    double *ww = gw + (size_t)P * 32;
    for (int idx = lane; idx < 32 * P; idx += 32) {
        const int c = idx / P, q = idx - c * P;
        const long long cell = cell0 + c;
        gw[q * 32 + c] = cell < n_cells ? g[cell * P + q] : 0.0;
        ww[q * 32 + c] = 0.0;
    }
    __syncwarp();
    const long long cell = cell0 + lane;
    for (int r = 0; r < R; ++r) {
        const double m = cell < n_cells ? mu[cell * R + r] : 0.0;
        for (int p = prange[2 * r]; p < prange[2 * r + 1]; ++p) {
            const int q0 = qlo[r * P + p], q1 = qhi[r * P + p];
            if (q0 >= q1) continue;
            const double *Trow = T + ((size_t)r * P + p) * P;
            const double mg = m * gw[p * 32 + lane];
            double y = 0.0;
            for (int q = q0; q < q1; ++q) {
                const double t = __ldg(Trow + q);
                y = fma(t, gw[q * 32 + lane], y);
                ww[q * 32 + lane] = fma(mg, t, ww[q * 32 + lane]);
            }
            ww[p * 32 + lane] = fma(m, y, ww[p * 32 + lane]);
        }
    }
    __syncwarp();
    for (int idx = lane; idx < 32 * P; idx += 32) {
        const int c = idx / P, q = idx - c * P;
        const long long cl = cell0 + c;
        if (cl < n_cells) w[cl * P + q] = ww[q * 32 + c];
    }
}

// ------------------------------------------------------------------ limiter derivative
__device__ __forceinline__ double poly_at(const double *c, int k, double xi, double *P)
{
    dev_legendre(k, xi, P, nullptr);
    double s = 0.0;
    for (int i = 0; i <= k; ++i) s += c[i] * P[i];
    return s;
}

// minimum of sum_i c_i phi_i on [-1, 1] and its location
__device__ double argmin_bin(const double *c, int k, double *xstar)
{
    double P[kB];
    double m = poly_at(c, k, -1.0, P), t;
    *xstar = -1.0;
    t = poly_at(c, k, 1.0, P);
    if (t < m) { m = t; *xstar = 1.0; }
    double r[2];
    int nr = 0;
    if (k == 2 && c[2] != 0.0) r[nr++] = -c[1] / (3.0 * c[2]);
    if (k == 3) {
        const double A = 7.5 * c[3], B = 3.0 * c[2], C = c[1] - 1.5 * c[3];
        if (A == 0.0) {
            if (B != 0.0) r[nr++] = -C / B;
        } else {
            const double disc = B * B - 4.0 * A * C;
            if (disc >= 0.0) {
                const double sq = sqrt(disc), qq = -0.5 * (B + copysign(sq, B));
                if (qq != 0.0) { r[nr++] = qq / A; r[nr++] = C / qq; }
                else r[nr++] = 0.0;
            }
        }
    }
    for (int n = 0; n < nr; ++n)
        if (r[n] > -1.0 && r[n] < 1.0) {
            t = poly_at(c, k, r[n], P);
            if (t < m) { m = t; *xstar = r[n]; }
        }
    return m;
}

// lambda_g = (d limit / d g)^T lambda_limited, in place on lam; g is the pre-limiter state
__global__ void limiter_vjp_kernel(DevGroup G, const double *g, double *lam, int n_cells)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_cells * G.N || G.k == 0 || !G.limiter) return;
    const long long cell = t / G.N;
    const int j = (int)(t - cell * G.N), k = G.k;
    const size_t base = (size_t)cell * G.P + (size_t)j * G.K1;
    double c[kB], l[kB];
    for (int i = 0; i <= k; ++i) { c[i] = g[base + i]; l[i] = lam[base + i]; }
    const double g0 = c[0];
    if (g0 < 0.0) {                       // gamma = 0: higher modes discarded
        for (int i = 1; i <= k; ++i) lam[base + i] = 0.0;
        return;
    }
    double xs;
    const double m = argmin_bin(c, k, &xs);
    const double den = g0 - m;
    if (!(den > 0.0) || g0 / den >= 1.0) return;   // gamma = 1: identity
    const double gamma = g0 / den;
    double P[kB];
    dev_legendre(k, xs, P, nullptr);
    double S = 0.0;
    for (int i = 1; i <= k; ++i) S += l[i] * c[i];
    // d gamma / d g^0 = 1 / (g0 - m), d gamma / d g^i = g0 phi_i(xi*) / (g0 - m)^2; written with
    // S / den and gamma = g0 / den so that tiny bins neither overflow nor produce 0 * inf
    const double sd = S / den;
    lam[base] = l[0] + sd;
    for (int j2 = 1; j2 <= k; ++j2) lam[base + j2] = gamma * l[j2] + sd * gamma * P[j2];
}

// ------------------------------------------------------------------ small vector kernels
// out = a * x + b * (y + dt_c * z)   (dt per cell; any of y, z may be null)
__global__ void axpby_dt_kernel(int P, long long n, double a, const double *x, double b, const double *y,
                                const double *z, const double *dt, double *out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const long long cell = t / P;
    double v = y ? y[t] : 0.0;
    if (z) v += dt[cell] * z[t];
    out[t] = (x ? a * x[t] : 0.0) + b * v;
}

// dtheta[cell][ip] += w * dt_c * sum_r mu_r Fp_r
__global__ void param_dot_kernel(int R, int n_cells, const double *mu, const double *Fp, const double *dt, double w,
                                 int n_params, int ip, double *dtheta)
{
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= n_cells) return;
    double s = 0.0;
    for (int r = 0; r < R; ++r) s = fma(mu[(size_t)cell * R + r], Fp[(size_t)cell * R + r], s);
    dtheta[(size_t)cell * n_params + ip] += w * dt[cell] * s;
}

// dtheta[cell][ip] += w dt mu . Fp with Fp from a tensor-core contraction ([tile][R][128]); only
// the functionals its tiles write (written[r]) count, the others are zero
__global__ void param_dot_f32_kernel(int R, int n_cells, const double *__restrict__ mu, const float *__restrict__ Fp,
                                     const int *__restrict__ written, const double *__restrict__ dt, double w,
                                     int n_params, int ip, double *__restrict__ dtheta)
{
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= n_cells) return;
    const long long ct = cell / kTileM;
    const int row = cell - (int)ct * kTileM;
    double s = 0.0;
    for (int r = 0; r < R; ++r)
        if (written[r]) s = fma(mu[(size_t)cell * R + r], (double)Fp[((size_t)ct * R + r) * kTileM + row], s);
    dtheta[(size_t)cell * n_params + ip] += w * dt[cell] * s;
}

// ------------------------------------------------------------------ tensor-form pieces
__device__ __forceinline__ double warp_max(double x)
{
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// mu (FP64 [cell][R]) -> mu * 2^-e in FP32, [tile][R][128] layout, with 2^e per cell so that
// the largest |mu| of the cell lies in [0.5, 1); one warp per cell
__global__ void mu_to_f32_kernel(int R, int n_cells, const double *__restrict__ mu, float *__restrict__ mu32,
                                 double *__restrict__ inv_scale)
{
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const double *m = mu + cell * R;
    double mx = 0.0;
    for (int r = lane; r < R; r += 32) mx = fmax(mx, fabs(m[r]));
    mx = warp_max(mx);
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
    const double sc = ldexp(1.0, -e);
    const long long ct = cell / kTileM;
    const int row = (int)(cell - ct * kTileM);
    for (int r = lane; r < R; r += 32) mu32[((size_t)ct * R + r) * kTileM + row] = (float)(m[r] * sc);
    if (lane == 0) inv_scale[cell] = ldexp(1.0, e);
}

// w[cell][p] = 2^e h_bin(p) (W0 + W1)[p]: the two epilogue planes of the VJP contraction, unscaled
__global__ void vjp_combine_kernel(DevGroup G, int Pw, int n_cells, int planes, const float *__restrict__ W,
                                   const double *__restrict__ inv_scale, double *__restrict__ w)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_cells * G.P) return;
    const long long cell = t / G.P;
    const int p = (int)(t - cell * G.P);
    const long long ct = cell / kTileM, tiles = (n_cells + kTileM - 1) / kTileM;
    const int row = (int)(cell - ct * kTileM);
    double s = 0.0;
    for (int q = 0; q < planes; ++q) s += (double)W[(((size_t)q * tiles + ct) * Pw + p) * kTileM + row];
    w[t] = inv_scale[cell] * G.hbin[p / G.K1] * s;
}

// a = g + eps v, b = g - eps v with eps = 2^(e_g - e_v) per cell (e: binary exponents of the
// largest |g| and |v|), one warp per cell
__global__ void polar_kernel(int P, int n_cells, const double *__restrict__ g, const double *__restrict__ v,
                             double *__restrict__ a, double *__restrict__ b, double *__restrict__ eps)
{
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const double *gc = g + cell * P, *vc = v + cell * P;
    double mg = 0.0, mv = 0.0;
    for (int q = lane; q < P; q += 32) {
        mg = fmax(mg, fabs(gc[q]));
        mv = fmax(mv, fabs(vc[q]));
    }
    mg = warp_max(mg);
    mv = warp_max(mv);
    int eg = 0, ev = 0;
    if (mg > 0.0 && isfinite(mg)) frexp(mg, &eg);
    if (mv > 0.0 && isfinite(mv)) frexp(mv, &ev);
    const double ep = ldexp(1.0, eg - ev);
    for (int q = lane; q < P; q += 32) {
        a[cell * P + q] = fma(ep, vc[q], gc[q]);
        b[cell * P + q] = fma(-ep, vc[q], gc[q]);
    }
    if (lane == 0) eps[cell] = ep;
}

// dF[cell][r] (+)= sign F32[tile][r][row] / (2 eps[cell])
__global__ void polar_accumulate_kernel(int R, int n_cells, const float *__restrict__ F32,
                                        const double *__restrict__ eps, double sign, int accumulate,
                                        double *__restrict__ dF)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_cells * R) return;
    const long long cell = t / R;
    const int r = (int)(t - cell * R);
    const long long ct = cell / kTileM;
    const int row = (int)(cell - ct * kTileM);
    const double v = sign * (double)F32[((size_t)ct * R + r) * kTileM + row] / (2.0 * eps[cell]);
    dF[t] = accumulate ? dF[t] + v : v;
}

// dF = (Fa - Fb) / (2 eps[cell]) in FP64 (per-cell-kernel JVP by polarization)
__global__ void polar_combine_kernel(int R, int n_cells, const double *__restrict__ Fa, const double *__restrict__ Fb,
                                     const double *__restrict__ eps, double *__restrict__ dF)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_cells * R) return;
    dF[t] = (Fa[t] - Fb[t]) / (2.0 * eps[t / R]);
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

size_t warp_tile_smem(int P, int arrays, int *wpb)
{
    const size_t per = (size_t)P * 32 * sizeof(double) * arrays;
    int w = (int)((200 * 1024) / per);
    if (w > 4) w = 4;
    *wpb = w;
    return per * (w > 0 ? w : 1);
}

}  // namespace

cudaError_t launch_jvp_contract(const DevGroup &g, const double *T, const int *qlo, const int *qhi,
                                const int *prange, const double *a, const double *b, int n, double *F,
                                cudaStream_t st)
{
    int wpb;
    const size_t smem = warp_tile_smem(g.P, 2, &wpb);
    if (wpb < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(contract_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(blocks(n, 32 * wpb), fp64_functional_chunks(n, g.R));
    contract_pair_kernel<<<grid, 32 * wpb, smem, st>>>(T, qlo, qhi, prange, g.R, g.P, a, b, n, F);
    return cudaGetLastError();
}

cudaError_t launch_vjp(const DevGroup &g, const double *T, const int *qlo, const int *qhi, const int *prange,
                       const double *gst, const double *lambda, double *mu_ws, int n, double *w, cudaStream_t st)
{
    dT_lambda_kernel<<<blocks((long long)n * g.R, 256), 256, 0, st>>>(g, lambda, n, mu_ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int wpb;
    const size_t smem = warp_tile_smem(g.P, 2, &wpb);
    if (wpb < 1) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(vjp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    vjp_kernel<<<blocks(n, 32 * wpb), 32 * wpb, smem, st>>>(T, qlo, qhi, prange, g.R, g.P, gst, mu_ws, n, w);
    return cudaGetLastError();
}

cudaError_t launch_mu(const DevGroup &g, const double *lambda, int n, double *mu, cudaStream_t st)
{
    dT_lambda_kernel<<<blocks((long long)n * g.R, 256), 256, 0, st>>>(g, lambda, n, mu);
    return cudaGetLastError();
}

cudaError_t launch_limiter_vjp(const DevGroup &g, const double *gpre, double *lam, int n, cudaStream_t st)
{
    limiter_vjp_kernel<<<blocks((long long)n * g.N, 256), 256, 0, st>>>(g, gpre, lam, n);
    return cudaGetLastError();
}

cudaError_t launch_axpby_dt(int P, int n, double a, const double *x, double b, const double *y, const double *z,
                            const double *dt, double *out, cudaStream_t st)
{
    const long long m = (long long)n * P;
    axpby_dt_kernel<<<blocks(m, 256), 256, 0, st>>>(P, m, a, x, b, y, z, dt, out);
    return cudaGetLastError();
}

cudaError_t launch_param_dot(int R, int n, const double *mu, const double *Fp, const double *dt, double w,
                             int n_params, int ip, double *dtheta, cudaStream_t st)
{
    param_dot_kernel<<<blocks(n, 128), 128, 0, st>>>(R, n, mu, Fp, dt, w, n_params, ip, dtheta);
    return cudaGetLastError();
}

}  // namespace grace

// ====================================================================== host side
namespace grace {

void free_param_derivs(Group &G)
{
    for (ParamDeriv &d : G.dparams) {
        for (auto &t : d.tc) free_tc_tiles(t);
        cudaFree(d.d_dT);
        cudaFree(d.d_qlo);
        cudaFree(d.d_qhi);
        cudaFree(d.d_prange);
    }
    G.dparams.clear();
}

namespace {

__global__ void central_diff_kernel(size_t n, const double *a, const double *b, double inv2h, double *out)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (a[i] - b[i]) * inv2h;
}

double *param_slot(grace_group_desc &d, int id)
{
    if (id < 0 || id >= 24) return nullptr;
    if (id < 8) return &d.coag_p[id];
    if (id < 16) return &d.frag_p[id - 8];
    return &d.break_p[id - 16];
}

// the adjoint calls work on batches of one group in the caller's order; groups with a per-cell
// kernel parameter (no fixed T) in FP64 only, once their parameters are set
grace_status single_part(grace_batch *b, const char *who, int precision = GRACE_FP64)
{
    if (b->parts.size() != 1 || !b->parts[0].direct) {
        set_error(std::string(who) + ": batches mixing groups are not supported");
        return GRACE_ERR_UNSUPPORTED;
    }
    if (b->ctx->groups[b->parts[0].group].dg.cell_alpha) {
        if (precision != GRACE_FP64) {
            set_error(std::string(who) + ": groups with a per-cell kernel parameter: FP64 only");
            return GRACE_ERR_UNSUPPORTED;
        }
        if (!b->alpha_set) {
            set_error(std::string(who) + ": per-cell kernel parameters not set: call grace_batch_cell_params first");
            return GRACE_ERR_ORDER;
        }
    }
    return GRACE_OK;
}

// per-cell-kernel groups: the adjoint's workspaces of the part (allocated on first use)
cudaError_t nc_adjoint_ws(grace_batch *b)
{
    Part &p = b->parts[0];
    const Group &G = b->ctx->groups[p.group];
    if (p.d_gamma) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p.d_gamma, (size_t)p.n * G.nc.NQ * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p.d_F2, (size_t)p.n * G.dg.R * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p.d_eps, (size_t)p.n * sizeof(double));
    return e;
}

// FP64 flux functionals of either kind of group into dF
cudaError_t functionals_fp64(grace_batch *b, const double *g, double *dF, cudaStream_t st)
{
    Part &p = b->parts[0];
    Group &G = b->ctx->groups[p.group];
    return G.dg.cell_alpha ? launch_nc_functionals(G.dg, G.nc, g, p.d_alpha, b->n_cells, p.d_G, p.d_H, dF, st)
                           : launch_contract_fp64(G.dg, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, g, b->n_cells, dF, st);
}

// FP64 J(gs)^T lambda into w for either kind of group; leaves mu = D^T lambda in the part's d_F
cudaError_t vjp_fp64(grace_batch *b, const double *gs, const double *lambda, double *w, cudaStream_t st)
{
    Part &p = b->parts[0];
    Group &G = b->ctx->groups[p.group];
    if (!G.dg.cell_alpha) return launch_vjp(G.dg, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, gs, lambda, p.d_F, b->n_cells, w, st);
    cudaError_t e = nc_adjoint_ws(b);
    if (e == cudaSuccess) e = launch_mu(G.dg, lambda, b->n_cells, p.d_F, st);
    if (e == cudaSuccess) e = launch_nc_vjp(G.dg, G.nc, gs, p.d_alpha, p.d_F, b->n_cells, p.d_G, p.d_H, p.d_gamma, w, st);
    return e;
}

// tensor forms: the precision's tiles (forward, and VJP tiles built on first use) and the
// workspaces of this file (VJP planes, FP32 mu, per-cell scales), allocated on first use
grace_status prepare_tc(grace_batch *b, int prec, bool vjp, const char *who)
{
    if (prec != GRACE_TF32 && prec != GRACE_BF16X3) {
        set_error(std::string(who) + ": unknown precision");
        return GRACE_ERR_ARG;
    }
    Group &G = b->ctx->groups[b->parts[0].group];
    Part &p = b->parts[0];
    if (!G.tc[prec].built || !p.d_opA) {
        set_error(std::string(who) + ": precision not precomputed: pass its bit to grace_precompute before binding the batch");
        return GRACE_ERR_ORDER;
    }
    if (vjp && !G.tcv[prec].built) {
        grace_status s = build_vjp_tiles(G, prec, b->ctx->stream);
        if (s != GRACE_OK) return s;
    }
    // parameter derivatives dT/dtheta of grace_param_grad_setup, contracted like T
    for (ParamDeriv &pd : G.dparams)
        if (vjp && !pd.tc[prec].built) {
            grace_status s = build_tc_tiles_from(G, pd.d_dT, prec, pd.tc[prec], b->ctx->stream);
            if (s != GRACE_OK) return s;
        }
    const size_t tiles = ((size_t)p.n + kTileM - 1) / kTileM;
    cudaError_t e = cudaSuccess;
    if (!p.d_W32)
        e = cudaMalloc(&p.d_W32, tc_vjp_planes() * tiles * vjp_window_cols(G.dg) * kTileM * sizeof(float));
    if (e == cudaSuccess && !p.d_mu32) e = cudaMalloc(&p.d_mu32, tiles * G.dg.R * kTileM * sizeof(float));
    if (e == cudaSuccess && !p.d_cscale) e = cudaMalloc(&p.d_cscale, (size_t)p.n * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string(who) + ": workspace allocation failed");
        return GRACE_ERR_NOMEM;
    }
    return GRACE_OK;
}

// J(g) v in a tensor form by polarization, into Jv
cudaError_t jvp_tc(grace_batch *b, int prec, const double *g, const double *v, double *Jv, cudaStream_t st)
{
    Group &G = b->ctx->groups[b->parts[0].group];
    Part &p = b->parts[0];
    const DevGroup &dg = G.dg;
    const int n = p.n;
    polar_kernel<<<blocks((long long)n * 32, 256), 256, 0, st>>>(dg.P, n, g, v, p.d_g1, p.d_g2, p.d_cscale);
    cudaError_t e = cudaGetLastError();
    const double *src[2] = {p.d_g1, p.d_g2};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = launch_pack_A(dg, src[k], n, p.d_opA, prec, G.tc[prec].k_pad, G.tc[prec].k_ofs, st);
        if (e == cudaSuccess) e = launch_contract_tc(dg, G.tc[prec], prec, p.d_opA, n, p.d_F32, b->d_err, st);
        if (e == cudaSuccess) {
            polar_accumulate_kernel<<<blocks((long long)n * dg.R, 256), 256, 0, st>>>(
                dg.R, n, p.d_F32, p.d_cscale, k == 0 ? 1.0 : -1.0, k, p.d_F);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        UpdateArgs u;
        u.F = p.d_F;
        u.gout = Jv;
        e = launch_update(dg, u, n, st);
    }
    return e;
}

// J(gs)^T lambda in a tensor form, into w; leaves mu = D^T lambda (FP64) in the part's d_F
cudaError_t vjp_tc(grace_batch *b, int prec, const double *gs, const double *lambda, double *w, cudaStream_t st)
{
    Group &G = b->ctx->groups[b->parts[0].group];
    Part &p = b->parts[0];
    const DevGroup &dg = G.dg;
    const int n = p.n;
    const size_t tiles = ((size_t)n + kTileM - 1) / kTileM;
    cudaError_t e = launch_mu(dg, lambda, n, p.d_F, st);
    if (e == cudaSuccess) {
        mu_to_f32_kernel<<<blocks((long long)n * 32, 256), 256, 0, st>>>(dg.R, n, p.d_F, p.d_mu32, p.d_cscale);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_pack_A(dg, gs, n, p.d_opA, prec, G.tc[prec].k_pad, G.tc[prec].k_ofs, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(p.d_W32, 0, tc_vjp_planes() * tiles * vjp_window_cols(dg) * kTileM * sizeof(float), st);
    if (e == cudaSuccess) e = launch_vjp_tc(dg, G.tcv[prec], prec, p.d_opA, p.d_mu32, n, p.d_W32, b->d_err, st);
    if (e == cudaSuccess) {
        vjp_combine_kernel<<<blocks((long long)n * dg.P, 256), 256, 0, st>>>(dg, vjp_window_cols(dg), n,
                                                                              tc_vjp_planes(), p.d_W32,
                                                                              p.d_cscale, w);
        e = cudaGetLastError();
    }
    return e;
}

// one forward SSP-RK3 step in a tensor form (FP64 stage rows, FP32 higher modes as in grace_step)
cudaError_t fwd_step_tc(grace_batch *b, int prec, const double *pre, double *gt, double *g1, double *g2,
                        double *next, const double *dt)
{
    Group &G = b->ctx->groups[b->parts[0].group];
    const DevGroup &dg = G.dg;
    Part &p = b->parts[0];
    cudaStream_t st = b->ctx->stream;
    const int n = b->n_cells;
    const size_t bytes = (size_t)n * dg.P * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(gt, pre, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && dg.limiter) e = launch_limit(dg, gt, n, nullptr, nullptr, 0, 0, 0, st);
    const double *gin[3] = {gt, g1, g2};
    double *gout[3] = {g1, g2, next};
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
        e = launch_pack_A(dg, gin[s], n, p.d_opA, prec, G.tc[prec].k_pad, G.tc[prec].k_ofs, st);
        if (e == cudaSuccess) e = launch_contract_tc(dg, G.tc[prec], prec, p.d_opA, n, p.d_F32, b->d_err, st);
        if (e != cudaSuccess) break;
        UpdateArgs u;
        u.F32 = p.d_F32;
        u.gn = gt;
        u.gs = gin[s];
        u.gout = gout[s];
        u.dt = dt;
        u.a = ca[s];
        u.b = cb[s];
        e = launch_update_tc(dg, u, n, st);
    }
    return e;
}

// one forward SSP-RK3 step in FP64 that keeps the stage states:
// pre -> gt (limited) -> g1 -> g2 -> next
cudaError_t fwd_step(grace_batch *b, const double *pre, double *gt, double *g1, double *g2, double *next,
                     const double *dt)
{
    Group &G = b->ctx->groups[b->parts[0].group];
    const DevGroup &dg = G.dg;
    cudaStream_t st = b->ctx->stream;
    const int n = b->n_cells;
    double *dF = b->parts[0].d_F;
    const size_t bytes = (size_t)n * dg.P * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(gt, pre, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && dg.limiter) e = launch_limit(dg, gt, n, nullptr, nullptr, 0, 0, 0, st);
    const double *gin[3] = {gt, g1, g2};
    double *gout[3] = {g1, g2, next};
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
        e = functionals_fp64(b, gin[s], dF, st);
        if (e != cudaSuccess) break;
        UpdateArgs u;
        u.F = dF;
        u.gn = gt;
        u.gs = gin[s];
        u.gout = gout[s];
        u.dt = dt;
        u.a = ca[s];
        u.b = cb[s];
        e = launch_update(dg, u, n, st);
    }
    return e;
}

}  // namespace
}  // namespace grace

using namespace grace;

extern "C" {

grace_status grace_rhs_jvp(grace_batch *b, const double *g, const double *v, double *Jv, int precision)
{
    if (!b || !g || !v || !Jv) {
        set_error("grace_rhs_jvp: null argument");
        return GRACE_ERR_ARG;
    }
    grace_status sp = single_part(b, "grace_rhs_jvp", precision);
    if (sp != GRACE_OK) return sp;
    Guard guard(b->ctx->device);
    if (precision != GRACE_FP64) {
        sp = prepare_tc(b, precision, false, "grace_rhs_jvp");
        if (sp != GRACE_OK) return sp;
        cudaError_t e = jvp_tc(b, precision, g, v, Jv, b->ctx->stream);
        return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_rhs_jvp");
    }
    Group &G = b->ctx->groups[b->parts[0].group];
    cudaStream_t st = b->ctx->stream;
    Part &p = b->parts[0];
    double *dF = p.d_F;
    cudaError_t e = cudaSuccess;
    if (G.dg.cell_alpha) {
        // no fixed T: polarization of the quadratic L, exact up to rounding, with eps = 2^(e_g - e_v)
        // per cell so that g +- eps v keep the size of g
        e = nc_adjoint_ws(b);
        if (e == cudaSuccess) {
            polar_kernel<<<blocks((long long)b->n_cells * 32, 256), 256, 0, st>>>(G.dg.P, b->n_cells, g, v, p.d_g1,
                                                                                   p.d_g2, p.d_eps);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = functionals_fp64(b, p.d_g1, dF, st);
        if (e == cudaSuccess) e = functionals_fp64(b, p.d_g2, p.d_F2, st);
        if (e == cudaSuccess) {
            polar_combine_kernel<<<blocks((long long)b->n_cells * G.dg.R, 256), 256, 0, st>>>(G.dg.R, b->n_cells, dF,
                                                                                               p.d_F2, p.d_eps, dF);
            e = cudaGetLastError();
        }
    } else {
        e = launch_jvp_contract(G.dg, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, g, v, b->n_cells, dF, st);
    }
    if (e == cudaSuccess) {
        UpdateArgs u;
        u.F = dF;
        u.gout = Jv;
        e = launch_update(G.dg, u, b->n_cells, st);
    }
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_rhs_jvp");
}

grace_status grace_rhs_vjp(grace_batch *b, const double *g, const double *lambda, double *w, int precision)
{
    if (!b || !g || !lambda || !w) {
        set_error("grace_rhs_vjp: null argument");
        return GRACE_ERR_ARG;
    }
    grace_status sp = single_part(b, "grace_rhs_vjp", precision);
    if (sp != GRACE_OK) return sp;
    Guard guard(b->ctx->device);
    if (precision != GRACE_FP64) {
        sp = prepare_tc(b, precision, true, "grace_rhs_vjp");
        if (sp != GRACE_OK) return sp;
        cudaError_t e = vjp_tc(b, precision, g, lambda, w, b->ctx->stream);
        return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_rhs_vjp");
    }
    cudaError_t e = vjp_fp64(b, g, lambda, w, b->ctx->stream);
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_rhs_vjp");
}

grace_status grace_param_grad_setup(grace_ctx *ctx, int group, int n_params, const int *param_ids,
                                    double rel_step)
{
    if (!ctx || group < 0 || group >= (int)ctx->groups.size() || n_params < 0 || (n_params > 0 && !param_ids)) {
        set_error("grace_param_grad_setup: bad argument");
        return GRACE_ERR_ARG;
    }
    if (!ctx->precomputed) {
        set_error("grace_param_grad_setup: call grace_precompute first");
        return GRACE_ERR_ORDER;
    }
    const bool exact = !(rel_step > 0.0);
    Guard guard(ctx->device);
    Group &G = ctx->groups[group];
    if (G.dg.cell_alpha) {
        set_error("grace_param_grad_setup: groups with a per-cell kernel parameter have no fixed T (not supported)");
        return GRACE_ERR_UNSUPPORTED;
    }
    free_param_derivs(G);
    const DevGroup &dg = G.dg;
    const size_t nT = (size_t)dg.R * dg.P * dg.P;
    for (int i = 0; i < n_params; ++i)
        if (param_ids[i] < 0 || param_ids[i] >= 24) {
            set_error("grace_param_grad_setup: parameter id out of range (0..23)");
            return GRACE_ERR_ARG;
        }
    double *tp = nullptr, *tm = nullptr;
    cudaError_t e = cudaSuccess;
    if (!exact) {
        e = cudaMalloc(&tp, nT * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&tm, nT * sizeof(double));
    }
    for (int i = 0; i < n_params && e == cudaSuccess; ++i) {
        ParamDeriv pd;
        pd.id = param_ids[i];
        pd.step = 0.0;
        e = cudaMalloc(&pd.d_dT, nT * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&pd.d_qlo, sizeof(int) * dg.R * dg.P);
        if (e == cudaSuccess) e = cudaMalloc(&pd.d_qhi, sizeof(int) * dg.R * dg.P);
        if (e == cudaSuccess) e = cudaMalloc(&pd.d_prange, sizeof(int) * 2 * dg.R);
        G.dparams.push_back(pd);
        if (e != cudaSuccess) break;
        if (exact) {
            // forward mode through the FP64 precompute: the kernels' and breakage functions'
            // derivatives (eqs. break, inte1, inte2, App. B; the Maxwellian probabilities of
            // Sec. 4.5) carried through the same quadrature sums
            double dbc = 0.0, dbf = 0.0;
            maxwell_beta_derivs(G.desc, pd.id, &dbc, &dbf);
            e = launch_build_dT(dg, pd.id, dbc, dbf, G.dparams.back().d_dT, ctx->stream);
        } else {
            grace_group_desc dplus = G.desc, dminus = G.desc;
            double *sp = param_slot(dplus, pd.id), *sm = param_slot(dminus, pd.id);
            const double h = *sp != 0.0 ? rel_step * std::fabs(*sp) : rel_step;
            *sp += h;
            *sm -= h;
            G.dparams.back().step = h;
            e = launch_build_T(make_devgroup(dplus, G.d_edges), tp, ctx->stream);
            if (e == cudaSuccess) e = launch_build_T(make_devgroup(dminus, G.d_edges), tm, ctx->stream);
            if (e == cudaSuccess) {
                central_diff_kernel<<<1024, 256, 0, ctx->stream>>>(nT, tp, tm, 0.5 / h, G.dparams.back().d_dT);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess) e = launch_row_extents(dg, pd.d_dT, pd.d_qlo, pd.d_qhi, pd.d_prange, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(tp);
    cudaFree(tm);
    if (e != cudaSuccess) {
        free_param_derivs(G);
        return cuda_fail(e, "grace_param_grad_setup");
    }
    return GRACE_OK;
}

grace_status grace_adjoint(grace_batch *b, const double *g0, const double *dt, int n_steps, int ckpt_every,
                           const double *lambda_T, double *lambda_0, double *dtheta, int precision)
{
    if (!b || !g0 || !dt || !lambda_T || !lambda_0 || n_steps < 0 || ckpt_every < 1) {
        set_error("grace_adjoint: null argument, negative step count or ckpt_every < 1");
        return GRACE_ERR_ARG;
    }
    grace_status sp = single_part(b, "grace_adjoint", precision);
    if (sp != GRACE_OK) return sp;
    Guard guard(b->ctx->device);
    const bool tc = precision != GRACE_FP64;
    if (tc) {
        sp = prepare_tc(b, precision, true, "grace_adjoint");
        if (sp != GRACE_OK) return sp;
    }
    Group &G = b->ctx->groups[b->parts[0].group];
    const DevGroup &dg = G.dg;
    cudaStream_t st = b->ctx->stream;
    const int n = b->n_cells, P = dg.P, R = dg.R;
    double *dF = b->parts[0].d_F;
    const size_t vec = (size_t)n * P;
    const int n_ck = n_steps > 0 ? (n_steps + ckpt_every - 1) / ckpt_every : 1;
    const int np = (int)G.dparams.size();
    // workspace: checkpoints, per-step (pre, gt, g1, g2) of one segment, 6 adjoint vectors, Fp
    const size_t need = sizeof(double) * (vec * (size_t)n_ck + vec * 4 * (size_t)ckpt_every + 6 * vec +
                                          (size_t)n * R);
    cudaError_t e = cudaSuccess;
    if (b->adj_bytes < need) {
        cudaFree(b->d_adj);
        b->d_adj = nullptr;
        b->adj_bytes = 0;
        e = cudaMalloc(&b->d_adj, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("grace_adjoint: workspace allocation failed");
            return GRACE_ERR_NOMEM;
        }
        b->adj_bytes = need;
    }
    double *ck = b->d_adj;
    double *seg = ck + vec * n_ck;
    double *lam = seg + vec * 4 * ckpt_every;
    double *lt = lam + vec, *l1 = lt + vec, *l2 = l1 + vec, *tmp = l2 + vec, *cur = tmp + vec;
    double *Fp = cur + vec;
    const size_t bytes = vec * sizeof(double);
    if (dtheta && np > 0) e = cudaMemsetAsync(dtheta, 0, sizeof(double) * n * np, st);

    // forward sweep: checkpoints every ckpt_every steps
    if (e == cudaSuccess) e = cudaMemcpyAsync(cur, g0, bytes, cudaMemcpyDeviceToDevice, st);
    for (int s = 0; s < n_steps && e == cudaSuccess; ++s) {
        if (s % ckpt_every == 0) e = cudaMemcpyAsync(ck + vec * (s / ckpt_every), cur, bytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = tc ? fwd_step_tc(b, precision, cur, seg, seg + vec, seg + 2 * vec, cur, dt)
                   : fwd_step(b, cur, seg, seg + vec, seg + 2 * vec, cur, dt);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam, lambda_T, bytes, cudaMemcpyDeviceToDevice, st);

    auto vjp_at = [&](const double *gs, const double *l, double *out) {
        return tc ? vjp_tc(b, precision, gs, l, out, st) : vjp_fp64(b, gs, l, out, st);
    };
    // dtheta += w dt mu(l) . g^T dT g (mu of the last vjp is in b->d_F).  Tensor forms: the
    // A operand of gs is still packed by the VJP; g^T dT g goes to the FP32 mu buffer, free
    // once the VJP contraction has run
    auto param_terms = [&](const double *gs, double w) {
        cudaError_t r = cudaSuccess;
        for (int i = 0; i < np && r == cudaSuccess && dtheta; ++i) {
            const ParamDeriv &pd = G.dparams[i];
            if (tc) {
                const TcTiles &t = pd.tc[precision];
                if (t.n_tiles == 0) continue;      // T does not depend on this parameter
                Part &p = b->parts[0];
                r = launch_contract_tc(dg, t, precision, p.d_opA, n, p.d_mu32, b->d_err, st);
                if (r == cudaSuccess) {
                    param_dot_f32_kernel<<<blocks(n, 128), 128, 0, st>>>(R, n, dF, p.d_mu32, t.d_written, dt, w, np,
                                                                         i, dtheta);
                    r = cudaGetLastError();
                }
                continue;
            }
            r = launch_contract_fp64(dg, pd.d_dT, pd.d_qlo, pd.d_qhi, pd.d_prange, gs, n, Fp, st);
            if (r == cudaSuccess) r = launch_param_dot(R, n, dF, Fp, dt, w, np, i, dtheta, st);
        }
        return r;
    };

    for (int sg = n_ck - 1; sg >= 0 && e == cudaSuccess && n_steps > 0; --sg) {
        const int s0 = sg * ckpt_every, s1 = std::min(s0 + ckpt_every, n_steps);
        // recompute the segment, keeping (pre, gt, g1, g2) of every step
        e = cudaMemcpyAsync(cur, ck + vec * sg, bytes, cudaMemcpyDeviceToDevice, st);
        for (int s = s0; s < s1 && e == cudaSuccess; ++s) {
            double *S = seg + vec * 4 * (s - s0);
            e = cudaMemcpyAsync(S, cur, bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = tc ? fwd_step_tc(b, precision, S, S + vec, S + 2 * vec, S + 3 * vec, cur, dt)
                       : fwd_step(b, S, S + vec, S + 2 * vec, S + 3 * vec, cur, dt);
        }
        for (int s = s1 - 1; s >= s0 && e == cudaSuccess; --s) {
            const double *S = seg + vec * 4 * (s - s0);
            const double *pre = S, *gt = S + vec, *g1 = S + 2 * vec, *g2 = S + 3 * vec;
            // stage 3: g' = 1/3 gt + 2/3 (g2 + dt L(g2))
            e = vjp_at(g2, lam, tmp);
            if (e == cudaSuccess) e = param_terms(g2, 2.0 / 3.0);
            if (e == cudaSuccess) e = launch_axpby_dt(P, n, 0.0, nullptr, 2.0 / 3.0, lam, tmp, dt, l2, st);
            if (e == cudaSuccess) e = launch_axpby_dt(P, n, 0.0, nullptr, 1.0 / 3.0, lam, nullptr, dt, lt, st);
            // stage 2: g2 = 3/4 gt + 1/4 (g1 + dt L(g1))
            if (e == cudaSuccess) e = vjp_at(g1, l2, tmp);
            if (e == cudaSuccess) e = param_terms(g1, 0.25);
            if (e == cudaSuccess) e = launch_axpby_dt(P, n, 0.0, nullptr, 0.25, l2, tmp, dt, l1, st);
            if (e == cudaSuccess) e = launch_axpby_dt(P, n, 1.0, lt, 0.75, l2, nullptr, dt, lt, st);
            // stage 1: g1 = gt + dt L(gt)
            if (e == cudaSuccess) e = vjp_at(gt, l1, tmp);
            if (e == cudaSuccess) e = param_terms(gt, 1.0);
            if (e == cudaSuccess) e = launch_axpby_dt(P, n, 1.0, lt, 1.0, l1, tmp, dt, lam, st);
            // reconstruction (limiter) of this step
            if (e == cudaSuccess) e = launch_limiter_vjp(dg, pre, lam, n, st);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(lambda_0, lam, bytes, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_adjoint");
}

}  // extern "C"
