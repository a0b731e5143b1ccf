// C ABI of the GRACE-DG hot path: context, precompute, batches, RHS and SSP-RK3 stepping.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "grace_dual.cuh"
#include "grace_internal.h"
#include "grace_tc_layout.cuh"

namespace grace {

static thread_local std::string t_error;

void set_error(const std::string &msg) { t_error = msg; }

grace_status cuda_fail(cudaError_t e, const char *where)
{
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return GRACE_ERR_CUDA;
}

// Gauss-Legendre rule on [-1, 1] (eq. quad): Newton iterations on P_Q from the
// asymptotic guess cos(pi (4i + 3) / (4Q + 2)); ascending nodes.
void gauss_rule(int Q, double *s, double *w)
{
    const double pi = 3.141592653589793;
    for (int i = 0; i < Q; ++i) {
        double x = std::cos(pi * (4.0 * i + 3.0) / (4.0 * Q + 2.0));
        double pq = 0.0, pm = 0.0;
        for (int it = 0; it < 60; ++it) {
            double a = 1.0, b = x;   // P_0, P_1
            if (Q == 1) { pq = x; pm = 1.0; }
            for (int n = 2; n <= Q; ++n) {
                double c = ((2.0 * n - 1.0) * x * b - (n - 1.0) * a) / n;
                a = b;
                b = c;
            }
            if (Q >= 2) { pq = b; pm = a; }
            const double d = Q * (pm - x * pq) / ((1.0 - x) * (1.0 + x));
            const double step = pq / d;
            x -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        double a = 1.0, b = x;
        for (int n = 2; n <= Q; ++n) {
            double c = ((2.0 * n - 1.0) * x * b - (n - 1.0) * a) / n;
            a = b;
            b = c;
        }
        if (Q == 1) { b = x; a = 1.0; }
        const double d = Q * (a - x * b) / ((1.0 - x) * (1.0 + x));
        s[Q - 1 - i] = x;
        w[Q - 1 - i] = 2.0 / ((1.0 - x) * (1.0 + x) * d * d);
    }
}

int n_functionals(const grace_group_desc &d)
{
    const int n_if = d.flux_mode == GRACE_FLUX_CONSERVATIVE ? d.n_bins - 1 : d.n_bins;
    return n_if + d.n_bins * d.order_k;
}

// P(v < vth) for the Maxwellian of relative speeds with rms dv (Sec. 4.5); S = double, or Dual
// for its derivative along one parameter
template <class S>
static S maxwell_cdf_below(S vth, S dv)
{
    using std::erf;
    using std::exp;
    const double pi = 3.141592653589793;
    return erf(std::sqrt(1.5) * vth / dv) - vth * std::sqrt(6.0 / pi) / dv * exp(-1.5 * vth * vth / (dv * dv));
}

void maxwell_beta_derivs(const grace_group_desc &d, int id, double *dbeta_coag, double *dbeta_frag)
{
    *dbeta_coag = 0.0;
    *dbeta_frag = 0.0;
    if (d.coag_kind == GRACE_COAG_MAXWELL && (id == 0 || id == 1))
        *dbeta_coag = maxwell_cdf_below(Dual(d.coag_p[1], id == 1 ? 1.0 : 0.0), Dual(d.coag_p[0], id == 0 ? 1.0 : 0.0)).der;
    if (d.frag_kind == GRACE_FRAG_MAXWELL && (id == 8 || id == 9))
        *dbeta_frag = -maxwell_cdf_below(Dual(d.frag_p[1], id == 9 ? 1.0 : 0.0), Dual(d.frag_p[0], id == 8 ? 1.0 : 0.0)).der;
}

DevGroup make_devgroup(const grace_group_desc &d, const double *d_edges)
{
    DevGroup g;
    std::memset(&g, 0, sizeof(g));
    g.N = d.n_bins;
    g.k = d.order_k;
    g.K1 = d.order_k + 1;
    g.Q = d.quad_q > 0 ? d.quad_q : d.order_k + 1;
    g.P = g.N * g.K1;
    g.n_if = d.flux_mode == GRACE_FLUX_CONSERVATIVE ? g.N - 1 : g.N;
    g.R = n_functionals(d);
    g.flux_mode = d.flux_mode;
    g.coag_kind = d.coag_kind;
    g.frag_kind = d.frag_kind;
    g.break_kind = d.break_kind;
    g.cutoff_mode = d.cutoff_mode;
    g.mfrag_mode = d.mfrag_mode;
    g.limiter = d.limiter;
    g.has_delta = d.frag_kind != GRACE_FRAG_NONE && d.break_kind == GRACE_BREAK_POWERLAW_REMNANT;
    g.cell_alpha = d.cell_alpha;
    g.x_min = d.x_min;
    g.x_max = d.x_max;
    for (int i = 0; i < 8; ++i) {
        g.coag_p[i] = d.coag_p[i];
        g.frag_p[i] = d.frag_p[i];
        g.break_p[i] = d.break_p[i];
    }
    // beta_coag = P(v < v_b), beta_frag = P(v > v_f) for the Maxwellian of Sec. 4.5
    if (d.coag_kind == GRACE_COAG_MAXWELL) g.beta_coag = maxwell_cdf_below<double>(d.coag_p[1], d.coag_p[0]);
    if (d.frag_kind == GRACE_FRAG_MAXWELL) g.beta_frag = 1.0 - maxwell_cdf_below<double>(d.frag_p[1], d.frag_p[0]);
    gauss_rule(g.Q, g.gs, g.gw);
    g.edges = d_edges;
    g.hbin = d_edges ? d_edges + g.N + 1 : nullptr;
    g.inv_h = d_edges ? d_edges + 2 * g.N + 1 : nullptr;
    g.inv_h32 = d_edges ? reinterpret_cast<const float *>(d_edges + 3 * g.N + 1) : nullptr;
    g.h32 = d_edges ? reinterpret_cast<const float *>(d_edges + 3 * g.N + 1) + g.N : nullptr;
    return g;
}

static grace_status validate(const grace_group_desc &d, int idx)
{
    auto bad = [&](const char *why) {
        set_error("group " + std::to_string(idx) + ": " + why);
        return GRACE_ERR_ARG;
    };
    if (d.n_bins < 2 || d.n_bins > 4096) return bad("n_bins must be in [2, 4096]");
    if (d.order_k < 0) return bad("order_k must be >= 0");
    if (d.order_k > kKMax) {
        set_error("group " + std::to_string(idx) + ": order_k > 4 is not supported");
        return GRACE_ERR_UNSUPPORTED;
    }
    const int Q = d.quad_q > 0 ? d.quad_q : d.order_k + 1;
    if (d.quad_q < 0 || Q > kQMax) return bad("quad_q must be in [0, 16]");
    if (!(d.x_min > 0.0) || !(d.x_max > d.x_min) || !std::isfinite(d.x_max)) return bad("need 0 < x_min < x_max");
    if (d.flux_mode != GRACE_FLUX_CONSERVATIVE && d.flux_mode != GRACE_FLUX_NONCONSERVATIVE) return bad("flux_mode");
    if (d.coag_kind < GRACE_COAG_NONE || d.coag_kind > GRACE_COAG_BALLISTIC) return bad("coag_kind");
    if (d.frag_kind < GRACE_FRAG_NONE || d.frag_kind > GRACE_FRAG_BALLISTIC) return bad("frag_kind");
    if (d.break_kind < GRACE_BREAK_UNIFORM_BINARY || d.break_kind > GRACE_BREAK_COAG_DELTA) return bad("break_kind");
    if (d.coag_kind == GRACE_COAG_NONE && d.frag_kind == GRACE_FRAG_NONE) return bad("no collision kernel");
    if (d.cell_alpha != 0 && d.cell_alpha != 1) return bad("cell_alpha must be 0 or 1");
    if (d.cell_alpha) {
        if (d.coag_kind != GRACE_COAG_BALLISTIC) return bad("cell_alpha needs coag_kind BALLISTIC");
        if (d.order_k > 3) return bad("cell_alpha groups support order_k <= 3");
        if (d.frag_kind != GRACE_FRAG_NONE && d.frag_kind != GRACE_FRAG_BALLISTIC)
            return bad("cell_alpha needs frag_kind NONE or BALLISTIC");
        if (d.frag_kind == GRACE_FRAG_BALLISTIC)
            for (int i = 0; i < 7; ++i)
                if (i != 3 && d.frag_p[i] != d.coag_p[i])
                    return bad("cell_alpha: fragmentation must use the coagulation's ballistic parameters");
        if (!(d.coag_p[5] > 0.0) || !(d.coag_p[4] > 0.0)) return bad("cell_alpha: v_frag and the ramp width must be > 0");
    }
    if (d.coag_kind == GRACE_COAG_MAXWELL && !(d.coag_p[0] > 0.0)) return bad("Maxwellian dv_rms must be > 0");
    if (d.frag_kind == GRACE_FRAG_MAXWELL && !(d.frag_p[0] > 0.0)) return bad("Maxwellian dv_rms must be > 0");
    if (d.frag_kind != GRACE_FRAG_NONE && d.break_kind == GRACE_BREAK_POWERLAW_REMNANT && d.break_p[0] == -2.0)
        return bad("power-law index -2 is not supported");
    if (d.limiter != 0 && d.limiter != 1) return bad("limiter must be 0 or 1");
    if (d.edges) {
        if (d.edges[0] != d.x_min || d.edges[d.n_bins] != d.x_max)
            return bad("edges[0] and edges[n_bins] must equal x_min and x_max");
        for (int j = 0; j < d.n_bins; ++j)
            if (!(d.edges[j + 1] > d.edges[j]) || !std::isfinite(d.edges[j + 1]))
                return bad("edges must be finite and strictly increasing");
    }
    return GRACE_OK;
}

static void free_group(Group &G)
{
    free_nc_tables(G.nc);
    cudaFree(G.d_edges);
    cudaFree(G.d_T);
    cudaFree(G.d_qlo);
    cudaFree(G.d_qhi);
    cudaFree(G.d_prange);
    G.d_edges = nullptr;
    G.d_T = nullptr;
    G.d_qlo = G.d_qhi = G.d_prange = nullptr;
    for (auto &t : G.tc) free_tc_tiles(t);
    for (auto &t : G.tcv) free_tc_tiles(t);
    for (auto &t : G.tcs) free_tc_tiles(t);
    free_param_derivs(G);
}

__global__ void count_nnz_kernel(const double *T, size_t n, unsigned long long *out)
{
    unsigned long long c = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        c += T[i] != 0.0;
    atomicAdd(out, c);
}

}  // namespace grace

using namespace grace;

extern "C" {

int grace_version(void) { return 1; }

const char *grace_status_string(grace_status s)
{
    switch (s) {
    case GRACE_OK: return "ok";
    case GRACE_ERR_ARG: return "invalid argument";
    case GRACE_ERR_ORDER: return "call order violated";
    case GRACE_ERR_CUDA: return "CUDA error";
    case GRACE_ERR_NOMEM: return "out of memory";
    case GRACE_ERR_UNSUPPORTED: return "unsupported";
    case GRACE_ERR_TIMEOUT: return "device wait timed out";
    case GRACE_WARN_CELLS: return "some cells have status bits set";
    default: return "unknown status";
    }
}

const char *grace_last_error(void) { return t_error.c_str(); }

grace_status grace_setup(grace_ctx **out, int n_groups, const grace_group_desc *groups, int device)
{
    try {
        t_error.clear();
        if (!out || n_groups < 1 || !groups) {
            set_error("grace_setup: null output, no groups or null group array");
            return GRACE_ERR_ARG;
        }
        *out = nullptr;
        for (int i = 0; i < n_groups; ++i) {
            grace_status s = validate(groups[i], i);
            if (s != GRACE_OK) return s;
        }
        if (device < 0) {
            set_error("grace_setup: negative device index");
            return GRACE_ERR_ARG;
        }
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
        if (device >= ndev) {
            set_error("grace_setup: no such CUDA device");
            return GRACE_ERR_ARG;
        }
        Guard guard(device);
        grace_ctx *ctx = new grace_ctx();
        ctx->device = device;
        ctx->groups.resize(n_groups);
        for (int i = 0; i < n_groups; ++i) {
            Group &G = ctx->groups[i];
            G.desc = groups[i];
            G.desc.edges = nullptr;   // the caller's array is copied, not kept
            const int N = G.desc.n_bins;
            G.h_edges.resize(N + 1);
            if (groups[i].edges) {
                for (int j = 0; j <= N; ++j) G.h_edges[j] = groups[i].edges[j];
            } else {
                // logarithmic grid of Sec. 3.1
                for (int j = 0; j <= N; ++j)
                    G.h_edges[j] = G.desc.x_min * std::pow(G.desc.x_max / G.desc.x_min, (double)j / N);
                G.h_edges[0] = G.desc.x_min;
                G.h_edges[N] = G.desc.x_max;
            }
            // one allocation: edges (N+1), h (N), 1/h (N) in FP64, then 1/h (N) and h (N) in FP32
            std::vector<double> tab(3 * (size_t)N + 1 + N, 0.0);
            for (int j = 0; j <= N; ++j) tab[j] = G.h_edges[j];
            for (int j = 0; j < N; ++j) {
                const double h = G.h_edges[j + 1] - G.h_edges[j];
                tab[N + 1 + j] = h;
                tab[2 * N + 1 + j] = 1.0 / h;
                reinterpret_cast<float *>(tab.data() + 3 * N + 1)[j] = (float)(1.0 / h);
                reinterpret_cast<float *>(tab.data() + 3 * N + 1)[N + j] = (float)h;
            }
            e = cudaMalloc(&G.d_edges, sizeof(double) * tab.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(G.d_edges, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                grace_destroy(ctx);
                return cuda_fail(e, "grace_setup: edges");
            }
            G.dg = make_devgroup(G.desc, G.d_edges);
        }
        *out = ctx;
        return GRACE_OK;
    } catch (const std::bad_alloc &) {
        set_error("grace_setup: host allocation failed");
        return GRACE_ERR_NOMEM;
    } catch (...) {
        set_error("grace_setup: unexpected exception");
        return GRACE_ERR_ARG;
    }
}

grace_status grace_set_stream(grace_ctx *ctx, void *stream)
{
    if (!ctx) {
        set_error("grace_set_stream: null context");
        return GRACE_ERR_ARG;
    }
    ctx->stream = (cudaStream_t)stream;
    return GRACE_OK;
}

// A lower bound of the shared memory a contraction launch over tiles t needs: the A tile of 128
// cells, a 2-deep ring of the smallest B copies (one k-step of the widest tile) and the barrier
// block.  Tiles that cannot fit it in a block's 227 KB could never launch, so they are refused here.
static grace_status check_tc_fits(const TcTiles &t, int prec, int group)
{
    if (!t.built || t.n_tiles == 0) return GRACE_OK;
    const size_t planes = prec == GRACE_TF32 ? 1 : 2;
    const size_t slot = ((size_t)t.max_rows * 32 * planes + 1023) / 1024 * 1024;
    const size_t need = 1024 + 64 + opA_tile_bytes(prec, t.k_pad) + 2 * slot;
    if (need <= (size_t)227 * 1024) return GRACE_OK;
    set_error("grace_precompute: group " + std::to_string(group) + " has " + std::to_string(t.k_pad) +
              " padded coefficients per cell, too many for a tensor-core A tile in shared memory; "
              "use GRACE_FP64 for it");
    return GRACE_ERR_UNSUPPORTED;
}

grace_status grace_precompute(grace_ctx *ctx, unsigned mask)
{
    try {
        if (!ctx) {
            set_error("grace_precompute: null context");
            return GRACE_ERR_ARG;
        }
        Guard guard(ctx->device);
        cudaStream_t st = ctx->stream;
        for (Group &G : ctx->groups) {
            const DevGroup &g = G.dg;
            if (g.cell_alpha) {
                // per-cell kernel: no fixed T exists; node-space tables.
                // nnz reports the multiply-adds of one RHS per cell: the non-zeros of the
                // two tables plus 2 (k+1) + 2 per partial entry
                if (!G.nc.built) {
                    grace_status s = build_nc_tables(G, st);
                    if (s != GRACE_OK) return s;
                    const size_t nt = (size_t)g.R * G.nc.NQ * G.nc.NQ;
                    unsigned long long *d_cnt = nullptr, cnt = 0;
                    cudaError_t e = cudaMalloc(&d_cnt, sizeof(unsigned long long));
                    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
                    if (e == cudaSuccess) {
                        count_nnz_kernel<<<256, 256, 0, st>>>(G.nc.d_Cc, nt, d_cnt);
                        count_nnz_kernel<<<256, 256, 0, st>>>(G.nc.d_Cf, nt, d_cnt);
                        e = cudaGetLastError();
                    }
                    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                    cudaFree(d_cnt);
                    if (e != cudaSuccess) return cuda_fail(e, "grace_precompute: node-space tables");
                    G.nnz = (long long)cnt + G.nc.n_entries * (2LL * g.K1 + 2);
                }
                // reduced-precision forms: tensor-core tiles of the fixed part, FP32 partial entries
                for (int prec = GRACE_TF32; prec <= GRACE_BF16X3; ++prec) {
                    if (!(mask & (1u << prec)) || G.tc[prec].built) continue;
                    grace_status s = build_nc_tc_entries(G, st);
                    if (s == GRACE_OK) s = build_nc_tc_tiles(G, prec, st);
                    if (s == GRACE_OK) s = check_tc_fits(G.tc[prec], prec, (int)(&G - ctx->groups.data()));
                    if (s != GRACE_OK) return s;
                }
                continue;
            }
            if (!G.d_T) {
                const size_t nT = (size_t)g.R * g.P * g.P;
                cudaError_t e = cudaMalloc(&G.d_T, nT * sizeof(double));
                if (e == cudaSuccess) e = cudaMalloc(&G.d_qlo, sizeof(int) * g.R * g.P);
                if (e == cudaSuccess) e = cudaMalloc(&G.d_qhi, sizeof(int) * g.R * g.P);
                if (e == cudaSuccess) e = cudaMalloc(&G.d_prange, sizeof(int) * 2 * g.R);
                if (e != cudaSuccess) {
                    free_group(G);
                    cudaGetLastError();
                    set_error(std::string("grace_precompute: allocation: ") + cudaGetErrorString(e));
                    return GRACE_ERR_NOMEM;
                }
                e = launch_build_T(g, G.d_T, st);
                if (e == cudaSuccess) e = launch_row_extents(g, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, st);
                unsigned long long *d_cnt = nullptr;
                if (e == cudaSuccess) e = cudaMalloc(&d_cnt, sizeof(unsigned long long));
                if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
                if (e == cudaSuccess) {
                    count_nnz_kernel<<<256, 256, 0, st>>>(G.d_T, nT, d_cnt);
                    e = cudaGetLastError();
                }
                unsigned long long cnt = 0;
                if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                cudaFree(d_cnt);
                if (e != cudaSuccess) return cuda_fail(e, "grace_precompute: T build");
                G.nnz = (long long)cnt;
            }
            for (int prec = GRACE_TF32; prec <= GRACE_BF16X3; ++prec) {
                if (!(mask & (1u << prec)) || G.tc[prec].built) continue;
                grace_status s = build_tc_tiles(G, prec, st);
                if (s == GRACE_OK) s = check_tc_fits(G.tc[prec], prec, (int)(&G - ctx->groups.data()));
                if (s != GRACE_OK) return s;
            }
        }
        ctx->precomputed = 1;
        ctx->precision_mask |= mask | 1u;
        return GRACE_OK;
    } catch (const std::bad_alloc &) {
        set_error("grace_precompute: host allocation failed");
        return GRACE_ERR_NOMEM;
    } catch (...) {
        set_error("grace_precompute: unexpected exception");
        return GRACE_ERR_ARG;
    }
}

grace_status grace_group_info(const grace_ctx *ctx, int group, int *n_coef, int *n_func)
{
    if (!ctx || group < 0 || group >= (int)ctx->groups.size()) {
        set_error("grace_group_info: bad context or group");
        return GRACE_ERR_ARG;
    }
    if (n_coef) *n_coef = ctx->groups[group].dg.P;
    if (n_func) *n_func = ctx->groups[group].dg.R;
    return GRACE_OK;
}

grace_status grace_profile_enable(grace_ctx *ctx, int enable)
{
    if (!ctx) {
        set_error("grace_profile_enable: null context");
        return GRACE_ERR_ARG;
    }
    ctx->profiling = enable ? 1 : 0;
    return GRACE_OK;
}

grace_status grace_profile_read(grace_ctx *ctx, int kernel, double *total_ms, long long *launches)
{
    if (!ctx || kernel < 0 || kernel > 2) {
        set_error("grace_profile_read: bad context or kernel index");
        return GRACE_ERR_ARG;
    }
    Guard guard(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "grace_profile_read");
    double tot = 0.0;
    for (auto &pr : ctx->ev_pairs[kernel]) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess) return cuda_fail(e, "grace_profile_read: elapsed");
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (long long)ctx->ev_pairs[kernel].size();
    ctx->ev_pairs[kernel].clear();
    if (ctx->ev_pairs[0].empty() && ctx->ev_pairs[1].empty() && ctx->ev_pairs[2].empty()) ctx->ev_used = 0;
    return GRACE_OK;
}

grace_status grace_group_stats(const grace_ctx *ctx, int group, int prec, long long *nnz, long long *tile_macs)
{
    if (!ctx || group < 0 || group >= (int)ctx->groups.size() || prec < 0 || prec > 2) {
        set_error("grace_group_stats: bad argument");
        return GRACE_ERR_ARG;
    }
    const Group &G = ctx->groups[group];
    if (nnz) *nnz = G.nnz;
    if (tile_macs) *tile_macs = prec == GRACE_FP64 ? G.nnz : G.tc[prec].mac_per_cell;
    return GRACE_OK;
}

grace_status grace_tile_info(const grace_ctx *ctx, int group, int prec, long long *info)
{
    if (!ctx || !info || group < 0 || group >= (int)ctx->groups.size() || (prec != GRACE_TF32 && prec != GRACE_BF16X3)) {
        set_error("grace_tile_info: bad argument");
        return GRACE_ERR_ARG;
    }
    if (!ctx->groups[group].tc[prec].built) {
        set_error("grace_tile_info: precision not precomputed");
        return GRACE_ERR_ORDER;
    }
    const TcTiles &t = tc_forward_tiles(ctx->groups[group].tc[prec]);
    info[0] = t.n_tiles;
    info[1] = t.mma_per_tile;
    info[2] = t.mac_per_cell;
    info[3] = (long long)t.b_bytes;
    info[4] = (long long)(t.pred_clk + 0.5);
    info[5] = t.max_rows;
    info[6] = t.nnz_fold;
    info[7] = t.folded;
    return GRACE_OK;
}

void grace_destroy(grace_ctx *ctx)
{
    if (!ctx) return;
    Guard guard(ctx->device);
    for (Group &G : ctx->groups) free_group(G);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
}

}  // extern "C"
