// C ABI of the GRACE-DG hot path: context, precompute, batches, RHS and SSP-RK3 stepping.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

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

static double maxwell_cdf_below(double vth, double dv)
{
    const double pi = 3.141592653589793;
    return std::erf(std::sqrt(1.5) * vth / dv) - vth * std::sqrt(6.0 / pi) / dv * std::exp(-1.5 * vth * vth / (dv * dv));
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
    g.x_min = d.x_min;
    g.x_max = d.x_max;
    for (int i = 0; i < 8; ++i) {
        g.coag_p[i] = d.coag_p[i];
        g.frag_p[i] = d.frag_p[i];
        g.break_p[i] = d.break_p[i];
    }
    // beta_coag = P(v < v_b), beta_frag = P(v > v_f) for the Maxwellian of Sec. 4.5
    if (d.coag_kind == GRACE_COAG_MAXWELL) g.beta_coag = maxwell_cdf_below(d.coag_p[1], d.coag_p[0]);
    if (d.frag_kind == GRACE_FRAG_MAXWELL) g.beta_frag = 1.0 - maxwell_cdf_below(d.frag_p[1], d.frag_p[0]);
    gauss_rule(g.Q, g.gs, g.gw);
    g.edges = d_edges;
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
        set_error("group " + std::to_string(idx) + ": order_k > 3 is not supported by this build");
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
    if (d.coag_kind == GRACE_COAG_MAXWELL && !(d.coag_p[0] > 0.0)) return bad("Maxwellian dv_rms must be > 0");
    if (d.frag_kind == GRACE_FRAG_MAXWELL && !(d.frag_p[0] > 0.0)) return bad("Maxwellian dv_rms must be > 0");
    if (d.frag_kind != GRACE_FRAG_NONE && d.break_kind == GRACE_BREAK_POWERLAW_REMNANT && d.break_p[0] == -2.0)
        return bad("power-law index -2 is not supported");
    if (d.limiter != 0 && d.limiter != 1) return bad("limiter must be 0 or 1");
    return GRACE_OK;
}

struct Guard {   // switches to the context's device for the duration of a call
    int prev = -1;
    explicit Guard(int dev)
    {
        cudaGetLastError();   // a stale error of an earlier, unrelated call must not be reported as ours
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard()
    {
        int cur;
        if (cudaGetDevice(&cur) == cudaSuccess && prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

static void free_group(Group &G)
{
    cudaFree(G.d_edges);
    cudaFree(G.d_T);
    cudaFree(G.d_qlo);
    cudaFree(G.d_qhi);
    cudaFree(G.d_prange);
    G.d_edges = nullptr;
    G.d_T = nullptr;
    G.d_qlo = G.d_qhi = G.d_prange = nullptr;
    for (auto &t : G.tc) free_tc_tiles(t);
}

__global__ void count_nnz_kernel(const double *T, size_t n, unsigned long long *out)
{
    unsigned long long c = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        c += T[i] != 0.0;
    atomicAdd(out, c);
}

// events around one launch when profiling is enabled
struct LaunchTimer {
    grace_ctx *ctx;
    int kind;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchTimer(grace_ctx *c, int k) : ctx(c), kind(k)
    {
        if (!ctx->profiling) return;
        while (ctx->ev_pool.size() < ctx->ev_used + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            ctx->ev_pool.push_back(e);
        }
        a = ctx->ev_pool[ctx->ev_used++];
        b = ctx->ev_pool[ctx->ev_used++];
        cudaEventRecord(a, ctx->stream);
    }
    ~LaunchTimer()
    {
        if (!a) return;
        cudaEventRecord(b, ctx->stream);
        ctx->ev_pairs[kind].push_back({a, b});
    }
};

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
            const int N = G.desc.n_bins;
            G.h_edges.resize(N + 1);
            // logarithmic grid of Sec. 3.1
            for (int j = 0; j <= N; ++j)
                G.h_edges[j] = G.desc.x_min * std::pow(G.desc.x_max / G.desc.x_min, (double)j / N);
            G.h_edges[0] = G.desc.x_min;
            G.h_edges[N] = G.desc.x_max;
            e = cudaMalloc(&G.d_edges, sizeof(double) * (N + 1));
            if (e == cudaSuccess)
                e = cudaMemcpy(G.d_edges, G.h_edges.data(), sizeof(double) * (N + 1), cudaMemcpyHostToDevice);
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

grace_status grace_bind_batch(grace_ctx *ctx, int n_cells, const int *cell_group, grace_batch **out)
{
    try {
        if (!ctx || !out || n_cells < 1) {
            set_error("grace_bind_batch: null context/output or n_cells < 1");
            return GRACE_ERR_ARG;
        }
        *out = nullptr;
        if (!ctx->precomputed) {
            set_error("grace_bind_batch: call grace_precompute first");
            return GRACE_ERR_ORDER;
        }
        Guard guard(ctx->device);
        grace_batch *b = new grace_batch();
        b->ctx = ctx;
        b->n_cells = n_cells;
        b->h_group.assign(n_cells, 0);
        if (cell_group) {
            for (int c = 0; c < n_cells; ++c) {
                if (cell_group[c] < 0 || cell_group[c] >= (int)ctx->groups.size()) {
                    delete b;
                    set_error("grace_bind_batch: cell group out of range");
                    return GRACE_ERR_ARG;
                }
                b->h_group[c] = cell_group[c];
                if (cell_group[c] != 0) b->single_group = 0;
            }
        }
        if (!b->single_group) {
            delete b;
            set_error("grace_bind_batch: batches mixing groups are not supported by this build");
            return GRACE_ERR_UNSUPPORTED;
        }
        const DevGroup &g = ctx->groups[0].dg;
        b->h_off.resize(n_cells + 1);
        for (int c = 0; c <= n_cells; ++c) b->h_off[c] = (long long)c * g.P;
        const size_t n = (size_t)n_cells;
        cudaError_t e = cudaMalloc(&b->d_F, n * g.R * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_g1, n * g.P * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_g2, n * g.P * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
        if (e == cudaSuccess && (ctx->precision_mask & ((1u << GRACE_TF32) | (1u << GRACE_BF16X3)))) {
            e = cudaMalloc(&b->d_F32, n * g.R * sizeof(float));
            if (e == cudaSuccess) e = cudaMemset(b->d_F32, 0, n * g.R * sizeof(float));
            size_t bytes = 0;
            for (int prec = GRACE_TF32; prec <= GRACE_BF16X3; ++prec)
                if (ctx->precision_mask & (1u << prec)) {
                    int kpad = 0;
                    size_t s = opA_bytes_for(g, prec, n_cells, &kpad);
                    if (s > bytes) bytes = s;
                }
            if (e == cudaSuccess) e = cudaMalloc(&b->d_opA, bytes);
            if (e == cudaSuccess) e = cudaMemset(b->d_opA, 0, bytes);
            b->opA_bytes = bytes;
        }
        if (e != cudaSuccess) {
            grace_batch_destroy(b);
            cudaGetLastError();
            set_error(std::string("grace_bind_batch: allocation: ") + cudaGetErrorString(e));
            return GRACE_ERR_NOMEM;
        }
        *out = b;
        return GRACE_OK;
    } catch (const std::bad_alloc &) {
        set_error("grace_bind_batch: host allocation failed");
        return GRACE_ERR_NOMEM;
    } catch (...) {
        set_error("grace_bind_batch: unexpected exception");
        return GRACE_ERR_ARG;
    }
}

grace_status grace_batch_offsets(const grace_batch *b, long long *out)
{
    if (!b || !out) {
        set_error("grace_batch_offsets: null argument");
        return GRACE_ERR_ARG;
    }
    std::memcpy(out, b->h_off.data(), sizeof(long long) * (b->n_cells + 1));
    return GRACE_OK;
}

static grace_status check_prec(grace_batch *b, int prec)
{
    if (prec < GRACE_FP64 || prec > GRACE_BF16X3) {
        set_error("unknown precision");
        return GRACE_ERR_ARG;
    }
    if (prec != GRACE_FP64 && !b->ctx->groups[0].tc[prec].built) {
        set_error("precision not precomputed: pass its bit to grace_precompute before binding the batch");
        return GRACE_ERR_ORDER;
    }
    if (prec != GRACE_FP64 && !b->d_opA) {
        set_error("batch bound before the tensor-core precompute");
        return GRACE_ERR_ORDER;
    }
    return GRACE_OK;
}

// F <- functionals of g (FP64 path) or of the packed A operand (tensor path)
static grace_status contract(grace_batch *b, const double *g, int prec, UpdateArgs &u)
{
    Group &G = b->ctx->groups[0];
    cudaStream_t st = b->ctx->stream;
    cudaError_t e;
    LaunchTimer timer(b->ctx, 0);
    if (prec == GRACE_FP64) {
        e = launch_contract_fp64(G.dg, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, g, b->n_cells, b->d_F, st);
        u.F = b->d_F;
        u.F32 = nullptr;
    } else {
        e = launch_contract_tc(G.dg, G.tc[prec], prec, b->d_opA, b->n_cells, b->d_F32, b->d_err, st);
        u.F = nullptr;
        u.F32 = b->d_F32;
    }
    if (e != cudaSuccess) return cuda_fail(e, "contraction launch");
    return GRACE_OK;
}

grace_status grace_rhs(grace_batch *b, const double *g, double *L, int prec)
{
    if (!b || !g || !L) {
        set_error("grace_rhs: null argument");
        return GRACE_ERR_ARG;
    }
    grace_status s = check_prec(b, prec);
    if (s != GRACE_OK) return s;
    Guard guard(b->ctx->device);
    Group &G = b->ctx->groups[0];
    cudaStream_t st = b->ctx->stream;
    if (prec != GRACE_FP64) {
        cudaError_t e = launch_pack_A(G.dg, g, b->n_cells, b->d_opA, prec, G.tc[prec].k_pad, st);
        if (e != cudaSuccess) return cuda_fail(e, "grace_rhs: operand pack");
    }
    UpdateArgs u;
    s = contract(b, g, prec, u);
    if (s != GRACE_OK) return s;
    u.gout = L;
    cudaError_t e;
    {
        LaunchTimer timer(b->ctx, 1);
        e = launch_update(G.dg, u, b->n_cells, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "grace_rhs: update");
    return GRACE_OK;
}

grace_status grace_step(grace_batch *b, double *g, const double *dt, int n_steps, int prec, double *mass,
                        unsigned char *flags)
{
    if (!b || !g || !dt || n_steps < 0) {
        set_error("grace_step: null argument or negative step count");
        return GRACE_ERR_ARG;
    }
    grace_status s = check_prec(b, prec);
    if (s != GRACE_OK) return s;
    Guard guard(b->ctx->device);
    Group &G = b->ctx->groups[0];
    const DevGroup &dg = G.dg;
    cudaStream_t st = b->ctx->stream;
    const int n = b->n_cells;
    const bool tc = prec != GRACE_FP64;
    const int kpad = tc ? G.tc[prec].k_pad : 0;
    void *opA = tc ? b->d_opA : nullptr;
    cudaError_t e = cudaSuccess;
    if (flags) e = cudaMemsetAsync(flags, 0, n, st);
    if (e != cudaSuccess) return cuda_fail(e, "grace_step: flags");
    if (n_steps == 0) {
        if (mass) {
            e = launch_mass(dg, g, n, mass, st);
            if (e != cudaSuccess) return cuda_fail(e, "grace_step: mass");
        }
        return GRACE_OK;
    }
    // reconstruction of the first step (Sec. 3.2.2); later ones are fused into stage 3
    if (dg.limiter || tc) {
        DevGroup d0 = dg;
        e = launch_limit(d0, g, n, flags, opA, prec, kpad, st);
        if (e != cudaSuccess) return cuda_fail(e, "grace_step: limiter");
    }
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int step = 0; step < n_steps; ++step) {
        const bool last = step == n_steps - 1;
        const double *gin[3] = {g, b->d_g1, b->d_g2};
        double *gout[3] = {b->d_g1, b->d_g2, g};
        for (int stage = 0; stage < 3; ++stage) {
            UpdateArgs u;
            s = contract(b, gin[stage], prec, u);
            if (s != GRACE_OK) return s;
            u.gn = g;
            u.gs = gin[stage];
            u.gout = gout[stage];
            u.dt = dt;
            u.a = ca[stage];
            u.b = cb[stage];
            u.flags = flags;
            if (stage == 2) {
                u.apply_limiter = (!last && dg.limiter) ? 1 : 0;
                u.mass = last ? mass : nullptr;
            }
            if (tc && !(stage == 2 && last)) {
                u.opA = opA;
                u.opA_prec = prec;
                u.opA_kpad = kpad;
            }
            {
                LaunchTimer timer(b->ctx, 1);
                e = launch_update(dg, u, n, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "grace_step: update");
        }
    }
    return GRACE_OK;
}

grace_status grace_mass(grace_batch *b, const double *g, double *mass)
{
    if (!b || !g || !mass) {
        set_error("grace_mass: null argument");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    cudaError_t e = launch_mass(b->ctx->groups[0].dg, g, b->n_cells, mass, b->ctx->stream);
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_mass");
}

grace_status grace_limit(grace_batch *b, double *g, unsigned char *flags)
{
    if (!b || !g) {
        set_error("grace_limit: null argument");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    cudaError_t e = cudaSuccess;
    if (flags) e = cudaMemsetAsync(flags, 0, b->n_cells, b->ctx->stream);
    if (e == cudaSuccess) e = launch_limit(b->ctx->groups[0].dg, g, b->n_cells, flags, nullptr, 0, 0, b->ctx->stream);
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_limit");
}

grace_status grace_project(grace_batch *b, int ic_kind, const double *ic_params, double *g)
{
    if (!b || !ic_params || !g || ic_kind < GRACE_IC_EXP || ic_kind > GRACE_IC_FIRST_BIN) {
        set_error("grace_project: bad argument");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    cudaError_t e = launch_project(b->ctx->groups[0].dg, ic_kind, ic_params, b->n_cells, g, b->ctx->stream);
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_project");
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
    if (!ctx || kernel < 0 || kernel > 1) {
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
    if (ctx->ev_pairs[0].empty() && ctx->ev_pairs[1].empty()) ctx->ev_used = 0;
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

grace_status grace_batch_error(grace_batch *b, int *code)
{
    if (!b) {
        set_error("grace_batch_error: null batch");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "grace_batch_error");
    if (code) *code = h;
    if (h) {
        set_error("a bounded device wait timed out (code " + std::to_string(h) + ")");
        return GRACE_ERR_TIMEOUT;
    }
    return GRACE_OK;
}

void grace_batch_destroy(grace_batch *b)
{
    if (!b) return;
    Guard guard(b->ctx->device);
    cudaFree(b->d_F);
    cudaFree(b->d_F32);
    cudaFree(b->d_g1);
    cudaFree(b->d_g2);
    cudaFree(b->d_opA);
    cudaFree(b->d_flags);
    cudaFree(b->d_err);
    delete b;
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
