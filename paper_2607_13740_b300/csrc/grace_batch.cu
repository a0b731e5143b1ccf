// Batches: binding, per-group parts, RHS, SSP-RK3 stepping, mass, limiter,
// projection, device error word and CUDA-graph replay of grace_step.
//
// A batch may mix cells of several groups (different N, k or physics) in any
// order.  Cells are partitioned by group into parts; each part gathers its
// cells' rows from the caller's packed layout into contiguous workspaces, runs
// the group's kernels on its own stream (parts overlap on the GPU), and
// scatters results back.  A batch whose cells all belong to one group in the
// caller's order is a single direct part that works on the caller's arrays.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "grace_internal.h"
#include "grace_tc_layout.cuh"

namespace grace {
namespace {

__global__ void gather_rows_kernel(int n, int P, const long long *off, const double *src, double *dst)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * P) return;
    const long long c = t / P;
    dst[t] = src[off[c] + (t - c * P)];
}

__global__ void scatter_rows_kernel(int n, int P, const long long *off, const double *src, double *dst)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * P) return;
    const long long c = t / P;
    dst[off[c] + (t - c * P)] = src[t];
}

// ---------------------------------------------------------------- grouped (one launch per batch)
// one part of a grouped gather / scatter: its first element (state doubles) and first cell in the
// grouped index spaces, its rows' offsets in the caller's arrays and its workspaces
struct MovePart {
    long long elem0, cell0;
    int n, P;
    const long long *off;
    const int *idx;
    double *g, *dt, *mass;
    unsigned char *flags;
};

__device__ __forceinline__ int find_part(const MovePart *m, int np, long long t, bool by_elem)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((by_elem ? m[mid].elem0 : m[mid].cell0) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// state rows: caller -> parts (scatter = 0) or parts -> caller (scatter = 1)
__global__ void grouped_rows_kernel(const MovePart *__restrict__ m, int np, long long total, const double *src,
                                    double *dst, int scatter)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const MovePart &p = m[find_part(m, np, t, true)];
    const long long e = t - p.elem0, c = e / p.P;
    const long long o = p.off[c] + (e - c * p.P);
    if (scatter) dst[o] = p.g[e];
    else p.g[e] = src[o];
}

// per-cell arrays: before the step dt -> parts and the parts' flags cleared (mode 0); after it
// the parts' mass and flags -> caller (mode 1)
__global__ void grouped_cells_kernel(const MovePart *__restrict__ m, int np, long long total, const double *dt,
                                     double *mass, unsigned char *flags, int mode)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const MovePart &p = m[find_part(m, np, t, false)];
    const long long c = t - p.cell0;
    const int ci = p.idx[c];
    if (mode == 0) {
        p.dt[c] = dt[ci];
        p.flags[c] = 0;
    } else {
        if (mass) mass[ci] = p.mass[c];
        if (flags) flags[ci] = p.flags[c];
    }
}

template <typename T>
__global__ void gather_kernel(int n, int w, const int *idx, const T *src, T *dst)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * w) return;
    const long long c = t / w;
    dst[t] = src[(long long)idx[c] * w + (t - c * w)];
}

template <typename T>
__global__ void scatter_kernel(int n, const int *idx, const T *src, T *dst)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[idx[t]] = src[t];
}

inline unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

cudaStream_t part_stream(const grace_batch *b, const Part &p) { return p.direct ? b->ctx->stream : p.stream; }

void free_part(Part &p)
{
    cudaFree(p.d_idx);
    cudaFree(p.d_off);
    cudaFree(p.d_g);
    cudaFree(p.d_out);
    cudaFree(p.d_dt);
    cudaFree(p.d_mass);
    cudaFree(p.d_flags);
    cudaFree(p.d_ic);
    cudaFree(p.d_F);
    cudaFree(p.d_F32);
    cudaFree(p.d_g1);
    cudaFree(p.d_g2);
    cudaFree(p.d_opA);
    cudaFree(p.d_mx);
    cudaFree(p.d_alpha);
    cudaFree(p.d_G);
    cudaFree(p.d_H);
    cudaFree(p.d_gh);
    cudaFree(p.d_s);
    cudaFree(p.d_W32);
    cudaFree(p.d_mu32);
    cudaFree(p.d_cscale);
    cudaFree(p.d_gamma);
    cudaFree(p.d_F2);
    cudaFree(p.d_eps);
    if (p.stream) cudaStreamDestroy(p.stream);
    if (p.done) cudaEventDestroy(p.done);
    p = Part();
}

grace_status check_prec(grace_batch *b, int prec)
{
    if (prec < GRACE_FP64 || prec > GRACE_BF16X3) {
        set_error("unknown precision");
        return GRACE_ERR_ARG;
    }
    for (const Part &p : b->parts) {
        if (b->ctx->groups[p.group].dg.cell_alpha && !b->alpha_set) {
            set_error("per-cell kernel parameters not set: call grace_batch_cell_params first");
            return GRACE_ERR_ORDER;
        }
        if (prec != GRACE_FP64 && !b->ctx->groups[p.group].tc[prec].built) {
            set_error("precision not precomputed: pass its bit to grace_precompute before binding the batch");
            return GRACE_ERR_ORDER;
        }
        if (prec != GRACE_FP64 && !p.d_opA) {
            set_error("batch bound before the tensor-core precompute");
            return GRACE_ERR_ORDER;
        }
    }
    return GRACE_OK;
}

// ------------------------------------------------------------------ per-part compute
// flux functionals of a per-cell kernel group in a reduced-precision form, into p.d_F32
cudaError_t nc_tc_functionals(grace_batch *b, Group &G, Part &p, int prec, const double *g, cudaStream_t st)
{
    const TcTiles &t = G.tc[prec];
    cudaError_t e;
    {
        LaunchTimer timer(b->ctx, 2, st);
        e = launch_nc_pack_tc(G.dg, t, prec, g, p.d_alpha, p.n, p.d_opA, p.d_gh, p.d_s, st);
    }
    if (e != cudaSuccess) return e;
    {
        LaunchTimer timer(b->ctx, 0, st);
        e = launch_contract_tc(G.dg, t, prec, p.d_opA, p.n, p.d_F32, b->d_err, st, p.d_s);
    }
    if (e != cudaSuccess) return e;
    LaunchTimer timer(b->ctx, 2, st);
    return launch_nc_partial_tc(G.dg, G.nc, t, p.n, p.d_gh, p.d_s, p.d_F32, st);
}

cudaError_t part_rhs(grace_batch *b, Part &p, const double *g, double *L, int prec)
{
    Group &G = b->ctx->groups[p.group];
    cudaStream_t st = part_stream(b, p);
    cudaError_t e;
    if (prec != GRACE_FP64) {
        if (G.dg.cell_alpha) {
            e = nc_tc_functionals(b, G, p, prec, g, st);
        } else {
            e = launch_pack_A(G.dg, g, p.n, p.d_opA, prec, G.tc[prec].k_pad, G.tc[prec].k_ofs, st);
            if (e != cudaSuccess) return e;
            LaunchTimer timer(b->ctx, 0, st);
            e = launch_contract_tc(G.dg, G.tc[prec], prec, p.d_opA, p.n, p.d_F32, b->d_err, st);
        }
        if (e != cudaSuccess) return e;
        UpdateArgs u;
        u.F32 = p.d_F32;
        u.gout = L;
        LaunchTimer timer(b->ctx, 1, st);
        return launch_update_tc(G.dg, u, p.n, st);
    }
    {
        LaunchTimer timer(b->ctx, 0, st);
        e = G.dg.cell_alpha ? launch_nc_functionals(G.dg, G.nc, g, p.d_alpha, p.n, p.d_G, p.d_H, p.d_F, st)
                            : launch_contract_fp64(G.dg, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, g, p.n, p.d_F, st);
    }
    if (e != cudaSuccess) return e;
    UpdateArgs u;
    u.F = p.d_F;
    u.gout = L;
    LaunchTimer timer(b->ctx, 1, st);
    return launch_update(G.dg, u, p.n, st);
}

cudaError_t part_step(grace_batch *b, Part &p, double *g, const double *dt, int n_steps, int prec, double *mass,
                      unsigned char *flags)
{
    Group &G = b->ctx->groups[p.group];
    const DevGroup &dg = G.dg;
    cudaStream_t st = part_stream(b, p);
    const int n = p.n;
    const bool tc = prec != GRACE_FP64;
    const int kpad = tc ? G.tc[prec].k_pad : 0, kofs = tc ? G.tc[prec].k_ofs : 0;
    void *opA = tc ? p.d_opA : nullptr;
    cudaError_t e = cudaSuccess;
    if (flags) e = cudaMemsetAsync(flags, 0, n, st);
    if (e != cudaSuccess) return e;
    if (n_steps == 0) return mass ? launch_mass(dg, g, n, mass, st) : cudaSuccess;
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    if (tc && dg.cell_alpha) {
        // Per-cell kernels, reduced-precision forms: FP64 stage rows (the contraction dominates,
        // so the compact layout buys nothing here); functionals from nc_tc_functionals, FP32 K-c.
        if (dg.limiter) {
            e = launch_limit(dg, g, n, flags, nullptr, 0, 0, 0, st);
            if (e != cudaSuccess) return e;
        }
        for (int step = 0; step < n_steps; ++step) {
            const bool last = step == n_steps - 1;
            const double *gin[3] = {g, p.d_g1, p.d_g2};
            double *gout[3] = {p.d_g1, p.d_g2, g};
            for (int stage = 0; stage < 3; ++stage) {
                e = nc_tc_functionals(b, G, p, prec, gin[stage], st);
                if (e != cudaSuccess) return e;
                UpdateArgs u;
                u.F32 = p.d_F32;
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
                LaunchTimer timer(b->ctx, 1, st);
                e = launch_update_tc(dg, u, n, st);
                if (e != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    }
    if (tc) {
        // Tensor path.  Inside the call the state lives in the compact stage layout (FP64
        // means, FP32 higher modes): X[0] = g^n, X[1] = g^(1), X[2] = g^(2).  The step-start
        // limiter (Sec. 3.2.2) converts the caller's rows into X[0] and writes the A operand;
        // later reconstructions are fused into stage 3, and the last stage writes the
        // caller's FP64 rows.
        const size_t xs = (mixed_bytes_for(dg, n) + 15) / 16 * 2;   // doubles per compact state
        double *X[3] = {p.d_mx, p.d_mx + xs, p.d_mx + 2 * xs};
        e = launch_limit_pack(dg, g, n, flags, X[0], opA, prec, kpad, kofs, st);
        if (e != cudaSuccess) return e;
        for (int step = 0; step < n_steps; ++step) {
            const bool last = step == n_steps - 1;
            for (int stage = 0; stage < 3; ++stage) {
                {
                    LaunchTimer timer(b->ctx, 0, st);
                    e = launch_contract_tc(dg, G.tc[prec], prec, opA, n, p.d_F32, b->d_err, st);
                }
                if (e != cudaSuccess) return e;
                UpdateArgs u;
                u.F32 = p.d_F32;
                u.gn = X[0];
                u.gs = X[stage];
                u.in_mixed = 1;
                u.dt = dt;
                u.a = ca[stage];
                u.b = cb[stage];
                u.flags = flags;
                const bool final_stage = stage == 2 && last;
                u.gout = stage < 2 ? X[stage + 1] : (last ? g : X[0]);
                u.out_mixed = final_stage ? 0 : 1;
                if (stage == 2) {
                    u.apply_limiter = (!last && dg.limiter) ? 1 : 0;
                    u.mass = last ? mass : nullptr;
                }
                if (!final_stage) {
                    u.opA = opA;
                    u.opA_prec = prec;
                    u.opA_kpad = kpad;
                    u.opA_kofs = kofs;
                }
                LaunchTimer timer(b->ctx, 1, st);
                e = launch_update_tc(dg, u, n, st);
                if (e != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    }
    // reconstruction of the first step (Sec. 3.2.2); later ones are fused into stage 3
    if (dg.limiter) {
        e = launch_limit(dg, g, n, flags, nullptr, 0, 0, 0, st);
        if (e != cudaSuccess) return e;
    }
    for (int step = 0; step < n_steps; ++step) {
        const bool last = step == n_steps - 1;
        const double *gin[3] = {g, p.d_g1, p.d_g2};
        double *gout[3] = {p.d_g1, p.d_g2, g};
        for (int stage = 0; stage < 3; ++stage) {
            UpdateArgs u;
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
            {
                {
                    LaunchTimer timer(b->ctx, 0, st);
                    e = dg.cell_alpha
                            ? launch_nc_functionals(dg, G.nc, gin[stage], p.d_alpha, n, p.d_G, p.d_H, p.d_F, st)
                            : launch_contract_fp64(dg, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, gin[stage], n, p.d_F, st);
                }
                if (e != cudaSuccess) return e;
                u.F = p.d_F;
                LaunchTimer timer(b->ctx, 1, st);
                e = launch_update(dg, u, n, st);
            }
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// runs fn(part, stream) for every part: direct parts on the context stream, the
// others on their own streams forked from and joined back to it
template <typename Fn>
cudaError_t for_parts(grace_batch *b, Fn fn)
{
    cudaStream_t st = b->ctx->stream;
    cudaError_t e = cudaSuccess;
    const bool fork = !(b->parts.size() == 1 && b->parts[0].direct);
    if (fork) e = cudaEventRecord(b->fork, st);
    for (Part &p : b->parts) {
        if (e != cudaSuccess) break;
        if (!p.direct) e = cudaStreamWaitEvent(p.stream, b->fork, 0);
        if (e == cudaSuccess) e = fn(p, part_stream(b, p));
        if (e == cudaSuccess && !p.direct) e = cudaEventRecord(p.done, p.stream);
    }
    if (fork)
        for (Part &p : b->parts)
            if (e == cudaSuccess && !p.direct) e = cudaStreamWaitEvent(st, p.done, 0);
    return e;
}

cudaError_t gather_state(const Part &p, int P, const double *src, double *dst, cudaStream_t st)
{
    gather_rows_kernel<<<nb((long long)p.n * P), 256, 0, st>>>(p.n, P, p.d_off, src, dst);
    return cudaGetLastError();
}

cudaError_t scatter_state(const Part &p, int P, const double *src, double *dst, cudaStream_t st)
{
    scatter_rows_kernel<<<nb((long long)p.n * P), 256, 0, st>>>(p.n, P, p.d_off, src, dst);
    return cudaGetLastError();
}

}  // namespace
}  // namespace grace

using namespace grace;

extern "C" {

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
        const int ng = (int)ctx->groups.size();
        if (cell_group)
            for (int c = 0; c < n_cells; ++c) {
                if (cell_group[c] < 0 || cell_group[c] >= ng) {
                    delete b;
                    set_error("grace_bind_batch: cell group out of range");
                    return GRACE_ERR_ARG;
                }
                b->h_group[c] = cell_group[c];
            }
        b->h_off.resize(n_cells + 1);
        b->h_off[0] = 0;
        for (int c = 0; c < n_cells; ++c) b->h_off[c + 1] = b->h_off[c] + ctx->groups[b->h_group[c]].dg.P;
        // one part per group present
        std::vector<std::vector<int>> members(ng);
        for (int c = 0; c < n_cells; ++c) members[b->h_group[c]].push_back(c);
        int present = 0;
        for (int gi = 0; gi < ng; ++gi) present += !members[gi].empty();
        const bool direct = present == 1 && members[b->h_group[0]].size() == (size_t)n_cells;
        cudaError_t e = cudaMalloc(&b->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        const bool tc_any = (ctx->precision_mask & ((1u << GRACE_TF32) | (1u << GRACE_BF16X3))) != 0;
        for (int gi = 0; gi < ng && e == cudaSuccess; ++gi) {
            if (members[gi].empty()) continue;
            b->parts.emplace_back();
            Part &p = b->parts.back();
            p.group = gi;
            p.n = (int)members[gi].size();
            p.direct = direct;
            const DevGroup &g = ctx->groups[gi].dg;
            const size_t n = (size_t)p.n;
            e = cudaMalloc(&p.d_F, n * g.R * sizeof(double));
            if (e == cudaSuccess && g.cell_alpha) {
                const size_t nq = (size_t)g.N * g.Q;
                e = cudaMalloc(&p.d_alpha, n * sizeof(double));
                if (e == cudaSuccess) e = cudaMalloc(&p.d_G, n * nq * sizeof(double));
                if (e == cudaSuccess) e = cudaMalloc(&p.d_H, 2 * n * nq * sizeof(double));
            }
            if (e == cudaSuccess) e = cudaMalloc(&p.d_g1, n * g.P * sizeof(double));
            if (e == cudaSuccess) e = cudaMalloc(&p.d_g2, n * g.P * sizeof(double));
            if (e == cudaSuccess && !direct) {
                std::vector<long long> off(n);
                for (size_t c = 0; c < n; ++c) off[c] = b->h_off[members[gi][c]];
                e = cudaMalloc(&p.d_idx, n * sizeof(int));
                if (e == cudaSuccess) e = cudaMalloc(&p.d_off, n * sizeof(long long));
                if (e == cudaSuccess) e = cudaMemcpy(p.d_idx, members[gi].data(), n * sizeof(int), cudaMemcpyHostToDevice);
                if (e == cudaSuccess) e = cudaMemcpy(p.d_off, off.data(), n * sizeof(long long), cudaMemcpyHostToDevice);
                if (e == cudaSuccess) e = cudaMalloc(&p.d_g, n * g.P * sizeof(double));
                if (e == cudaSuccess) e = cudaMalloc(&p.d_out, n * g.P * sizeof(double));
                if (e == cudaSuccess) e = cudaMalloc(&p.d_dt, n * sizeof(double));
                if (e == cudaSuccess) e = cudaMalloc(&p.d_mass, n * sizeof(double));
                if (e == cudaSuccess) e = cudaMalloc(&p.d_flags, n);
                if (e == cudaSuccess) e = cudaMalloc(&p.d_ic, n * 4 * sizeof(double));
                if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming);
            }
            if (e == cudaSuccess && tc_any) {
                e = cudaMalloc(&p.d_F32, f32_bytes_for(g, (int)n));
                if (e == cudaSuccess) e = cudaMemset(p.d_F32, 0, f32_bytes_for(g, (int)n));
                size_t bytes = 0;
                for (int prec = GRACE_TF32; prec <= GRACE_BF16X3; ++prec)
                    if (ctx->precision_mask & (1u << prec)) bytes = std::max(bytes, opA_bytes_for(g, prec, p.n, nullptr));
                if (e == cudaSuccess) e = cudaMalloc(&p.d_opA, bytes);
                if (e == cudaSuccess) e = cudaMalloc(&p.d_mx, 3 * ((mixed_bytes_for(g, (int)n) + 15) / 16 * 16));
                if (e == cudaSuccess) e = cudaMemset(p.d_opA, 0, bytes);
                p.opA_bytes = bytes;
                if (e == cudaSuccess && g.cell_alpha) {
                    const size_t tiles = (n + kTileM - 1) / kTileM;
                    e = cudaMalloc(&p.d_gh, tiles * g.P * kTileM * sizeof(float));
                    if (e == cudaSuccess) e = cudaMemset(p.d_gh, 0, tiles * g.P * kTileM * sizeof(float));
                    if (e == cudaSuccess) e = cudaMalloc(&p.d_s, n * sizeof(float));
                }
            }
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

grace_status grace_rhs(grace_batch *b, const double *g, double *L, int prec)
{
    if (!b || !g || !L) {
        set_error("grace_rhs: null argument");
        return GRACE_ERR_ARG;
    }
    grace_status s = check_prec(b, prec);
    if (s != GRACE_OK) return s;
    Guard guard(b->ctx->device);
    cudaError_t e = for_parts(b, [&](Part &p, cudaStream_t st) {
        if (p.direct) return part_rhs(b, p, g, L, prec);
        const int P = b->ctx->groups[p.group].dg.P;
        cudaError_t r = gather_state(p, P, g, p.d_g, st);
        if (r == cudaSuccess) r = part_rhs(b, p, p.d_g, p.d_out, prec);
        if (r == cudaSuccess) r = scatter_state(p, P, p.d_out, L, st);
        return r;
    });
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_rhs");
}

// Grouped tensor-form step: every part of the batch in a fixed number of launches per stage
// (gather, step-start limiter, per stage one multi-group contraction and one grouped K-c,
// scatter).  The descriptors depend on the precision and on whether mass / flags are asked for;
// they are built (allocating, synchronising) before the launches and kept with the batch.
struct GroupedPlan {
    int prec = -1, with_mass = -1, with_flags = -1;
    TcMulti multi;
    UpdPart *d_upd = nullptr;        // [5][n_parts]: limiter, stage 1, stage 2, stage 3, last stage 3
    MovePart *d_move = nullptr;
    int n_parts = 0, n_blocks = 0;
    size_t smem[5] = {0, 0, 0, 0, 0};
    long long total_elems = 0, total_cells = 0;
};

static void free_grouped(grace_batch *b)
{
    GroupedPlan *gp = (GroupedPlan *)b->grouped;
    if (!gp) return;
    free_tc_multi(gp->multi);
    cudaFree(gp->d_upd);
    cudaFree(gp->d_move);
    delete gp;
    b->grouped = nullptr;
}

static bool grouped_applies(grace_batch *b, int prec, int n_steps)
{
    if (!b->use_grouped || prec == GRACE_FP64 || n_steps < 1 || b->parts.size() < 2) return false;
    const size_t limit = update_smem_limit();
    for (const Part &p : b->parts) {
        const Group &G = b->ctx->groups[p.group];
        if (p.direct || G.dg.cell_alpha) return false;
        // a group whose grouped stage update does not fit a block runs per group
        if (update_tc_grouped_max_smem(G.dg, G.tc[prec].k_pad) > limit) return false;
    }
    return true;
}

static grace_status grouped_prepare(grace_batch *b, int prec, bool with_mass, bool with_flags)
{
    GroupedPlan *gp = (GroupedPlan *)b->grouped;
    if (gp && gp->prec == prec && gp->with_mass == (int)with_mass && gp->with_flags == (int)with_flags)
        return GRACE_OK;
    free_grouped(b);
    gp = new GroupedPlan();
    b->grouped = gp;
    const int np = (int)b->parts.size();
    std::vector<TcMultiPart> mp;
    std::vector<UpdPart> up((size_t)5 * np);
    std::vector<MovePart> mv(np);
    const int cpb = update_tc_grouped_cpb();
    int blocks = 0;
    long long elems = 0, cells = 0;
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int i = 0; i < np; ++i) {
        Part &p = b->parts[i];
        Group &G = b->ctx->groups[p.group];
        const DevGroup &dg = G.dg;
        mp.push_back({&G.tc[prec], p.d_opA, p.d_F32, p.n, dg.R});
        const int kpad = G.tc[prec].k_pad, kofs = G.tc[prec].k_ofs;
        const size_t xs = (mixed_bytes_for(dg, p.n) + 15) / 16 * 2;
        double *X[3] = {p.d_mx, p.d_mx + xs, p.d_mx + 2 * xs};
        unsigned char *fl = with_flags ? p.d_flags : nullptr;
        UpdateArgs u[5];
        // step-start limiter: FP64 part rows -> compact X[0] + A operand
        u[0].gs = p.d_g;
        u[0].gout = X[0];
        u[0].apply_limiter = dg.limiter;
        u[0].flags = fl;
        u[0].opA = p.d_opA;
        u[0].opA_prec = prec;
        u[0].opA_kpad = kpad;
        u[0].opA_kofs = kofs;
        u[0].out_mixed = 1;
        // stages 1, 2, 3 (not the call's last step), 3 of the last step
        for (int c = 1; c < 5; ++c) {
            const int stage = c <= 3 ? c - 1 : 2;
            const bool last = c == 4;
            UpdateArgs &v = u[c];
            v.F32 = p.d_F32;
            v.gn = X[0];
            v.gs = X[stage];
            v.in_mixed = 1;
            v.dt = p.d_dt;
            v.a = ca[stage];
            v.b = cb[stage];
            v.flags = fl;
            v.gout = stage < 2 ? X[stage + 1] : (last ? p.d_g : X[0]);
            v.out_mixed = last ? 0 : 1;
            if (stage == 2) {
                v.apply_limiter = (!last && dg.limiter) ? 1 : 0;
                v.mass = last && with_mass ? p.d_mass : nullptr;
            }
            if (!last) {
                v.opA = p.d_opA;
                v.opA_prec = prec;
                v.opA_kpad = kpad;
                v.opA_kofs = kofs;
            }
        }
        for (int c = 0; c < 5; ++c) {
            UpdPart &q = up[(size_t)c * np + i];
            q.G = dg;
            q.A = u[c];
            q.n_cells = p.n;
            q.first_block = blocks;
            gp->smem[c] = std::max(gp->smem[c], update_tc_grouped_smem(dg, u[c]));
        }
        blocks += (p.n + cpb - 1) / cpb;
        MovePart &m = mv[i];
        m.elem0 = elems;
        m.cell0 = cells;
        m.n = p.n;
        m.P = dg.P;
        m.off = p.d_off;
        m.idx = p.d_idx;
        m.g = p.d_g;
        m.dt = p.d_dt;
        m.mass = p.d_mass;
        m.flags = p.d_flags;
        elems += (long long)p.n * dg.P;
        cells += p.n;
    }
    grace_status s = build_tc_multi(prec, mp, gp->multi);
    if (s != GRACE_OK) {
        free_grouped(b);
        return s;
    }
    cudaError_t e = cudaMalloc(&gp->d_upd, up.size() * sizeof(UpdPart));
    if (e == cudaSuccess) e = cudaMalloc(&gp->d_move, mv.size() * sizeof(MovePart));
    if (e == cudaSuccess) e = cudaMemcpy(gp->d_upd, up.data(), up.size() * sizeof(UpdPart), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(gp->d_move, mv.data(), mv.size() * sizeof(MovePart), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_grouped(b);
        return cuda_fail(e, "grace_step: grouped plan");
    }
    gp->prec = prec;
    gp->with_mass = with_mass;
    gp->with_flags = with_flags;
    gp->n_parts = np;
    gp->n_blocks = blocks;
    gp->total_elems = elems;
    gp->total_cells = cells;
    return GRACE_OK;
}

static cudaError_t grouped_step(grace_batch *b, double *g, const double *dt, int n_steps, double *mass,
                                unsigned char *flags)
{
    GroupedPlan &gp = *(GroupedPlan *)b->grouped;
    cudaStream_t st = b->ctx->stream;
    const int np = gp.n_parts;
    grouped_rows_kernel<<<nb(gp.total_elems), 256, 0, st>>>(gp.d_move, np, gp.total_elems, g, nullptr, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        grouped_cells_kernel<<<nb(gp.total_cells), 256, 0, st>>>(gp.d_move, np, gp.total_cells, dt, nullptr,
                                                                 nullptr, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        LaunchTimer timer(b->ctx, 1, st);
        e = launch_update_tc_grouped(GROUPED_LIMIT, false, true, gp.d_upd, np, gp.n_blocks, gp.smem[0], st);
    }
    for (int step = 0; step < n_steps && e == cudaSuccess; ++step) {
        const bool last = step == n_steps - 1;
        for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
            {
                LaunchTimer timer(b->ctx, 0, st);
                e = launch_contract_tc_multi(gp.multi, b->d_err, st);
            }
            if (e != cudaSuccess) break;
            const int c = stage < 2 ? stage + 1 : (last ? 4 : 3);
            LaunchTimer timer(b->ctx, 1, st);
            e = launch_update_tc_grouped(GROUPED_STAGE, true, c != 4, gp.d_upd + (size_t)c * np, np, gp.n_blocks,
                                         gp.smem[c], st);
        }
    }
    if (e == cudaSuccess) {
        grouped_rows_kernel<<<nb(gp.total_elems), 256, 0, st>>>(gp.d_move, np, gp.total_elems, nullptr, g, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && (mass || flags)) {
        grouped_cells_kernel<<<nb(gp.total_cells), 256, 0, st>>>(gp.d_move, np, gp.total_cells, nullptr, mass,
                                                                 flags, 1);
        e = cudaGetLastError();
    }
    return e;
}

static cudaError_t step_body(grace_batch *b, double *g, const double *dt, int n_steps, int prec, double *mass,
                             unsigned char *flags)
{
    if (grouped_applies(b, prec, n_steps)) return grouped_step(b, g, dt, n_steps, mass, flags);
    return for_parts(b, [&](Part &p, cudaStream_t st) {
        if (p.direct) return part_step(b, p, g, dt, n_steps, prec, mass, flags);
        const int P = b->ctx->groups[p.group].dg.P;
        cudaError_t r = gather_state(p, P, g, p.d_g, st);
        if (r == cudaSuccess) {
            gather_kernel<double><<<nb(p.n), 256, 0, st>>>(p.n, 1, p.d_idx, dt, p.d_dt);
            r = cudaGetLastError();
        }
        if (r == cudaSuccess)
            r = part_step(b, p, p.d_g, p.d_dt, n_steps, prec, mass ? p.d_mass : nullptr, flags ? p.d_flags : nullptr);
        if (r == cudaSuccess) r = scatter_state(p, P, p.d_g, g, st);
        if (r == cudaSuccess && mass) {
            scatter_kernel<double><<<nb(p.n), 256, 0, st>>>(p.n, p.d_idx, p.d_mass, mass);
            r = cudaGetLastError();
        }
        if (r == cudaSuccess && flags) {
            scatter_kernel<unsigned char><<<nb(p.n), 256, 0, st>>>(p.n, p.d_idx, p.d_flags, flags);
            r = cudaGetLastError();
        }
        return r;
    });
}

static cudaError_t mass_body(grace_batch *b, const double *g, double *mass)
{
    return for_parts(b, [&](Part &p, cudaStream_t st) {
        const DevGroup &dg = b->ctx->groups[p.group].dg;
        if (p.direct) return launch_mass(dg, g, p.n, mass, st);
        cudaError_t r = gather_state(p, dg.P, g, p.d_g, st);
        if (r == cudaSuccess) r = launch_mass(dg, p.d_g, p.n, p.d_mass, st);
        if (r == cudaSuccess) {
            scatter_kernel<double><<<nb(p.n), 256, 0, st>>>(p.n, p.d_idx, p.d_mass, mass);
            r = cudaGetLastError();
        }
        return r;
    });
}

// mass-drift bit: M_1 of a cell of a conservative group changed over the call by more than
// drift_tol(n_steps) of its value (or became NaN) although every stage kept eq. (dt) and left the
// means non-negative and finite.  With conservative fluxes the flux differences of eq. (g0)
// telescope exactly, so M_1 moves only by the rounding of the stage updates: under eq. (dt)
// (sum_j h_j dt |L_j^0| <= 2 M_1 per stage) at most 27.1 u M_1 per SSP-RK3 step plus 2 N u for
// the two mass sums, u = 2^-53.  The tolerance is 32 u per step with a floor of 1e-10.  Cells
// with one of the skipped bits set are already flagged, and their M_1 can move by round-off of
// a much larger state.
constexpr unsigned char kDriftSkip = GRACE_FLAG_NEGATIVE_MEAN | GRACE_FLAG_NONFINITE | GRACE_FLAG_CFL;

static double drift_tol(int n_steps) { return std::max(1e-10, 32.0 * std::ldexp(1.0, -53) * n_steps); }

__global__ void drift_kernel(int n, double tol, const double *__restrict__ m0, const double *__restrict__ m1,
                             const unsigned char *__restrict__ cons, unsigned char *__restrict__ flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && cons[i] && !(flags[i] & kDriftSkip) && !(fabs(m1[i] - m0[i]) <= tol * fabs(m0[i])))
        flags[i] |= (unsigned char)GRACE_FLAG_MASS_DRIFT;
}

// the workspaces of the drift bit, allocated outside any graph capture
static cudaError_t ensure_drift(grace_batch *b)
{
    if (b->d_drift) return cudaSuccess;
    const int n = b->n_cells;
    std::vector<unsigned char> cons(n);
    for (int c = 0; c < n; ++c) cons[c] = b->ctx->groups[b->h_group[c]].dg.flux_mode == 0 ? 1 : 0;
    cudaError_t e = cudaMalloc(&b->d_drift, (size_t)2 * n * sizeof(double) + n);
    if (e != cudaSuccess) {
        b->d_drift = nullptr;
        return e;
    }
    return cudaMemcpy(reinterpret_cast<unsigned char *>(b->d_drift + 2 * (size_t)n), cons.data(), n,
                      cudaMemcpyHostToDevice);
}

// step_body, plus the mass-drift bit when flags are requested
static cudaError_t step_flagged(grace_batch *b, double *g, const double *dt, int n_steps, int prec, double *mass,
                                unsigned char *flags)
{
    if (!flags) return step_body(b, g, dt, n_steps, prec, mass, flags);
    const int n = b->n_cells;
    double *m0 = b->d_drift, *m1 = b->d_drift + n;
    const unsigned char *cons = reinterpret_cast<const unsigned char *>(b->d_drift + 2 * (size_t)n);
    cudaError_t e = mass_body(b, g, m0);
    if (e == cudaSuccess) e = step_body(b, g, dt, n_steps, prec, mass, flags);
    if (e == cudaSuccess) e = mass_body(b, g, m1);
    if (e == cudaSuccess) {
        drift_kernel<<<(n + 255) / 256, 256, 0, b->ctx->stream>>>(n, drift_tol(n_steps), m0, m1, cons, flags);
        e = cudaGetLastError();
    }
    return e;
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
    cudaError_t e = cudaSuccess;
    if (grouped_applies(b, prec, n_steps)) {
        // descriptors are built outside any graph capture
        s = grouped_prepare(b, prec, mass != nullptr, flags != nullptr);
        if (s != GRACE_OK) return s;
    }
    if (flags) {
        e = ensure_drift(b);
        if (e != cudaSuccess) return cuda_fail(e, "grace_step: mass-drift workspace");
    }
    if (!b->use_graph) {
        e = step_flagged(b, g, dt, n_steps, prec, mass, flags);
        return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_step");
    }
    // CUDA graph: capture the whole call once per argument set, then replay it
    const void *key[4] = {g, dt, mass, flags};
    const bool same = b->graph && b->graph_steps == n_steps && b->graph_prec == prec &&
                      std::equal(key, key + 4, b->graph_key);
    cudaStream_t st = b->ctx->stream;
    if (!same) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        if (!st) {
            set_error("grace_step: graph replay needs a non-default stream (grace_set_stream)");
            return GRACE_ERR_ARG;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            b->ctx->capturing = 1;
            cudaError_t body = step_flagged(b, g, dt, n_steps, prec, mass, flags);
            b->ctx->capturing = 0;
            e = cudaStreamEndCapture(st, &graph);
            if (body != cudaSuccess) e = body;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return cuda_fail(e, "grace_step: graph capture");
        }
        std::copy(key, key + 4, b->graph_key);
        b->graph_steps = n_steps;
        b->graph_prec = prec;
    }
    e = cudaGraphLaunch(b->graph, st);
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_step: graph launch");
}

grace_status grace_batch_set_grouped(grace_batch *b, int enable)
{
    if (!b) {
        set_error("grace_batch_set_grouped: null batch");
        return GRACE_ERR_ARG;
    }
    b->use_grouped = enable ? 1 : 0;
    if (b->graph) {
        Guard guard(b->ctx->device);
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return GRACE_OK;
}

grace_status grace_batch_set_graph(grace_batch *b, int enable)
{
    if (!b) {
        set_error("grace_batch_set_graph: null batch");
        return GRACE_ERR_ARG;
    }
    b->use_graph = enable ? 1 : 0;
    if (!enable && b->graph) {
        Guard guard(b->ctx->device);
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
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
    const cudaError_t e = mass_body(b, g, mass);
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_mass");
}

grace_status grace_limit(grace_batch *b, double *g, unsigned char *flags)
{
    if (!b || !g) {
        set_error("grace_limit: null argument");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    cudaError_t e = for_parts(b, [&](Part &p, cudaStream_t st) {
        const DevGroup &dg = b->ctx->groups[p.group].dg;
        double *gs = p.direct ? g : p.d_g;
        unsigned char *fl = flags ? (p.direct ? flags : p.d_flags) : nullptr;
        cudaError_t r = cudaSuccess;
        if (!p.direct) r = gather_state(p, dg.P, g, p.d_g, st);
        if (r == cudaSuccess && fl) r = cudaMemsetAsync(fl, 0, p.n, st);
        if (r == cudaSuccess) r = launch_limit(dg, gs, p.n, fl, nullptr, 0, 0, 0, st);
        if (r == cudaSuccess && !p.direct) r = scatter_state(p, dg.P, p.d_g, g, st);
        if (r == cudaSuccess && fl && !p.direct) {
            scatter_kernel<unsigned char><<<nb(p.n), 256, 0, st>>>(p.n, p.d_idx, p.d_flags, flags);
            r = cudaGetLastError();
        }
        return r;
    });
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_limit");
}

grace_status grace_project(grace_batch *b, int ic_kind, const double *ic_params, double *g)
{
    if (!b || !ic_params || !g || ic_kind < GRACE_IC_EXP || ic_kind > GRACE_IC_FIRST_BIN) {
        set_error("grace_project: bad argument");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    cudaError_t e = for_parts(b, [&](Part &p, cudaStream_t st) {
        const DevGroup &dg = b->ctx->groups[p.group].dg;
        if (p.direct) return launch_project(dg, ic_kind, ic_params, p.n, g, st);
        gather_kernel<double><<<nb((long long)p.n * 4), 256, 0, st>>>(p.n, 4, p.d_idx, ic_params, p.d_ic);
        cudaError_t r = cudaGetLastError();
        if (r == cudaSuccess) r = launch_project(dg, ic_kind, p.d_ic, p.n, p.d_g, st);
        if (r == cudaSuccess) r = scatter_state(p, dg.P, p.d_g, g, st);
        return r;
    });
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_project");
}

grace_status grace_batch_cell_params(grace_batch *b, const double *alpha)
{
    if (!b || !alpha) {
        set_error("grace_batch_cell_params: null argument");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    cudaError_t e = for_parts(b, [&](Part &p, cudaStream_t st) {
        if (!b->ctx->groups[p.group].dg.cell_alpha) return cudaSuccess;
        if (p.direct) return cudaMemcpyAsync(p.d_alpha, alpha, (size_t)p.n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        gather_kernel<double><<<nb(p.n), 256, 0, st>>>(p.n, 1, p.d_idx, alpha, p.d_alpha);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return cuda_fail(e, "grace_batch_cell_params");
    b->alpha_set = 1;
    return GRACE_OK;
}

__global__ void flags_or_kernel(int n, const unsigned char *__restrict__ flags, unsigned *__restrict__ out)
{
    unsigned v = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v |= flags[i];
    v = __reduce_or_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicOr(out, v);
}

grace_status grace_flags_check(grace_batch *b, const unsigned char *flags, unsigned *any)
{
    if (!b || !flags) {
        set_error("grace_flags_check: null argument");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    cudaStream_t st = b->ctx->stream;
    cudaError_t e = cudaSuccess;
    if (!b->d_flag_or) e = cudaMalloc(&b->d_flag_or, sizeof(unsigned));
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flag_or, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        const int blocks = (int)std::min<long long>(((long long)b->n_cells + 255) / 256, 1184);
        flags_or_kernel<<<blocks, 256, 0, st>>>(b->n_cells, flags, b->d_flag_or);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, b->d_flag_or, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "grace_flags_check");
    if (any) *any = h;
    return h ? GRACE_WARN_CELLS : GRACE_OK;
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
    if (b->graph) cudaGraphExecDestroy(b->graph);
    free_host_io(b);
    free_hydro(b);
    free_species(b);
    free_implicit(b);
    free_grouped(b);
    for (Part &p : b->parts) free_part(p);
    cudaFree(b->d_err);
    cudaFree(b->d_adj);
    cudaFree(b->d_drift);
    cudaFree(b->d_flag_or);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

}  // extern "C"
