// Species of mixed grains (Sec. 5.3): grains are mixtures of S constituent species, and the state
// of a cell is the partial mass density g_s of each species on the common mass grid, with
// g = sum_s g_s.  Every flux integral of eqs. (Fcoagtrun), (Ffragtrun) carries the share of the
// products of its outer collider (mass u); a species' flux takes g_s in that slot and the total g in
// the partner's, so its rate is the bilinear form L_s = L[g_s; g] on the tables T of L[g] (T as
// built, not folded: the two slots differ).  The FP64 contraction shares the row sums over the
// partner between the species; the tensor forms run one tcgen05 pass over T with the cells' total
// as the A operand (Y[c, (r, p)] = sum_q That_r[p, q] ghat_q, shared by every species) and an
// epilogue that contracts Y with each species' coefficients.  The flux difference, stage update,
// limiter, mass and status bits of each species are the single-distribution kernels applied to
// that species.
//
// Layout: gs[S][n_cells][P] (species-major), so each species is a packed state of the batch.
#include <algorithm>
#include <cmath>
#include <string>

#include "grace_convert.cuh"
#include "grace_internal.h"
#include "grace_tc_layout.cuh"

namespace grace {

namespace {

struct SpeciesWs {
    int S = 0;
    double *gt = nullptr;        // [n][P] total of the current stage input
    double *F = nullptr;         // [S][n][R] functionals
    double *g1 = nullptr, *g2 = nullptr;   // [S][n][P] stage states
    double *m = nullptr;         // [2][S][n] per-species M_1 before / after (drift bit)
    // tensor forms: the total's A operand, the species' scaled coefficients in FP32
    // ([S][cell tile][kpad][128]) and the FP32 functionals ([S][cell tile][R][128])
    int tc_kpad = 0;
    void *opA = nullptr;
    float *gsp = nullptr, *F32 = nullptr;
};

// ghat_s = h_bin g_s of every species in FP32 at the A operand's columns (coefficient p at column
// kofs + p, zero elsewhere and for the rows past the last cell), one 128-cell column per coefficient
__global__ void species_pack_kernel(int n, int S, int P, int K1, int kpad, int kofs, const double *__restrict__ gs,
                                    const double *__restrict__ hbin, float *__restrict__ gsp)
{
    const int n_ct = (n + kTileM - 1) / kTileM;
    const long long total = (long long)S * n_ct * kpad * kTileM;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(i % kTileM);
        long long rest = i / kTileM;
        const int col = (int)(rest % kpad);
        rest /= kpad;
        const int ct = (int)(rest % n_ct);
        const int sp = (int)(rest / n_ct);
        const long long cell = (long long)ct * kTileM + row;
        const int p = col - kofs;
        float v = 0.f;
        if (cell < n && p >= 0 && p < P) v = d2f_fast(hbin[p / K1] * gs[((size_t)sp * n + cell) * P + p]);
        gsp[i] = v;
    }
}

__global__ void species_sum_kernel(long long n_elems, int S, const double *__restrict__ gs, double *__restrict__ g)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_elems) return;
    double s = 0.0;
    for (int sp = 0; sp < S; ++sp) s += gs[(size_t)sp * n_elems + i];
    g[i] = s;
}

// bit 16 from the cell's total M_1 over the call (eq. g0 with eq. dt kept: conserved to round-off)
__global__ void species_drift_kernel(int n, int S, double tol, const double *__restrict__ m0,
                                     const double *__restrict__ m1, unsigned char *__restrict__ flags)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double a = 0.0, b = 0.0;
    for (int sp = 0; sp < S; ++sp) {
        a += m0[(size_t)sp * n + c];
        b += m1[(size_t)sp * n + c];
    }
    const unsigned char skip = GRACE_FLAG_NEGATIVE_MEAN | GRACE_FLAG_NONFINITE | GRACE_FLAG_CFL;
    if (!(flags[c] & skip) && !(fabs(b - a) <= tol * fabs(a))) flags[c] |= (unsigned char)GRACE_FLAG_MASS_DRIFT;
}

}  // namespace

static grace_status species_ws(grace_batch *b, int S, SpeciesWs **out)
{
    SpeciesWs *w = static_cast<SpeciesWs *>(b->species);
    if (w && w->S >= S) {
        *out = w;
        return GRACE_OK;
    }
    free_species(b);
    w = new SpeciesWs();
    const DevGroup &g = b->ctx->groups[b->parts[0].group].dg;
    const size_t n = (size_t)b->n_cells;
    cudaError_t e = cudaMalloc(&w->gt, n * g.P * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->F, (size_t)S * n * g.R * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->g1, (size_t)S * n * g.P * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->g2, (size_t)S * n * g.P * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->m, 2 * (size_t)S * n * sizeof(double));
    w->S = S;
    b->species = w;
    if (e != cudaSuccess) {
        free_species(b);
        return cuda_fail(e, "species workspace");
    }
    *out = w;
    return GRACE_OK;
}

void free_species(grace_batch *b)
{
    SpeciesWs *w = static_cast<SpeciesWs *>(b->species);
    if (!w) return;
    cudaFree(w->gt);
    cudaFree(w->F);
    cudaFree(w->g1);
    cudaFree(w->g2);
    cudaFree(w->m);
    cudaFree(w->opA);
    cudaFree(w->gsp);
    cudaFree(w->F32);
    delete w;
    b->species = nullptr;
}

// tensor-form buffers and species tiles for precision prec (allocates and plans on first use)
static grace_status species_tc(grace_batch *b, SpeciesWs *w, int prec)
{
    Group &G = b->ctx->groups[b->parts[0].group];
    if (!G.tcs[prec].built) {
        grace_status s = build_species_tiles(G, prec, b->ctx->stream);
        if (s != GRACE_OK) return s;
    }
    const int kpad = G.tcs[prec].k_pad;
    if (w->tc_kpad == kpad && w->opA) return GRACE_OK;
    cudaFree(w->opA);
    cudaFree(w->gsp);
    cudaFree(w->F32);
    w->opA = nullptr;
    w->gsp = w->F32 = nullptr;
    w->tc_kpad = 0;
    const size_t n_ct = ((size_t)b->n_cells + kTileM - 1) / kTileM;
    // the A tile takes 4 bytes per element in both forms (TF32, or BF16 hi + lo)
    cudaError_t e = cudaMalloc(&w->opA, n_ct * opA_tile_bytes(prec, kpad));
    if (e == cudaSuccess) e = cudaMalloc(&w->gsp, (size_t)w->S * n_ct * kpad * kTileM * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&w->F32, (size_t)w->S * n_ct * G.dg.R * kTileM * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "species tensor workspace");
    w->tc_kpad = kpad;
    return GRACE_OK;
}

static grace_status species_check(grace_batch *b, int S, const void *gs, int prec, const char *who)
{
    if (!b || !gs || S < 1 || S > 4 || prec < GRACE_FP64 || prec > GRACE_BF16X3) {
        set_error(std::string(who) + ": null argument, n_species outside [1, 4] or unknown precision");
        return GRACE_ERR_ARG;
    }
    if (prec != GRACE_FP64 && !b->ctx->groups[b->parts[0].group].tc[prec].built) {
        set_error(std::string(who) + ": precision not precomputed (pass its bit to grace_precompute)");
        return GRACE_ERR_ORDER;
    }
    if (b->parts.size() != 1 || !b->parts[0].direct || b->ctx->groups[b->parts[0].group].dg.cell_alpha) {
        set_error(std::string(who) + ": batches of one group in caller order without per-cell kernel parameters only");
        return GRACE_ERR_UNSUPPORTED;
    }
    return GRACE_OK;
}

// F_s of every species for the stage input x (species-major), total into w->gt: FP64 into w->F
// ([S][n][R]), or a tensor form into w->F32 ([S][cell tile][R][128])
static cudaError_t species_functionals(grace_batch *b, SpeciesWs *w, int S, const double *x, int prec,
                                       cudaStream_t st)
{
    const Group &G = b->ctx->groups[b->parts[0].group];
    const int n = b->n_cells;
    const long long elems = (long long)n * G.dg.P;
    species_sum_kernel<<<(unsigned)((elems + 255) / 256), 256, 0, st>>>(elems, S, x, w->gt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (prec == GRACE_FP64) {
        LaunchTimer timer(b->ctx, 0, st);
        return launch_contract_fp64_species(G.dg, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, S, x, w->gt, n, w->F, st);
    }
    const TcTiles &t = G.tcs[prec];
    e = launch_pack_A(G.dg, w->gt, n, w->opA, prec, t.k_pad, t.k_ofs, st);
    if (e == cudaSuccess) {
        species_pack_kernel<<<1184, 256, 0, st>>>(n, S, G.dg.P, G.dg.K1, t.k_pad, t.k_ofs, x, G.dg.hbin, w->gsp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        LaunchTimer timer(b->ctx, 0, st);
        e = launch_contract_tc_species(G.dg, t, prec, w->opA, n, w->gsp, S, w->F32, b->d_err, st);
    }
    return e;
}

}  // namespace grace

using namespace grace;

// the update arguments' functionals of species sp: FP64 [n][R] rows, or the tensor forms' FP32 tiles
static void species_F(const SpeciesWs *w, const DevGroup &dg, int n, int sp, int prec, UpdateArgs &u)
{
    if (prec == GRACE_FP64) {
        u.F = w->F + (size_t)sp * n * dg.R;
    } else {
        const size_t n_ct = ((size_t)n + kTileM - 1) / kTileM;
        u.F32 = w->F32 + (size_t)sp * n_ct * dg.R * kTileM;
    }
}

static cudaError_t species_update(const DevGroup &dg, const UpdateArgs &u, int n, int prec, cudaStream_t st)
{
    return prec == GRACE_FP64 ? launch_update(dg, u, n, st) : launch_update_tc(dg, u, n, st);
}

extern "C" grace_status grace_rhs_species(grace_batch *b, int n_species, const double *gs, double *Ls, int precision)
{
    grace_status s = species_check(b, n_species, gs, precision, "grace_rhs_species");
    if (s != GRACE_OK) return s;
    if (!Ls) {
        set_error("grace_rhs_species: null output");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    SpeciesWs *w = nullptr;
    s = species_ws(b, n_species, &w);
    if (s == GRACE_OK && precision != GRACE_FP64) s = species_tc(b, w, precision);
    if (s != GRACE_OK) return s;
    const Group &G = b->ctx->groups[b->parts[0].group];
    const int n = b->n_cells;
    cudaStream_t st = b->ctx->stream;
    cudaError_t e = species_functionals(b, w, n_species, gs, precision, st);
    for (int sp = 0; sp < n_species && e == cudaSuccess; ++sp) {
        UpdateArgs u;
        species_F(w, G.dg, n, sp, precision, u);
        u.gout = Ls + (size_t)sp * n * G.dg.P;
        LaunchTimer timer(b->ctx, 1, st);
        e = species_update(G.dg, u, n, precision, st);
    }
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_rhs_species");
}

extern "C" grace_status grace_step_species(grace_batch *b, int n_species, double *gs, const double *dt, int n_steps,
                                           int precision, double *mass, unsigned char *flags)
{
    grace_status s = species_check(b, n_species, gs, precision, "grace_step_species");
    if (s != GRACE_OK) return s;
    if (!dt || n_steps < 0) {
        set_error("grace_step_species: null dt or negative step count");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    SpeciesWs *w = nullptr;
    s = species_ws(b, n_species, &w);
    if (s == GRACE_OK && precision != GRACE_FP64) s = species_tc(b, w, precision);
    if (s != GRACE_OK) return s;
    const Group &G = b->ctx->groups[b->parts[0].group];
    const DevGroup &dg = G.dg;
    const int n = b->n_cells, S = n_species;
    const size_t sP = (size_t)n * dg.P;
    cudaStream_t st = b->ctx->stream;
    cudaError_t e = cudaSuccess;
    if (flags) e = cudaMemsetAsync(flags, 0, n, st);
    for (int sp = 0; sp < S && e == cudaSuccess && flags; ++sp) e = launch_mass(dg, gs + sp * sP, n, w->m + (size_t)sp * n, st);
    // the reconstruction of the first step; later ones are fused into stage 3
    for (int sp = 0; sp < S && e == cudaSuccess && dg.limiter && n_steps > 0; ++sp)
        e = launch_limit(dg, gs + sp * sP, n, flags, nullptr, 0, 0, 0, st);
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int step = 0; step < n_steps && e == cudaSuccess; ++step) {
        const bool last = step == n_steps - 1;
        const double *gin[3] = {gs, w->g1, w->g2};
        double *gout[3] = {w->g1, w->g2, gs};
        for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
            e = species_functionals(b, w, S, gin[stage], precision, st);
            for (int sp = 0; sp < S && e == cudaSuccess; ++sp) {
                UpdateArgs u;
                species_F(w, dg, n, sp, precision, u);
                u.gn = gs + sp * sP;
                u.gs = gin[stage] + sp * sP;
                u.gout = gout[stage] + sp * sP;
                u.dt = dt;
                u.a = ca[stage];
                u.b = cb[stage];
                u.flags = flags;
                if (stage == 2) {
                    u.apply_limiter = (!last && dg.limiter) ? 1 : 0;
                    u.mass = last && mass ? mass + (size_t)sp * n : nullptr;
                }
                LaunchTimer timer(b->ctx, 1, st);
                e = species_update(dg, u, n, precision, st);
            }
        }
    }
    if (e == cudaSuccess && n_steps == 0 && mass)
        for (int sp = 0; sp < S && e == cudaSuccess; ++sp) e = launch_mass(dg, gs + sp * sP, n, mass + (size_t)sp * n, st);
    if (e == cudaSuccess && flags) {
        for (int sp = 0; sp < S && e == cudaSuccess; ++sp)
            e = launch_mass(dg, gs + sp * sP, n, w->m + (size_t)(S + sp) * n, st);
        if (e == cudaSuccess && dg.flux_mode == 0) {
            const double tol = std::max(1e-10, 32.0 * std::ldexp(1.0, -53) * n_steps);
            species_drift_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, S, tol, w->m, w->m + (size_t)S * n, flags);
            e = cudaGetLastError();
        }
    }
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_step_species");
}
