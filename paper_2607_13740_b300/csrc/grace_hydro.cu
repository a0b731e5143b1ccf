// Operator-split coupling to a hydrodynamics code (Sec. 5.2, "Toward Hydrodynamic Implementation"):
// the coagulation-fragmentation step of every cell over the hydro step dt_hydro, sub-cycled with
// the eq. (dt) positivity bound.
//
// At the start of the call the RHS L[g] of every cell gives its bound
//     B_c = min over bins losing mass (L_j^0 < 0) of g_j^0 / |L_j^0|      (eq. dt)
// and its sub-step count n_c = ceil(dt_hydro_c / (cfl B_c)) (1 for a cell with no bin losing mass).
// The batch then takes N = max_c n_c (at most max_substeps) SSP-RK3 steps in which cell c moves by
// dt_hydro_c / N <= cfl B_c: every cell covers its own interval with its own step size, and the
// batch stays one launch sequence (no cell idles through steps of zero length).  Status bit 8
// (eq. dt broken in a stage) reports cells whose bound tightened during the interval.
#include <algorithm>
#include <cmath>
#include <vector>

#include "grace_internal.h"

namespace grace {

namespace {

struct HydroWs {
    double *L = nullptr;          // RHS of the state at the start [packed]
    double *dtc = nullptr;        // [n] sub-step size per cell
    long long *off = nullptr;     // [n + 1] packed offsets
    int *bins = nullptr;          // [n] N of the cell's group, K1 << 16
    int *count = nullptr;         // [n] n_c per cell, then the reduction word at [n]
};

// one thread per cell: B_c, n_c = ceil(dt_hydro / (cfl B_c)), clamped to [1, 2^30]
__global__ void substep_count_kernel(int n, const long long *__restrict__ off, const int *__restrict__ bins,
                                     const double *__restrict__ g, const double *__restrict__ L,
                                     const double *__restrict__ dt_hydro, double cfl, int *__restrict__ count)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int N = bins[c] & 0xFFFF, K1 = bins[c] >> 16;
    const double *gc = g + off[c], *Lc = L + off[c];
    double B = INFINITY;
    for (int j = 0; j < N; ++j) {
        const double L0 = Lc[(size_t)j * K1], g0 = gc[(size_t)j * K1];
        if (L0 < 0.0) B = fmin(B, g0 / -L0);
    }
    const double want = dt_hydro[c] / (cfl * B);   // 0 for B = inf; NaN or inf for a broken state
    int nc = 1;
    if (want > 1.0) nc = want < 1073741824.0 ? (int)ceil(want) : 1073741824;
    else if (!(want >= 0.0)) nc = 1073741824;       // NaN: let the flags report the broken cell
    count[c] = nc;
    atomicMax(count + n, nc);
}

__global__ void substep_dt_kernel(int n, const double *__restrict__ dt_hydro, int N, double *__restrict__ dtc)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) dtc[c] = dt_hydro[c] / (double)N;
}

}  // namespace

static cudaError_t ensure_hydro(grace_batch *b, HydroWs **out)
{
    if (b->hydro) {
        *out = static_cast<HydroWs *>(b->hydro);
        return cudaSuccess;
    }
    HydroWs *w = new HydroWs();
    const int n = b->n_cells;
    std::vector<int> bins(n);
    for (int c = 0; c < n; ++c) {
        const DevGroup &dg = b->ctx->groups[b->h_group[c]].dg;
        bins[c] = dg.N | (dg.K1 << 16);
    }
    cudaError_t e = cudaMalloc(&w->L, (size_t)b->h_off[n] * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->dtc, (size_t)n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->off, (size_t)(n + 1) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&w->bins, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&w->count, (size_t)(n + 1) * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(w->off, b->h_off.data(), (size_t)(n + 1) * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->bins, bins.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(w->L);
        cudaFree(w->dtc);
        cudaFree(w->off);
        cudaFree(w->bins);
        cudaFree(w->count);
        delete w;
        return e;
    }
    b->hydro = w;
    *out = w;
    return cudaSuccess;
}

void free_hydro(grace_batch *b)
{
    if (!b->hydro) return;
    HydroWs *w = static_cast<HydroWs *>(b->hydro);
    cudaFree(w->L);
    cudaFree(w->dtc);
    cudaFree(w->off);
    cudaFree(w->bins);
    cudaFree(w->count);
    delete w;
    b->hydro = nullptr;
}

}  // namespace grace

using namespace grace;

extern "C" grace_status grace_substep(grace_batch *b, double *g, const double *dt_hydro, double cfl, int max_substeps,
                                      int precision, double *mass, unsigned char *flags, int *n_sub)
{
    if (!b || !g || !dt_hydro || !(cfl > 0.0) || max_substeps < 1) {
        set_error("grace_substep: null argument, cfl <= 0 or max_substeps < 1");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    HydroWs *w = nullptr;
    cudaError_t e = ensure_hydro(b, &w);
    if (e != cudaSuccess) return cuda_fail(e, "grace_substep: workspace");
    // the bound at the start of the interval, from the FP64 RHS (the bound decides the step count)
    grace_status s = grace_rhs(b, g, w->L, GRACE_FP64);
    if (s != GRACE_OK) return s;
    cudaStream_t st = b->ctx->stream;
    const int n = b->n_cells;
    e = cudaMemsetAsync(w->count + n, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        substep_count_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, w->off, w->bins, g, w->L, dt_hydro, cfl, w->count);
        e = cudaGetLastError();
    }
    int N = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&N, w->count + n, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "grace_substep: step count");
    N = std::max(1, std::min(N, max_substeps));
    substep_dt_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, dt_hydro, N, w->dtc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "grace_substep: step size");
    s = grace_step(b, g, w->dtc, N, precision, mass, flags);
    if (s != GRACE_OK) return s;
    if (n_sub) *n_sub = N;
    return GRACE_OK;
}
