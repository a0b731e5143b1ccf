// Plain FP64 contraction on CUDA cores:  F[c, r] = sum_p g_c[p] sum_q T_r[p, q] g_c[q].
//
// One warp owns 32 cells; their coefficients sit in shared memory transposed
// ([q][lane], conflict-free), and the warp walks every non-empty row (r, p) of
// T once, reading each T entry as a warp-wide broadcast.  Warps of a block walk
// T in the same order, so T is served from L1.  The kernel is bound by the
// FP64 FMA rate, which on this part is a small fraction of the FP32 rate.
// Batches with fewer warps than the GPU holds split the functionals over
// blockIdx.y (each F_r is computed exactly as in one pass).
#include <algorithm>

#include "grace_internal.h"

namespace grace {

namespace {

// CPW cells per warp: 32 (one lane per cell), or 8 for groups whose 32-cell tile would not fit in
// shared memory (P > 800 coefficients, e.g. N = 200 bins of degree 4): then four lanes share a cell,
// each summing every fourth q of a row, and the row sums are combined with shuffles.  CPW = 1 for
// batches of a few cells (single-cell studies): the whole warp shares each row, reading T coalesced.
template <int CPW>
__global__ void __launch_bounds__(128) contract_fp64_kernel(
    const double *__restrict__ T, const int *__restrict__ qlo, const int *__restrict__ qhi,
    const int *__restrict__ prange, int R, int P, const double *__restrict__ g, int n_cells,
    double *__restrict__ F)
{
    constexpr int SUB = 32 / CPW;    // lanes per cell
    extern __shared__ double gsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const long long cell0 = ((long long)blockIdx.x * nwarps + warp) * CPW;
    double *gw = gsm + (size_t)warp * P * CPW;

    // coalesced load of CPW consecutive cells, stored transposed
    for (int idx = lane; idx < CPW * P; idx += 32) {
        const int c = idx / P, q = idx - c * P;
        const long long cell = cell0 + c;
        gw[q * CPW + c] = cell < n_cells ? g[cell * P + q] : 0.0;
    }
    __syncwarp();

    const int c = lane % CPW, sub = lane / CPW;
    const long long cell = cell0 + c;
    const int r_per = (R + gridDim.y - 1) / gridDim.y;
    const int r_begin = blockIdx.y * r_per, r_end = min(R, r_begin + r_per);
    for (int r = r_begin; r < r_end; ++r) {
        const int p0 = prange[2 * r], p1 = prange[2 * r + 1];
        double Fr = 0.0;
        for (int p = p0; p < p1; ++p) {
            const int q0 = qlo[r * P + p], q1 = qhi[r * P + p];
            if (q0 >= q1) continue;
            const double *Trow = T + ((size_t)r * P + p) * P;
            double y0 = 0.0, y1 = 0.0;
            int q = q0 + sub;
            for (; q + SUB < q1; q += 2 * SUB) {
                y0 = fma(__ldg(Trow + q), gw[q * CPW + c], y0);
                y1 = fma(__ldg(Trow + q + SUB), gw[(q + SUB) * CPW + c], y1);
            }
            if (q < q1) y0 = fma(__ldg(Trow + q), gw[q * CPW + c], y0);
            double y = y0 + y1;
#pragma unroll
            for (int o = CPW; o < 32; o <<= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            Fr = fma(gw[p * CPW + c], y, Fr);
        }
        if (sub == 0 && cell < n_cells) F[cell * R + r] = Fr;
    }
}

// Species of mixed grains (Sec. 5.3): F_s[c, r] = sum_p gs_s[c, p] sum_q T_r[p, q] g[c, q] for S <= 4
// species, g = sum_s gs_s, with T as built (p the outer collider, q its partner).  The row sum over q
// with g is shared by the species; 32 cells per warp as above, the S outer tiles next to g in shared
// memory.  F layout [S][cells][R].
constexpr int kMaxSpecies = 4;
constexpr int kFewCells = 4;   // batches up to this size take one warp per cell

__global__ void __launch_bounds__(128) contract_fp64_species_kernel(
    const double *__restrict__ T, const int *__restrict__ qlo, const int *__restrict__ qhi,
    const int *__restrict__ prange, int R, int P, int S, const double *__restrict__ gs,
    const double *__restrict__ g, int n_cells, double *__restrict__ F)
{
    extern __shared__ double gsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const long long cell0 = ((long long)blockIdx.x * nwarps + warp) * 32;
    double *gw = gsm + (size_t)warp * P * 32 * (1 + S);   // g, then the S outer tiles
    for (int t = 0; t <= S; ++t) {
        const double *src = t == 0 ? g : gs + (size_t)(t - 1) * n_cells * P;
        double *dst = gw + (size_t)t * P * 32;
        for (int idx = lane; idx < 32 * P; idx += 32) {
            const int c = idx / P, q = idx - c * P;
            const long long cell = cell0 + c;
            dst[q * 32 + c] = cell < n_cells ? src[cell * P + q] : 0.0;
        }
    }
    __syncwarp();
    const long long cell = cell0 + lane;
    const int r_per = (R + gridDim.y - 1) / gridDim.y;
    const int r_begin = blockIdx.y * r_per, r_end = min(R, r_begin + r_per);
    for (int r = r_begin; r < r_end; ++r) {
        const int p0 = prange[2 * r], p1 = prange[2 * r + 1];
        double Fr[kMaxSpecies] = {0.0, 0.0, 0.0, 0.0};
        for (int p = p0; p < p1; ++p) {
            const int q0 = qlo[r * P + p], q1 = qhi[r * P + p];
            if (q0 >= q1) continue;
            const double *Trow = T + ((size_t)r * P + p) * P;
            double y0 = 0.0, y1 = 0.0;
            int q = q0;
            for (; q + 1 < q1; q += 2) {
                y0 = fma(__ldg(Trow + q), gw[q * 32 + lane], y0);
                y1 = fma(__ldg(Trow + q + 1), gw[(q + 1) * 32 + lane], y1);
            }
            if (q < q1) y0 = fma(__ldg(Trow + q), gw[q * 32 + lane], y0);
            const double y = y0 + y1;
#pragma unroll
            for (int sp = 0; sp < kMaxSpecies; ++sp)
                if (sp < S) Fr[sp] = fma(gw[(size_t)(1 + sp) * P * 32 + p * 32 + lane], y, Fr[sp]);
        }
        if (cell < n_cells)
#pragma unroll
            for (int sp = 0; sp < kMaxSpecies; ++sp)
                if (sp < S) F[((size_t)sp * n_cells + cell) * R + r] = Fr[sp];
    }
}

}  // namespace

cudaError_t launch_contract_fp64_species(const DevGroup &g, const double *d_T, const int *d_qlo, const int *d_qhi,
                                         const int *d_prange, int S, const double *d_gs, const double *d_g,
                                         int n_cells, double *d_F, cudaStream_t st)
{
    if (S < 1 || S > kMaxSpecies) return cudaErrorInvalidValue;
    const size_t per_warp = (size_t)g.P * 32 * sizeof(double) * (1 + S);
    int wpb = (int)((200 * 1024) / per_warp);
    if (wpb > 4) wpb = 4;
    if (wpb < 1) return cudaErrorInvalidValue;
    const size_t smem = per_warp * wpb;
    cudaError_t e = cudaFuncSetAttribute(contract_fp64_species_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int cells_per_block = 32 * wpb;
    const int blocks = (n_cells + cells_per_block - 1) / cells_per_block;
    const dim3 grid(blocks, fp64_functional_chunks(n_cells, g.R));
    contract_fp64_species_kernel<<<grid, 32 * wpb, smem, st>>>(d_T, d_qlo, d_qhi, d_prange, g.R, g.P, S, d_gs, d_g,
                                                               n_cells, d_F);
    return cudaGetLastError();
}

int fp64_functional_chunks(int n_cells, int R)
{
    // enough warps for about 8 per SM; larger batches keep one pass over all functionals
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const long long warps = ((long long)n_cells + 31) / 32, want = 8LL * n_sm;
    if (warps >= want) return 1;
    return (int)std::min<long long>(R, (want + warps - 1) / warps);
}

cudaError_t launch_contract_fp64(const DevGroup &g, const double *d_T, const int *d_qlo, const int *d_qhi,
                                 const int *d_prange, const double *d_g, int n_cells, double *d_F,
                                 cudaStream_t st)
{
    if (n_cells <= kFewCells) {
        // one warp per cell and block; functionals spread over blockIdx.y for about 8 warps per SM
        const size_t smem = (size_t)g.P * sizeof(double);
        cudaError_t e = cudaFuncSetAttribute(contract_fp64_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, n_sm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        const int chunks = std::max(1, std::min(g.R, (8 * n_sm + n_cells - 1) / std::max(n_cells, 1)));
        contract_fp64_kernel<1><<<dim3(std::max(n_cells, 1), chunks), 32, smem, st>>>(d_T, d_qlo, d_qhi, d_prange, g.R,
                                                                                      g.P, d_g, n_cells, d_F);
        return cudaGetLastError();
    }
    const bool wide = (size_t)g.P * 32 * sizeof(double) > 200 * 1024;   // 32-cell tile too large
    const int cpw = wide ? 8 : 32;
    const size_t per_warp = (size_t)g.P * cpw * sizeof(double);
    int wpb = (int)((200 * 1024) / per_warp);
    if (wpb > 4) wpb = 4;
    if (wpb < 1) return cudaErrorInvalidValue;   // P too large even for 8 cells per warp
    const size_t smem = per_warp * wpb;
    // the attribute belongs to the current device, so it is set on every launch
    cudaError_t e = wide ? cudaFuncSetAttribute(contract_fp64_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem)
                         : cudaFuncSetAttribute(contract_fp64_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem);
    if (e != cudaSuccess) return e;
    const int cells_per_block = cpw * wpb;
    const int blocks = (n_cells + cells_per_block - 1) / cells_per_block;
    const dim3 grid(blocks, fp64_functional_chunks(n_cells, g.R));
    if (wide)
        contract_fp64_kernel<8><<<grid, 32 * wpb, smem, st>>>(d_T, d_qlo, d_qhi, d_prange, g.R, g.P, d_g, n_cells, d_F);
    else
        contract_fp64_kernel<32><<<grid, 32 * wpb, smem, st>>>(d_T, d_qlo, d_qhi, d_prange, g.R, g.P, d_g, n_cells, d_F);
    return cudaGetLastError();
}

}  // namespace grace
