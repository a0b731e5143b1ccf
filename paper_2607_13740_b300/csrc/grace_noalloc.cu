// grace_rhs_noalloc: the FP64 right-hand side without any device allocation.
//
// The regular grace_rhs keeps its flux-functional workspace in memory that
// grace_bind_batch allocates.  Some callers cannot allocate device memory:
// codes whose device memory is owned by another framework's pool allocator,
// and solvers that call the RHS from a per-substep loop where a cudaMalloc
// (which synchronises the device) or a second allocator is not acceptable.
// For them this entry point keeps the workspace in a fixed array that lives
// in this file's module for as long as the library stays loaded.
#include <string>

#include "grace_internal.h"

namespace grace {
namespace {

// Workspace of the flux functionals F[cell][R] in FP64: 16 MiB per GPU that loads the library.
constexpr size_t kStaticScratchDoubles = size_t(2) << 20;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

// Device address of the array on the current device.  It is looked up on every call (a host-side
// query, no allocation), so a context torn down and re-created (cudaDeviceReset) never leaves a
// stale address behind.  The first lookup on a device may load the library's device code there,
// which is why the first call must come before any stream capture.
grace_status scratch_on_device(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "grace_rhs_noalloc: cudaGetSymbolAddress");
    *out = static_cast<double *>(p);
    return GRACE_OK;
}

}  // namespace
}  // namespace grace

using namespace grace;

extern "C" grace_status grace_rhs_noalloc(grace_ctx *ctx, int group, int n_cells, const double *g, double *L)
{
    if (!ctx || !g || !L || n_cells < 1 || group < 0 || group >= (int)ctx->groups.size()) {
        set_error("grace_rhs_noalloc: null pointer, n_cells < 1 or group out of range");
        return GRACE_ERR_ARG;
    }
    if (!ctx->precomputed) {
        set_error("grace_rhs_noalloc: call grace_precompute first");
        return GRACE_ERR_ORDER;
    }
    const Group &G = ctx->groups[group];
    if (G.dg.cell_alpha) {
        set_error("grace_rhs_noalloc: groups with a per-cell kernel parameter are not supported");
        return GRACE_ERR_UNSUPPORTED;
    }
    const size_t need = (size_t)n_cells * (size_t)G.dg.R;
    if (need > kStaticScratchDoubles) {
        set_error("grace_rhs_noalloc: n_cells * n_functionals = " + std::to_string(need) +
                  " exceeds the fixed workspace of " + std::to_string(kStaticScratchDoubles) +
                  " doubles; at most " + std::to_string(kStaticScratchDoubles / G.dg.R) +
                  " cells per call for this group");
        return GRACE_ERR_ARG;
    }
    cudaGetLastError();   // clear a stale error of an earlier, unrelated call
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return cuda_fail(e, "grace_rhs_noalloc: cudaGetDevice");
    if (prev != ctx->device && (e = cudaSetDevice(ctx->device)) != cudaSuccess)
        return cuda_fail(e, "grace_rhs_noalloc: cudaSetDevice");
    double *F = nullptr;
    grace_status s = scratch_on_device(&F);
    if (s == GRACE_OK) {
        e = launch_contract_fp64(G.dg, G.d_T, G.d_qlo, G.d_qhi, G.d_prange, g, n_cells, F, ctx->stream);
        if (e == cudaSuccess) {
            UpdateArgs u;
            u.F = F;
            u.gout = L;
            e = launch_update(G.dg, u, n_cells, ctx->stream);
        }
        if (e != cudaSuccess) s = cuda_fail(e, "grace_rhs_noalloc: launch");
    }
    if (prev != ctx->device) cudaSetDevice(prev);
    return s;
}
