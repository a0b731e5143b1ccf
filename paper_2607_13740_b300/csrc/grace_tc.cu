// K-b: tensor-core (tcgen05) contraction of the flux functionals.  (in progress)
#include "grace_internal.h"
#include "grace_tc_layout.cuh"

namespace grace {

void free_tc_tiles(TcTiles &t)
{
    cudaFree(t.d_b);
    cudaFree(t.d_desc);
    t = TcTiles();
}

size_t opA_bytes_for(const DevGroup &g, int prec, int n_cells, int *kpad)
{
    const int ae = atom_elems(prec);
    const int kp = (g.P + ae - 1) / ae * ae;
    if (kpad) *kpad = kp;
    const size_t tiles = ((size_t)n_cells + kTileM - 1) / kTileM;
    return tiles * opA_tile_bytes(prec, kp);
}

grace_status build_tc_tiles(Group &G, int prec, cudaStream_t st)
{
    (void)G;
    (void)prec;
    (void)st;
    set_error("tensor-core contraction not available in this build");
    return GRACE_ERR_UNSUPPORTED;
}

cudaError_t launch_contract_tc(const DevGroup &, const TcTiles &, int, const void *, int, float *, int *,
                               cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace grace
