// K-b: tensor-core contraction of the flux functionals on tcgen05 / TMEM.
//
// Every flux functional of a cell is a quadratic form of its coefficients,
//     F_r = sum_{p,q} T_r[p,q] g_p g_q                     (see grace_precompute.cu).
// Only the symmetric part of T_r matters, so it is folded onto the upper
// triangle, U_r[p,q] = T_r[p,q] + T_r[q,p] (q > p), U_r[p,p] = T_r[p,p], which
// halves the multiply-adds.  Over a batch the contraction is one GEMM per tile
// of 128 cells, factorised as
//     Y[c, (r,p)] = sum_{q >= p} ghat[c, q] * Uhat_r[p, q]    (tcgen05.mma, FP32 in TMEM)
//     F[c, r]     = sum_p        ghat[c, p] * Y[c, (r,p)]     (epilogue, one lane per cell)
// with ghat = g * h_bin (bin-mass scaling) and Uhat = U / (h_bin(p) h_bin(q)), so
// operands stay in a comfortable FP32/BF16 range for grids spanning 16 decades.
//
// An N-tile of the GEMM is a run of nf consecutive functionals (in bin order)
// times a window of 16 consecutive p (N = 16 nf <= 256); its K range is the union of
// the non-zero q extents of its rows, so the zero blocks of the staircase
// support are skipped.  One tcgen05.mma with M = 128 costs about the same time
// for any N on this part, so tiles are made as wide as the support allows; the
// grouping of functionals (hence N) is chosen by a dynamic program over a cost
// model (MMA issue, B-operand L2 traffic and the epilogue), i.e. the tile
// shapes are autotuned from T's sparsity.
//
// B (the tables) lives in global memory as ready-made shared-memory images, one
// block of N rows x 32 bytes per MMA k-step in the K-major SWIZZLE_32B layout;
// A (the cells' coefficients) as 128-row K-major SWIZZLE_128B tiles
// (grace_tc_layout.cuh).  Both move with cp.async.bulk (no tensor map).
//
// Warp roles (persistent, one CTA per SM, work items round-robin):
//   warps 0, 3    : B bulk-copy producers (lane 0), copies (up to 64 KB) alternating between the two issuers
//   warp 2 lane 0 : A-tile loader (after allocating TMEM)
//   warp 1        : MMA issuer (kind::tf32, or kind::f16 with bf16 hi/lo x3), converged, lane 0 issues
//   warp 2        : TMEM allocation / release (2 accumulators x 256 columns)
//   warps 4..19   : epilogue; TMEM lane quadrant = warp % 4, four warps per quadrant
//                   splitting the functionals of a tile; one cell per thread
// A work item is one 128-cell tile and a contiguous range of N-tiles (a split):
// splitting the tile list lets a batch of few cell tiles fill every SM.  Items are
// numbered split-major (item = split x cell tiles + cell tile) so that the
// round-robin assignment gives every CTA a mix of splits.
// Node-space tiles (groups with a per-cell kernel parameter, template NC): A holds the cells'
// values at the fixed Gauss nodes, the MMA contracts over the smaller node of each pair, and the
// epilogue weights the accumulator by the fragmentation ramp of the larger node (epi_tile_nc).
// Launch forms (template FORM): one CTA per work item with A in shared memory (the default); CTA
// pairs (cta_group::2, M = 256 over the two SMs of a cluster, grace_set_cta_pairs); A in tensor
// memory (tcgen05.cp of the A tile from a ring slot, grace_set_tc_a_in_tmem).  All three run the
// same tile schedule; the last two measured slower on this part and are off by default.
// Every wait on an mbarrier is bounded; on timeout the CTA records an error in
// the device error word, stops issuing work, drains its outstanding copies and
// releases its tensor memory before returning.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "grace_internal.h"
#include "grace_tc_layout.cuh"

namespace grace {

namespace {

constexpr int kWin = 16;            // p window width of every N tile
constexpr int kMaxF = 16;           // functionals per N tile (kMaxF * kWin = 256)
constexpr int kMaxN = 256;          // MMA N
constexpr int kMaxSlots = 8;        // B ring depth, sized at launch from free shared memory
constexpr int kAccCols = 256;       // TMEM columns per accumulator buffer
constexpr int kTmemCols = 512;      // two accumulator buffers
constexpr int kEpiWarps = 16;   // four per TMEM lane quadrant: the epilogue, not the MMA, set the pace with eight
constexpr int kEpiSplit = kEpiWarps / 4;   // epilogue warps per TMEM lane quadrant
constexpr int kEpiF = (kMaxF + kEpiSplit - 1) / kEpiSplit;   // functionals per epilogue warp and tile
constexpr int kThreads = 32 * (4 + kEpiWarps);
constexpr int kMaxSplits = 8;
constexpr int kSmemLimit = 227 * 1024;
constexpr long long kWaitCycles = 4000000000LL;   // default wait limit, ~2 s at 2 GHz

// cost model (SM cycles), from measurements on this part: in isolation (grace_probe_mma) one
// tcgen05.mma with M = 128 and N columns (K = 32 bytes) takes ~0.543 N cycles for N >= 128 (139 at
// N = 256, 69 at N = 128); inside this kernel the time per instruction hardly falls with N (tiles
// planned for N <= 128 ran 20 % slower than N <= 256 tiles with 13 % more multiply-adds: issue and
// operand delivery per instruction, not the tensor rate, set the pace), so an instruction is
// charged its N = 256 time whatever its N; L2 delivers ~45 B/cycle/SM to the B ring
constexpr double kMmaClk = 139.0;
constexpr double kL2BytesPerClk = 45.0;
constexpr double kTileClk = 60.0;        // accumulator hand-off per tile
constexpr double kEpiBaseClk = 250.0;    // epilogue per tile: fixed part (TMEM round trip, window load)
constexpr double kEpiColClk = 5.5;       // epilogue per tile and accumulator column (8 warps)
constexpr double kItemClk = 2500.0;      // A tile load + pipeline fill per work item

struct TileDesc {
    int b_off16;        // offset of the tile's first k-step block in the B images, in 16-byte units
    int n;              // MMA N = (nf - fs) * rows per functional
    int nf_flush;       // nf | fs << 8 | flush << 16: the group's functionals ford[f0 .. f0 + nf), of
                        // which fs .. nf - 1 have rows in this window (accumulator columns from fs
                        // on); flush: last window of the group (write F)
    int acol;           // A-operand column of the window's first coefficient (p0 + the A column offset)
    int p0;             // first p of the window
    int ks_lo, ks_hi;   // MMA k-steps [ks_lo, ks_hi)
    int f0;             // first functional (index into the functional order)
};
static_assert(sizeof(TileDesc) == 32, "TileDesc layout");

struct TcParams {
    const TileDesc *tiles;
    const int *ford;
    int n_tiles;
    int table_bytes;      // shared-memory copy of tiles + ford
    const uint8_t *B;
    const uint8_t *A;
    long long a_tile_bytes;
    int n_cells;
    int n_cell_tiles;
    int n_pair_tiles;     // CTA pairs: pairs of cell tiles (the last one may have no odd tile)
    // TMEM columns of accumulator buffer 0 and the distance to buffer 1; with A in TMEM, the
    // columns of one A plane (A occupies [0, planes x at_plane_cols))
    int acc_base, acc_stride, at_plane_cols;
    int R;
    float *F;
    int slot_bytes;       // bytes of one ring slot
    int kps;              // MMA k-steps per B copy
    int n_slots;          // ring depth
    int a_bufs;           // A tiles in shared memory (2: the next item's A loads during this one)
    int n_splits;
    int split[kMaxSplits + 1];
    int *err;
    // node-space tiles (per-cell kernels): ramp of the epilogue
    const float *D0;      // [n_d0] D0 of every fixed node
    int n_d0;
    const float *cell_s;  // [n_cells] s = sqrt(alpha)
    float ramp_a, ramp_b;
    // VJP tiles: functional weights mu in the [tile][R][128] layout, output planes
    // W[part][tile][Pw][128] (one per epilogue warp of a lane quadrant)
    const float *mu;
    float *W;
    int Pw;
    // multi-group mode: per-group descriptors and the work items (group, cell tile)
    const struct TcGroupDesc *groups;
    const int2 *items;
    // species mode: the species' scaled coefficients ghat_s in FP32, [S][cell tile][gsp_kpad][128]
    // (A columns, one 128-cell column per coefficient), and F_s at F + s f_sstride
    const float *gsp;
    long long gsp_sstride, f_sstride;
    int gsp_kpad, n_species;
    // failure detection: every mbarrier wait gives up after wait_cycles; withhold_b != 0 (a
    // test of that path only) issues no B copies, so the MMA issuer's first wait runs out
    long long wait_cycles;
    int withhold_b;
};

// one group of a multi-group launch (all its tiles form one split)
struct TcGroupDesc {
    const TileDesc *tiles;
    const int *ford;
    const uint8_t *B;
    const uint8_t *Bp;   // CTA-pair images of B (null when the group has none)
    const uint8_t *A;
    float *F;
    long long a_tile_bytes;
    int n_cells, R, t0, t1;
};

// contraction modes: flux functionals, node-space functionals (per-cell kernels), VJP, flux
// functionals of many groups in one launch (uneven batches)
constexpr int kModeF = 0, kModeNC = 1, kModeVJP = 2, kModeMulti = 3, kModeSpecies = 4;
constexpr int kMaxSpeciesTc = 4;   // species of mixed grains per launch

// the parameters of one work item: its group's tiles, operands and output, its tile range
struct ItemCtx {
    const TileDesc *tiles;
    const int *ford;
    const uint8_t *B;
    const uint8_t *A;        // the item's A tile in global memory
    float *F;
    long long a_bytes;
    int n_cells, R, t0, t1, ct;
};

// Work item `it`: a cell tile (or, for a CTA pair, the pair's cell tiles 2u and 2u + 1, this CTA taking
// 2u + rank) and a split of the tile list.  A pair without an odd tile loads the even tile's A again
// (its results are never written: no cell of that tile is live).
template <int MODE, int PAIR = 0>
__device__ __forceinline__ ItemCtx item_ctx(const TcParams &P, int it, const TileDesc *tiles, const int *ford,
                                            uint32_t rank = 0)
{
    ItemCtx c;
    if (MODE == kModeMulti) {
        // item (group, cell tile), or for a CTA pair (group, pair of the group's cell tiles)
        const int2 v = P.items[it];
        const TcGroupDesc &g = P.groups[v.x];
        const int n_ct = (g.n_cells + kTileM - 1) / kTileM;
        const int ct = PAIR ? 2 * v.y + (int)rank : v.y;
        c.tiles = g.tiles;
        c.ford = g.ford;
        c.B = PAIR ? g.Bp : g.B;
        c.a_bytes = g.a_tile_bytes;
        c.A = g.A + (size_t)(ct < n_ct ? ct : ct - 1) * g.a_tile_bytes;
        c.F = g.F;
        c.n_cells = g.n_cells;
        c.R = g.R;
        c.t0 = g.t0;
        c.t1 = g.t1;
        c.ct = ct;
    } else {
        const int nu = PAIR ? P.n_pair_tiles : P.n_cell_tiles;
        const int sp = it / nu, u = it - sp * nu;
        const int ct = PAIR ? 2 * u + (int)rank : u;
        const int ct_a = ct < P.n_cell_tiles ? ct : ct - 1;
        c.tiles = tiles;
        c.ford = ford;
        c.B = P.B;
        c.a_bytes = P.a_tile_bytes;
        c.A = P.A + (size_t)ct_a * P.a_tile_bytes;
        c.F = P.F;
        c.n_cells = P.n_cells;
        c.R = P.R;
        c.t0 = P.split[sp];
        c.t1 = P.split[sp + 1];
        c.ct = ct;
    }
    return c;
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// acquire at cluster scope: for barriers that the other CTA of a pair arrives on
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false on timeout or when another role (of this CTA or, for CTA pairs, of the
// peer) already aborted
template <int CLUSTER = 0>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, long long limit)
{
    const long long t0 = clock64();
    while (!(CLUSTER ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity))) {
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// ---- CTA pairs (cta_group::2): one tcgen05.mma with M = 256 runs on the tensor cores of both SMs of
// a 2-CTA cluster.  Each CTA holds its own 128 rows (cells) of A and one half of the rows of every B
// k-step block (the even-ranked CTA the first N / 2), at the same shared-memory offsets; each CTA's
// TMEM receives its own 128 x N accumulator.  Only the even-ranked CTA issues.
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared::cluster address of the same shared-memory variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// tcgen05.commit by the lanes with `issue` != 0 (the MMA warp runs converged; one lane issues).  For a
// CTA pair the commit arrives on the barrier at the same offset in every CTA of `mask`.
template <int PAIR = 0>
__device__ __forceinline__ void tc_commit_if(uint32_t bar, uint32_t issue, uint16_t mask = 3)
{
    if (PAIR)
        asm volatile(
            "{\n\t.reg .pred e;\n\tsetp.ne.b32 e, %1, 0;\n\t"
            "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %2;\n\t}" ::"r"(bar),
            "r"(issue), "h"(mask)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred e;\n\tsetp.ne.b32 e, %1, 0;\n\t"
            "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(bar),
            "r"(issue)
            : "memory");
}

// K-major shared-memory matrix descriptors: SWIZZLE_128B (A: 128-byte rows, 8-row groups 1024 B
// apart) and SWIZZLE_32B (B: 32-byte rows, 8-row groups 256 B apart).  The low 32 bits hold the
// start address >> 4 (14 bits) and the leading-byte-offset field (1); the high 32 bits the
// stride-byte offset >> 4, the descriptor version (bit 46) and the swizzle mode (bits 61-63);
// these high halves are the same for every operand of a kind:
constexpr uint32_t kDescHi128 = (1024u >> 4) | (1u << 14) | (2u << 29);
constexpr uint32_t kDescHi32 = (256u >> 4) | (1u << 14) | (6u << 29);

// instruction descriptor: FP32 accumulate, K-major A and B, M = m (128, or 256 for a CTA pair), N = n
__device__ __forceinline__ uint32_t instr_desc(int prec, int n, int m = 128)
{
    const uint32_t fmt = prec == GRACE_TF32 ? 2u : 1u;   // TF32 = 2, BF16 = 1
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// tcgen05.mma (kind::tf32, or kind::f16 with bf16 operands) with the operand descriptors given as
// their two 32-bit halves, issued by the lanes with `issue` != 0.  Only the low half (start
// address >> 4 | leading-byte-offset field) changes from one k-step to the next, so the issuing
// warp advances it with one 32-bit add per operand: measured on this part, an issue loop that
// rebuilds 64-bit descriptors per instruction keeps the tensor pipe about half idle.  The whole
// warp runs the issue loop (converged) and one lane's instructions are predicated on: a loop run
// by a lone lane of a diverged warp leaves the tensor pipe idle for ~400 cycles at every exit
// and re-entry of its inner loop (~200 for a converged warp), measured with groups of 11
// instructions.
template <int PREC, int PAIR = 0>
__device__ __forceinline__ void mma_lohi(uint32_t d, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo, uint32_t b_hi,
                                         uint32_t idesc, uint32_t acc, uint32_t issue)
{
    if (PAIR && PREC == GRACE_TF32)
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t.reg .b64 da, db;\n\t"
            "setp.ne.b32 p, %6, 0;\n\tsetp.ne.b32 e, %7, 0;\n\t"
            "mov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
            "@e tcgen05.mma.cta_group::2.kind::tf32 [%0], da, db, %5, p;\n\t}" ::"r"(d),
            "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(acc), "r"(issue)
            : "memory");
    else if (PAIR)
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t.reg .b64 da, db;\n\t"
            "setp.ne.b32 p, %6, 0;\n\tsetp.ne.b32 e, %7, 0;\n\t"
            "mov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
            "@e tcgen05.mma.cta_group::2.kind::f16 [%0], da, db, %5, p;\n\t}" ::"r"(d),
            "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(acc), "r"(issue)
            : "memory");
    else if (PREC == GRACE_TF32)
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t.reg .b64 da, db;\n\t"
            "setp.ne.b32 p, %6, 0;\n\tsetp.ne.b32 e, %7, 0;\n\t"
            "mov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
            "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], da, db, %5, p;\n\t}" ::"r"(d),
            "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(acc), "r"(issue)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t.reg .b64 da, db;\n\t"
            "setp.ne.b32 p, %6, 0;\n\tsetp.ne.b32 e, %7, 0;\n\t"
            "mov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}" ::"r"(d),
            "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(acc), "r"(issue)
            : "memory");
}

// A operand in tensor memory: tcgen05.cp of one k-step of A (128 rows x 32 bytes, the same K-major
// 128-byte-swizzled shared-memory descriptor as the MMA's A operand) into 8 TMEM columns, and
// tcgen05.mma reading A from TMEM (lane = cell, K packed along the columns), by the lanes with
// `issue` != 0.
__device__ __forceinline__ void tc_cp_a(uint32_t taddr, uint32_t desc_lo, uint32_t desc_hi, uint32_t issue)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t.reg .b64 d;\n\tsetp.ne.b32 e, %3, 0;\n\tmov.b64 d, {%1, %2};\n\t"
        "@e tcgen05.cp.cta_group::1.128x256b [%0], d;\n\t}" ::"r"(taddr),
        "r"(desc_lo), "r"(desc_hi), "r"(issue)
        : "memory");
}

template <int PREC>
__device__ __forceinline__ void mma_tmem_a(uint32_t d, uint32_t a_t, uint32_t b_lo, uint32_t b_hi, uint32_t idesc,
                                           uint32_t acc, uint32_t issue)
{
    if (PREC == GRACE_TF32)
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t.reg .b64 db;\n\t"
            "setp.ne.b32 p, %5, 0;\n\tsetp.ne.b32 e, %6, 0;\n\tmov.b64 db, {%2, %3};\n\t"
            "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], db, %4, p;\n\t}" ::"r"(d),
            "r"(a_t), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(acc), "r"(issue)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t.reg .b64 db;\n\t"
            "setp.ne.b32 p, %5, 0;\n\tsetp.ne.b32 e, %6, 0;\n\tmov.b64 db, {%2, %3};\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], db, %4, p;\n\t}" ::"r"(d),
            "r"(a_t), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(acc), "r"(issue)
            : "memory");
}

// TMEM -> registers, 32 lanes x 16 / 32 columns, no wait
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- kernel
struct Smem {
    uint64_t a_full[2], a_empty[2];
    uint64_t full[kMaxSlots], empty[kMaxSlots];
    uint64_t peer_a_full[2], peer_full[kMaxSlots];   // CTA pairs: the odd CTA's A / B halves landed
    uint64_t acc_full[2], acc_empty[2];
    uint64_t mma_drain;
    uint64_t a_free;             // A in TMEM: the MMAs of a work item have retired
    uint32_t tmem_base;
    int abort_flag;
    int slot_issued[kMaxSlots];  // copies issued per slot (producer)
    int slot_done[kMaxSlots];    // copies consumed per slot (MMA)
    int a_issued[2], a_done[2];
    int items_done;              // work items the epilogue finished
};

// records a failure and stops every role of this CTA (and of the peer CTA of a pair)
template <int PAIR = 0>
__device__ __forceinline__ void fail(const TcParams &P, volatile int *abort_flag, int code)
{
    if (P.err) atomicOr(P.err, code);
    *abort_flag = 1;
    if (PAIR) {
        const uint32_t peer = cluster_addr(smem_u32((const void *)abort_flag), cluster_rank() ^ 1u);
        asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(peer), "r"(1) : "memory");
    }
}

// One tile of the epilogue for a p window of width W: loads the cell's ghat
// window [p0, p0 + W) from its A tile in shared memory, then adds to Facc[m]
// (functional f = kEpiSplit m + part of the tile) the sum over the functional's W
// accumulator columns times the window; G functionals' TMEM loads are in
// flight before each wait.
template <int PREC, int W>
__device__ __forceinline__ void load_window(const uint8_t *a_gen, long long a_tile_bytes, int row, int p0, float *gw)
{
    // columns of the tile (TF32: 128 rows x 4 bytes, BF16: 128 rows x 2 planes x 2 bytes per column);
    // 16-byte chunks at or past the last column read as zeros (a window may reach past the padded row
    // when the A column offset is not zero; its coefficients there are absent)
    const int kcols = (int)(a_tile_bytes / (kTileM * 4));
    if (PREC == GRACE_TF32) {
#pragma unroll
        for (int c = 0; c < W / 4; ++c) {
            if (p0 + 4 * c >= kcols) {
                gw[4 * c] = gw[4 * c + 1] = gw[4 * c + 2] = gw[4 * c + 3] = 0.f;
                continue;
            }
            const float4 v = *reinterpret_cast<const float4 *>(a_gen + swz_offset(kTileM, row, p0 + 4 * c, 4));
            gw[4 * c] = v.x;
            gw[4 * c + 1] = v.y;
            gw[4 * c + 2] = v.z;
            gw[4 * c + 3] = v.w;
        }
    } else {
        const size_t lo_plane = (size_t)(a_tile_bytes / 2);
#pragma unroll
        for (int c = 0; c < W / 8; ++c) {
            if (p0 + 8 * c >= kcols) {
#pragma unroll
                for (int e = 0; e < 8; ++e) gw[8 * c + e] = 0.f;
                continue;
            }
            const size_t off = swz_offset(kTileM, row, p0 + 8 * c, 2);
            const uint4 hi = *reinterpret_cast<const uint4 *>(a_gen + off);
            const uint4 lo = *reinterpret_cast<const uint4 *>(a_gen + lo_plane + off);
            const uint32_t hw[4] = {hi.x, hi.y, hi.z, hi.w}, lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                gw[8 * c + 2 * e] = __uint_as_float(hw[e] << 16) + __uint_as_float(lw[e] << 16);
                gw[8 * c + 2 * e + 1] = __uint_as_float(hw[e] & 0xFFFF0000u) + __uint_as_float(lw[e] & 0xFFFF0000u);
            }
        }
    }
}

// Releases an accumulator buffer to the MMA warp once this warp's TMEM reads of it are complete (for a
// CTA pair, on the even CTA's barrier: its MMAs write both CTAs' accumulators).
template <int PAIR = 0>
__device__ __forceinline__ void release_acc(uint32_t bar, int lane)
{
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
        if (PAIR) mbar_arrive_remote(cluster_addr(bar, 0u));
        else mbar_arrive(bar);
    }
}

// The window gw is loaded before the accumulator is ready; the accumulator buffer is released
// (acc_empty) right after the last TMEM wait, before the last FMAs.
template <int W, int G, int PAIR>
__device__ __forceinline__ void epi_tile(const float *gw, uint32_t tcol, int nf, int fs, int part, float *Facc,
                                         uint32_t acc_empty, int lane)
{
    bool released = false;
#pragma unroll
    for (int m0 = 0; m0 < kEpiF; m0 += G) {
        if (kEpiSplit * m0 + part >= nf) break;
        if (kEpiSplit * (m0 + G - 1) + part < fs) continue;
        const bool last = m0 + G >= kEpiF || kEpiSplit * (m0 + G) + part >= nf;
        uint32_t y[G][W];
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
            const int f = kEpiSplit * (m0 + gg) + part;
            if (f >= fs && f < nf) {
                if (W == 32) tmem_ld32(tcol + (uint32_t)((f - fs) * W), y[gg]);
                else tmem_ld16(tcol + (uint32_t)((f - fs) * W), y[gg]);
            }
        }
        tmem_wait_ld();
        if (last) {
            release_acc<PAIR>(acc_empty, lane);
            released = true;
        }
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
            const int f = kEpiSplit * (m0 + gg) + part;
            if (f >= fs && f < nf) {
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int c = 0; c < W; c += 2) {
                    s0 = fmaf(gw[c], __uint_as_float(y[gg][c]), s0);
                    s1 = fmaf(gw[c + 1], __uint_as_float(y[gg][c + 1]), s1);
                }
                Facc[m0 + gg] += s0 + s1;
            }
        }
    }
    if (!released) release_acc<PAIR>(acc_empty, lane);
}

// Epilogue of a species tile (mixtures of Sec. 5.3): the accumulator holds, for the cell's total
// g in the partner slot, Y[c, (r, p)] = sum_q ghat_q That_r[p, q] (T as built, p the outer
// collider); species s contracts it with its own window ghat_{s, p} (FP32 from global memory,
// 128 cells per coefficient column, so a warp reads 128 contiguous bytes per coefficient).
template <int W>
__device__ __forceinline__ void epi_tile_species(const float *gsp_ct, long long sstride, int n_species, int kpad,
                                                 int row, int acol, uint32_t tcol, int nf, int fs, int part,
                                                 float (*FaccS)[kEpiF])
{
#pragma unroll
    for (int sp = 0; sp < kMaxSpeciesTc; ++sp) {
        if (sp >= n_species) break;
        float gw[W];
        const float *src = gsp_ct + (size_t)sp * sstride + (size_t)acol * kTileM + row;
#pragma unroll
        for (int c = 0; c < W; ++c) gw[c] = acol + c < kpad ? __ldg(src + (size_t)c * kTileM) : 0.f;   // the last
        // window of a group may run past the padded K extent (its accumulator columns there are zero)
#pragma unroll
        for (int m0 = 0; m0 < kEpiF; ++m0) {
            const int f = kEpiSplit * m0 + part;
            if (f >= nf) break;
            if (f < fs) continue;
            uint32_t y[W];
            if (W == 32) tmem_ld32(tcol + (uint32_t)((f - fs) * W), y);
            else tmem_ld16(tcol + (uint32_t)((f - fs) * W), y);
            tmem_wait_ld();
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int c = 0; c < W; c += 2) {
                s0 = fmaf(gw[c], __uint_as_float(y[c]), s0);
                s1 = fmaf(gw[c + 1], __uint_as_float(y[c + 1]), s1);
            }
            FaccS[sp][m0] += s0 + s1;
        }
    }
}

// Epilogue of a node-space tile (per-cell kernels).  Accumulator columns [32 f, 32 f + 16) of
// functional f hold, for the window's 16 larger nodes j, the coagulation sums over the smaller
// node, columns [32 f + 16, 32 f + 32) the fragmentation sums; they are weighted by
// s (1 - pf_j) Ghat_j and s pf_j Ghat_j, pf_j = clamp(ra s D0_j + rb, 0, 1), with Ghat_j the
// cell's node value from its A tile.
constexpr int kEpiFnc = (kMaxN / (2 * kWin) + kEpiSplit - 1) / kEpiSplit;

template <int PREC, int G>
__device__ __forceinline__ void epi_tile_nc(const uint8_t *a_gen, long long a_tile_bytes, int row, int p0,
                                            uint32_t tcol, int nf, int fs, int part, float s, const float *D0,
                                            float ra, float rb, float *Facc)
{
    float wc[kWin], wf[kWin];
    load_window<PREC, kWin>(a_gen, a_tile_bytes, row, p0, wc);
#pragma unroll
    for (int t = 0; t < kWin; ++t) {
        const float pf = fminf(fmaxf(fmaf(s * D0[p0 + t], ra, rb), 0.f), 1.f);
        const float sg = s * wc[t];
        wf[t] = pf * sg;
        wc[t] = sg - wf[t];
    }
#pragma unroll
    for (int m0 = 0; m0 < kEpiFnc; m0 += G) {
        if (kEpiSplit * m0 + part >= nf) break;
        if (kEpiSplit * (m0 + G - 1) + part < fs) continue;
        uint32_t y[G][2 * kWin];
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
            const int f = kEpiSplit * (m0 + gg) + part;
            if (f >= fs && f < nf) tmem_ld32(tcol + (uint32_t)((f - fs) * 2 * kWin), y[gg]);
        }
        tmem_wait_ld();
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
            const int f = kEpiSplit * (m0 + gg) + part;
            if (f >= fs && f < nf) {
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int t = 0; t < kWin; ++t) {
                    s0 = fmaf(wc[t], __uint_as_float(y[gg][t]), s0);
                    s1 = fmaf(wf[t], __uint_as_float(y[gg][kWin + t]), s1);
                }
                Facc[m0 + gg] += s0 + s1;
            }
        }
    }
}

// Epilogue of a VJP tile (window-major tiles of S_r = T_r + T_r^T): accumulator columns
// [16 f, 16 f + 16) of functional f hold (S_r ghat)_p for the window's 16 coefficients p; the
// functional's weight mu_r times them is added to the window accumulator Wacc.
template <int G>
__device__ __forceinline__ void epi_tile_vjp(uint32_t tcol, int nf, int fs, int part, const float *mu_cell,
                                             const int *ford, int f0, float *Wacc)
{
#pragma unroll
    for (int m0 = 0; m0 < kEpiF; m0 += G) {
        if (kEpiSplit * m0 + part >= nf) break;
        if (kEpiSplit * (m0 + G - 1) + part < fs) continue;
        uint32_t y[G][kWin];
        float mu[G];
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
            const int f = kEpiSplit * (m0 + gg) + part;
            mu[gg] = 0.f;
            if (f >= fs && f < nf) {
                tmem_ld16(tcol + (uint32_t)((f - fs) * kWin), y[gg]);
                mu[gg] = mu_cell[(size_t)ford[f0 + f] * kTileM];
            }
        }
        tmem_wait_ld();
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
            const int f = kEpiSplit * (m0 + gg) + part;
            if (f >= fs && f < nf) {
#pragma unroll
                for (int t = 0; t < kWin; ++t) Wacc[t] = fmaf(mu[gg], __uint_as_float(y[gg][t]), Wacc[t]);
            }
        }
    }
}

// FORM 0: one CTA per work item, A in shared memory.
// FORM 1 (CTA pair): launched in clusters of two CTAs that share every work item (cta_group::2,
// M = 256); the even-ranked CTA issues the MMAs, the odd-ranked CTA's MMA warp relays to it when its
// own A and B halves have landed (its copies arrive on its own barriers), and both epilogues
// release the accumulators on the even CTA's barrier.
// FORM 2 (A in tensor memory): a work item's A tile arrives as the first copy of its stream in a
// ring slot and the MMA warp moves it into TMEM columns [0, planes x at_plane_cols) with
// tcgen05.cp once the previous item's MMAs have retired; the MMAs read A from TMEM, so shared
// memory holds only the ring (three 64 KB slots instead of two beside a 64 KB A tile) and the
// accumulators shrink to 192 columns (N <= 192).  The epilogue reads its ghat windows from the A
// operand in global memory.
template <int PREC, int MODE, int FORM>
__global__ void __launch_bounds__(kThreads, 1) contract_tc_kernel(TcParams P)
{
    constexpr int PAIR = FORM == 1 ? 1 : 0;
    constexpr bool AT = FORM == 2;
    constexpr int planes = PREC == GRACE_TF32 ? 1 : 2;
    const int kps = P.kps;                             // MMA k-steps per B copy
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t a_smem = base;
    const uint32_t b_smem = base + (uint32_t)P.a_bufs * (uint32_t)P.a_tile_bytes;
    uint8_t *tab = gbase + P.a_bufs * P.a_tile_bytes + (size_t)P.n_slots * P.slot_bytes;
    const TileDesc *tiles = reinterpret_cast<const TileDesc *>(tab);
    const int *ford = reinterpret_cast<const int *>(tab + (size_t)P.n_tiles * sizeof(TileDesc));
    const float *D0s = reinterpret_cast<const float *>(ford + P.R);
    Smem *S = reinterpret_cast<Smem *>(tab + P.table_bytes);
    volatile int *abort_flag = &S->abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = P.n_slots;
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const bool lead = rank == 0;
    const int n_items = (PAIR ? P.n_pair_tiles : P.n_cell_tiles) * P.n_splits;
    const int item0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;     // a pair shares its items
    const int item_step = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;

    if (threadIdx.x == 0) {
        // the even CTA of a pair also counts the odd CTA's epilogue warps
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&S->a_full[b]), 1);
            mbar_init(smem_u32(&S->peer_a_full[b]), 1);
            mbar_init(smem_u32(&S->a_empty[b]), 1 + kEpiWarps);
            mbar_init(smem_u32(&S->acc_full[b]), 1);
            mbar_init(smem_u32(&S->acc_empty[b]), (PAIR ? 2 : 1) * kEpiWarps);
            S->a_issued[b] = S->a_done[b] = 0;
        }
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&S->full[s]), 1);
            mbar_init(smem_u32(&S->peer_full[s]), 1);
            mbar_init(smem_u32(&S->empty[s]), 1);
            S->slot_issued[s] = 0;
            S->slot_done[s] = 0;
        }
        mbar_init(smem_u32(&S->mma_drain), 1);
        mbar_init(smem_u32(&S->a_free), 1);
        S->abort_flag = 0;
        S->items_done = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // tile table and functional order into shared memory (read by every role for every tile)
    {
        const int4 *src = reinterpret_cast<const int4 *>(P.tiles);
        int4 *dst = reinterpret_cast<int4 *>(tab);
        for (int i = threadIdx.x; i < P.n_tiles * (int)(sizeof(TileDesc) / 16); i += blockDim.x) dst[i] = src[i];
        int *fo = const_cast<int *>(ford);
        for (int i = threadIdx.x; i < P.R; i += blockDim.x) fo[i] = P.ford[i];
        if (MODE == kModeNC) {
            float *d0 = const_cast<float *>(D0s);
            for (int i = threadIdx.x; i < P.n_d0; i += blockDim.x) d0[i] = P.D0[i];
        }
    }
    if (warp == 2) {
        // a pair allocates collectively (one warp of each CTA), the same columns in both SMs
        if (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&S->tmem_base)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&S->tmem_base)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync_all();   // both CTAs' barriers initialised and TMEM allocated
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == 2) {
        // ------------------------------------------------ A loader (after the TMEM allocation): the
        // next work item's A tile as soon as the previous use of that buffer is released
        int ctl = 0;
        for (int it = item0; it < n_items && !AT; it += item_step, ++ctl) {
            const ItemCtx c = item_ctx<MODE, PAIR>(P, it, tiles, ford, rank);
            const int ab = ctl % P.a_bufs, au = ctl / P.a_bufs;
            int ok = 1;
            if (lane == 0) {
                if (*abort_flag) ok = 0;
                else if (au > 0 && !mbar_wait<PAIR>(smem_u32(&S->a_empty[ab]), (au - 1) & 1, abort_flag, P.wait_cycles)) {
                    fail<PAIR>(P, abort_flag, 1);
                    ok = 0;
                }
                if (ok) {
                    mbar_expect_tx(smem_u32(&S->a_full[ab]), (uint32_t)c.a_bytes);
                    bulk_g2s(a_smem + (uint32_t)ab * (uint32_t)P.a_tile_bytes, c.A, (uint32_t)c.a_bytes,
                             smem_u32(&S->a_full[ab]));
                    S->a_issued[ab] = au + 1;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
        }
    } else if (warp == 0 || warp == 3) {
        // ------------------------------------------------ B producers: copy q is issued by warp 0
        // (q even) or warp 3 (q odd); each issuing thread retires about one bulk copy at a time, so
        // two issuers keep twice as many copies in flight.  The B stream runs ahead across work-item
        // boundaries, limited only by the ring.
        const int me = warp == 0 ? 0 : 1;
        int q = 0;
        for (int it = item0; it < n_items && !P.withhold_b; it += item_step) {
            const ItemCtx ic = item_ctx<MODE, PAIR>(P, it, tiles, ford, rank);
            int ok = *abort_flag ? 0 : 1;
            if (AT) {
                // the item's A tile: the first copy of its stream
                if (lane == 0 && ok && (q & 1) == me) {
                    const int slot = q % NS, use = q / NS;
                    if (use > 0 && !mbar_wait(smem_u32(&S->empty[slot]), (use - 1) & 1, abort_flag, P.wait_cycles)) {
                        fail(P, abort_flag, 2);
                        ok = 0;
                    } else {
                        mbar_expect_tx(smem_u32(&S->full[slot]), (uint32_t)ic.a_bytes);
                        bulk_g2s(b_smem + (uint32_t)slot * (uint32_t)P.slot_bytes, ic.A, (uint32_t)ic.a_bytes,
                                 smem_u32(&S->full[slot]));
                        S->slot_issued[slot] = use + 1;
                    }
                }
                ++q;
                ok = __shfl_sync(0xffffffffu, ok, 0);
            }
            for (int t = ic.t0; t < ic.t1 && ok; ++t) {
                const TileDesc td = ic.tiles[t];
                const int nks = td.ks_hi - td.ks_lo, n_copies = (nks + kps - 1) / kps;
                // a pair's B images hold each tile as [CTA half][k-step][plane][N / 2 rows x 32 B]
                const uint32_t ks_bytes = (uint32_t)td.n * (PAIR ? 16u : 32u) * planes;
                const uint8_t *bsrc = ic.B + (size_t)td.b_off16 * 16 + (PAIR ? (size_t)rank * nks * ks_bytes : 0);
                if (lane == 0)
                    for (int c = 0; c < n_copies; ++c, ++q) {
                        if ((q & 1) != me) continue;
                        const int slot = q % NS, use = q / NS;
                        if (use > 0 && !mbar_wait<PAIR>(smem_u32(&S->empty[slot]), (use - 1) & 1, abort_flag, P.wait_cycles)) {
                            fail<PAIR>(P, abort_flag, 2);
                            ok = 0;
                            break;
                        }
                        const int k0 = c * kps, kn = min(kps, nks - k0);
                        const uint32_t bytes = (uint32_t)kn * ks_bytes;
                        mbar_expect_tx(smem_u32(&S->full[slot]), bytes);
                        bulk_g2s(b_smem + (uint32_t)slot * (uint32_t)P.slot_bytes, bsrc + (size_t)k0 * ks_bytes, bytes,
                                 smem_u32(&S->full[slot]));
                        S->slot_issued[slot] = use + 1;
                    }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                q = __shfl_sync(0xffffffffu, q, 0);
            }
            if (!ok) break;
        }
    } else if (warp == 1 && PAIR && !lead) {
        // ------------------------------------------------ odd CTA of a pair: relays "A landed" and
        // "B landed" of its own copies to the even CTA's barriers, in the issuer's order
        int q = 0, ctl = 0;
        bool stop = __any_sync(0xffffffffu, *abort_flag != 0);
        const uint32_t lead_cta = 0u;
        for (int it = item0; it < n_items && !stop; it += item_step, ++ctl) {
            const ItemCtx ic = item_ctx<MODE, PAIR>(P, it, tiles, ford, rank);
            const int ab = ctl % P.a_bufs, au = ctl / P.a_bufs;
            if (!__all_sync(0xffffffffu, mbar_wait<PAIR>(smem_u32(&S->a_full[ab]), au & 1, abort_flag, P.wait_cycles))) {
                if (lane == 0) fail<PAIR>(P, abort_flag, 4);
                stop = true;
                break;
            }
            if (lane == 0) {
                S->a_done[ab] = au + 1;
                mbar_arrive_remote(cluster_addr(smem_u32(&S->peer_a_full[ab]), lead_cta));
            }
            for (int t = ic.t0; t < ic.t1 && !stop; ++t) {
                const TileDesc td = ic.tiles[t];
                const int nks = td.ks_hi - td.ks_lo, n_copies = (nks + kps - 1) / kps;
                for (int c = 0; c < n_copies; ++c, ++q) {
                    const int slot = q % NS, use = q / NS;
                    if (!__all_sync(0xffffffffu, mbar_wait<PAIR>(smem_u32(&S->full[slot]), use & 1, abort_flag, P.wait_cycles))) {
                        if (lane == 0) fail<PAIR>(P, abort_flag, 16);
                        stop = true;
                        break;
                    }
                    if (lane == 0) {
                        S->slot_done[slot] = use + 1;
                        mbar_arrive_remote(cluster_addr(smem_u32(&S->peer_full[slot]), lead_cta));
                    }
                }
                if (!stop) stop = __any_sync(0xffffffffu, *abort_flag != 0);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer: the warp runs converged, lane 0
        // issues; every wait and every abort test is made warp-uniform before it steers the loop
        const uint32_t leader = lane == 0 ? 1u : 0u;
        constexpr int kM = PAIR ? 2 * kTileM : kTileM;
        int q = 0, acc_use = 0, ctl = 0;
        bool stop = __any_sync(0xffffffffu, *abort_flag != 0);
        for (int it = item0; it < n_items && !stop; it += item_step, ++ctl) {
            const ItemCtx ic = item_ctx<MODE, PAIR>(P, it, tiles, ford, rank);
            const int ab = AT ? 0 : ctl % P.a_bufs, au = AT ? 0 : ctl / P.a_bufs;
            if (AT) {
                // the item's A tile is the next copy of the ring; it moves into TMEM once the previous
                // item's MMAs (which read the A columns) have retired
                const int slot = q % NS, use = q / NS;
                if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&S->full[slot]), use & 1, abort_flag, P.wait_cycles) &&
                                                 (ctl == 0 || mbar_wait(smem_u32(&S->a_free), (ctl - 1) & 1, abort_flag,
                                                                        P.wait_cycles)))) {
                    if (leader) fail(P, abort_flag, 4);
                    stop = true;
                    break;
                }
                if (leader) S->slot_done[slot] = use + 1;
                tc_fence_after();
                const uint32_t src_lo = (((b_smem + (uint32_t)slot * (uint32_t)P.slot_bytes) >> 4) & 0x3FFFu) | (1u << 16);
                const uint32_t plane16 = (uint32_t)(ic.a_bytes / planes) >> 4;            // A plane, 16-byte units
                const int ksa = (int)(ic.a_bytes / planes / (kTileM * 32));              // k-steps of a plane
                for (int pl = 0; pl < planes; ++pl)
                    for (int ks = 0; ks < ksa; ++ks)
                        tc_cp_a(tmem + (uint32_t)(pl * P.at_plane_cols + ks * 8),
                                src_lo + (uint32_t)pl * plane16 + (uint32_t)(ks >> 2) * (kTileM * 8u) + (uint32_t)(ks & 3) * 2u,
                                kDescHi128, leader);
                tc_commit_if(smem_u32(&S->empty[slot]), leader);   // the slot returns once the copies are done
                ++q;
            } else {
                if (!__all_sync(0xffffffffu, mbar_wait<PAIR>(smem_u32(&S->a_full[ab]), au & 1, abort_flag, P.wait_cycles) &&
                                                 (!PAIR || mbar_wait<PAIR>(smem_u32(&S->peer_a_full[ab]), au & 1, abort_flag,
                                                                            P.wait_cycles)))) {
                    if (leader) fail<PAIR>(P, abort_flag, 4);
                    stop = true;
                    break;
                }
                if (leader) S->a_done[ab] = au + 1;
                tc_fence_after();
            }
            const uint32_t a0 = a_smem + (uint32_t)ab * (uint32_t)P.a_tile_bytes;
            const uint32_t a0_lo = ((a0 >> 4) & 0x3FFFu) | (1u << 16);       // descriptor low half of A
            const uint32_t alo_delta = (uint32_t)(ic.a_bytes / 2) >> 4;      // to the lo plane (BF16)
            for (int t = ic.t0; t < ic.t1 && !stop; ++t) {
                const TileDesc td = ic.tiles[t];
                const int buf = acc_use & 1, bu = acc_use >> 1;
                if (bu > 0 &&
                    !__all_sync(0xffffffffu, mbar_wait<PAIR>(smem_u32(&S->acc_empty[buf]), (bu - 1) & 1, abort_flag, P.wait_cycles))) {
                    if (leader) fail<PAIR>(P, abort_flag, 8);
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(P.acc_base + buf * P.acc_stride);
                const uint32_t idesc = instr_desc(PREC, td.n, kM);
                // this CTA's rows of a k-step block: N (one CTA) or N / 2 (each CTA of a pair)
                const uint32_t ks_bytes = (uint32_t)td.n * (PAIR ? 16u : 32u) * planes;
                const int nks = td.ks_hi - td.ks_lo, n_copies = (nks + kps - 1) / kps;
                uint32_t acc = 0u;
                for (int c = 0; c < n_copies; ++c) {
                    const int slot = q % NS, use = q / NS;
                    if (!__all_sync(0xffffffffu, mbar_wait<PAIR>(smem_u32(&S->full[slot]), use & 1, abort_flag, P.wait_cycles) &&
                                                     (!PAIR || mbar_wait<PAIR>(smem_u32(&S->peer_full[slot]), use & 1, abort_flag,
                                                                                P.wait_cycles)))) {
                        if (leader) fail<PAIR>(P, abort_flag, 16);
                        stop = true;
                        break;
                    }
                    if (leader) S->slot_done[slot] = use + 1;
                    tc_fence_after();
                    const uint32_t bslot = b_smem + (uint32_t)slot * (uint32_t)P.slot_bytes;
                    const int k0 = c * kps, kn = min(kps, nks - k0);
                    // descriptor low halves in 16-byte units: A k-step ks sits in 128-byte atom ks / 4
                    // (128 rows x 128 B apart) at 32 B x (ks % 4); B k-step blocks follow each other
                    uint32_t b_lo = ((bslot >> 4) & 0x3FFFu) | (1u << 16);
                    const uint32_t b_step = ks_bytes >> 4, b_plane = (uint32_t)td.n * (PAIR ? 1u : 2u);
                    int ks = td.ks_lo + k0;
                    for (int kk = 0; kk < kn; ++kk, ++ks, b_lo += b_step) {
                        if (AT) {
                            // A k-step ks: 8 TMEM columns per plane
                            const uint32_t a_t = tmem + (uint32_t)(ks * 8);
                            mma_tmem_a<PREC>(d, a_t, b_lo, kDescHi32, idesc, acc, leader);
                            if (PREC != GRACE_TF32) {
                                mma_tmem_a<PREC>(d, a_t, b_lo + b_plane, kDescHi32, idesc, 1u, leader);
                                mma_tmem_a<PREC>(d, a_t + (uint32_t)P.at_plane_cols, b_lo, kDescHi32, idesc, 1u, leader);
                            }
                            acc = 1u;
                            continue;
                        }
                        const uint32_t a_lo16 = a0_lo + (uint32_t)(ks >> 2) * (kTileM * 8u) + (uint32_t)(ks & 3) * 2u;
                        if (PREC == GRACE_TF32) {
                            mma_lohi<PREC, PAIR>(d, a_lo16, kDescHi128, b_lo, kDescHi32, idesc, acc, leader);
                        } else {
                            mma_lohi<PREC, PAIR>(d, a_lo16, kDescHi128, b_lo, kDescHi32, idesc, acc, leader);
                            mma_lohi<PREC, PAIR>(d, a_lo16, kDescHi128, b_lo + b_plane, kDescHi32, idesc, 1u, leader);
                            mma_lohi<PREC, PAIR>(d, a_lo16 + alo_delta, kDescHi128, b_lo, kDescHi32, idesc, 1u, leader);
                        }
                        acc = 1u;
                    }
                    tc_commit_if<PAIR>(smem_u32(&S->empty[slot]), leader);   // frees the slot once these MMAs retire
                    ++q;
                }
                if (stop) break;
                if (!acc) {
                    if (leader) fail<PAIR>(P, abort_flag, 64);   // tiles are built with a non-empty K range
                    stop = true;
                    break;
                }
                tc_commit_if<PAIR>(smem_u32(&S->acc_full[buf]), leader);
                ++acc_use;
                stop = __any_sync(0xffffffffu, *abort_flag != 0);
            }
            if (stop) break;
            if (AT) tc_commit_if(smem_u32(&S->a_free), leader);      // the A columns may be overwritten once these MMAs retire
            else tc_commit_if<PAIR>(smem_u32(&S->a_empty[ab]), leader);   // the A tile may be overwritten once these MMAs retire
            stop = __any_sync(0xffffffffu, *abort_flag != 0);
        }
        __syncwarp();
        if (leader && *abort_flag) {
            // every MMA this warp issued has retired before the CTA (and its pair) may leave
            tc_commit_if<PAIR>(smem_u32(&S->mma_drain), 1u, 1);
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(&S->mma_drain), 0) && clock64() - t0 < kWaitCycles) {
            }
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ------------------------------------------------ epilogue: one thread per cell
        constexpr bool kPlainEpi = MODE == kModeF || MODE == kModeMulti;   // epi_tile: window loaded early
        const int part = (warp - 4) >> 2;    // functionals f with f % kEpiSplit == part
        const int qd = warp & 3;             // TMEM lane quadrant (warp % 4)
        const int row = qd * 32 + lane;
        const uint32_t tlane = (uint32_t)(qd * 32) << 16;
        int acc_use = 0, ctl = 0;
        for (int it = item0; it < n_items; it += item_step, ++ctl) {
            const ItemCtx ic = item_ctx<MODE, PAIR>(P, it, tiles, ford, rank);
            const int ct = ic.ct;
            const int ab = AT ? 0 : ctl % P.a_bufs, au = AT ? 0 : ctl / P.a_bufs;
            if (!AT && !__all_sync(0xffffffffu, mbar_wait<PAIR>(smem_u32(&S->a_full[ab]), au & 1, abort_flag, P.wait_cycles))) {
                fail<PAIR>(P, abort_flag, 32);
                break;
            }
            // the ghat windows: from the A tile in shared memory, or (A in TMEM) from the A operand in
            // global memory
            const uint8_t *a_gen = AT ? ic.A : gbase + (size_t)ab * P.a_tile_bytes;
            const long long cell = (long long)ct * kTileM + row;
            const bool live = cell < ic.n_cells;
            const float s_cell = MODE == kModeNC && live ? P.cell_s[cell] : 0.f;
            const float *mu_cell = MODE == kModeVJP ? P.mu + (size_t)ct * P.R * kTileM + row : nullptr;
            float Facc[kEpiF];
#pragma unroll
            for (int m = 0; m < kEpiF; ++m) Facc[m] = 0.f;
            float FaccS[MODE == kModeSpecies ? kMaxSpeciesTc : 1][kEpiF];
#pragma unroll
            for (int sp = 0; sp < (MODE == kModeSpecies ? kMaxSpeciesTc : 1); ++sp)
#pragma unroll
                for (int m = 0; m < kEpiF; ++m) FaccS[sp][m] = 0.f;
            float Wacc[MODE == kModeVJP ? kWin : 1];
#pragma unroll
            for (int t = 0; t < (MODE == kModeVJP ? kWin : 1); ++t) Wacc[t] = 0.f;
            bool aborted = false;
            for (int t = ic.t0; t < ic.t1; ++t) {
                if (__any_sync(0xffffffffu, *abort_flag)) {
                    aborted = true;
                    break;
                }
                const TileDesc td = ic.tiles[t];
                const int nf = td.nf_flush & 0xFF, fs = (td.nf_flush >> 8) & 0xFF;
                const int buf = acc_use & 1, bu = acc_use >> 1;
                float gw[kPlainEpi ? kWin : 1];
                if (kPlainEpi) load_window<PREC, kWin>(a_gen, ic.a_bytes, row, td.acol, gw);
                if (!__all_sync(0xffffffffu, mbar_wait<PAIR>(smem_u32(&S->acc_full[buf]), bu & 1, abort_flag, P.wait_cycles))) {
                    fail<PAIR>(P, abort_flag, 128);
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint32_t tcol = tmem + tlane + (uint32_t)(P.acc_base + buf * P.acc_stride);
                if (MODE == kModeNC)
                    epi_tile_nc<PREC, 1>(a_gen, ic.a_bytes, row, td.p0, tcol, nf, fs, part, s_cell, D0s, P.ramp_a,
                                         P.ramp_b, Facc);
                else if (MODE == kModeVJP)
                    epi_tile_vjp<2>(tcol, nf, fs, part, mu_cell, ford, td.f0, Wacc);
                else if (MODE == kModeSpecies)
                    epi_tile_species<kWin>(P.gsp + (size_t)ct * P.gsp_kpad * kTileM, P.gsp_sstride, P.n_species,
                                           P.gsp_kpad, row, td.acol, tcol, nf, fs, part, FaccS);
                else
                    epi_tile<kWin, 2, PAIR>(gw, tcol, nf, fs, part, Facc, smem_u32(&S->acc_empty[buf]), lane);
                if (!kPlainEpi) release_acc<PAIR>(smem_u32(&S->acc_empty[buf]), lane);
                ++acc_use;
                if (MODE == kModeVJP && (td.nf_flush >> 16)) {
                    // last tile of this coefficient window: this warp's partial sums over its functionals
                    if (live) {
                        float *Wo = P.W + (((size_t)part * P.n_cell_tiles + ct) * P.Pw + td.p0) * kTileM + row;
#pragma unroll
                        for (int t = 0; t < (MODE == kModeVJP ? kWin : 1); ++t) Wo[(size_t)t * kTileM] = Wacc[t];
                    }
#pragma unroll
                    for (int t = 0; t < (MODE == kModeVJP ? kWin : 1); ++t) Wacc[t] = 0.f;
                } else if (MODE == kModeSpecies && (td.nf_flush >> 16)) {
#pragma unroll
                    for (int sp = 0; sp < (MODE == kModeSpecies ? kMaxSpeciesTc : 1); ++sp) {
                        if (sp >= P.n_species) break;
                        if (live) {
                            float *Fo = ic.F + (size_t)sp * P.f_sstride + ((size_t)ct * ic.R) * kTileM + row;
#pragma unroll
                            for (int m = 0; m < kEpiF; ++m) {
                                const int f = kEpiSplit * m + part;
                                if (f < nf) Fo[(size_t)ic.ford[td.f0 + f] * kTileM] = FaccS[sp][m];
                            }
                        }
#pragma unroll
                        for (int m = 0; m < kEpiF; ++m) FaccS[sp][m] = 0.f;
                    }
                } else if (MODE != kModeVJP && (td.nf_flush >> 16)) {
                    if (live) {
                        float *Fo = ic.F + ((size_t)ct * ic.R) * kTileM + row;
#pragma unroll
                        for (int m = 0; m < kEpiF; ++m) {
                            const int f = kEpiSplit * m + part;
                            if (f < nf) Fo[(size_t)ic.ford[td.f0 + f] * kTileM] = Facc[m];
                        }
                    }
#pragma unroll
                    for (int m = 0; m < kEpiF; ++m) Facc[m] = 0.f;
                }
            }
            if (aborted) break;
            __syncwarp();
            if (!AT && lane == 0) mbar_arrive(smem_u32(&S->a_empty[ab]));
            if (warp == 4 && lane == 0) S->items_done = ctl + 1;
        }
    }

    // ---------------------------------------------------- teardown
    // every role has stopped issuing; after an abort, drain the copies still in flight
    __syncwarp();
    __syncthreads();
    if (PAIR && warp == 4 && lane == 0 && !*abort_flag && S->items_done > 0) {
        // the last item's A release is a commit multicast by the even CTA: it has landed here before
        // this CTA may leave (bounded)
        const int last = S->items_done - 1, ab = last % P.a_bufs, au = last / P.a_bufs;
        const long long t0 = clock64();
        while (!mbar_try_wait_cluster(smem_u32(&S->a_empty[ab]), au & 1) && clock64() - t0 < kWaitCycles) {
        }
    }
    if (warp == 0 && lane == 0 && *abort_flag) {
        // drain copies still in flight into this CTA's shared memory (bounded)
        for (int s = 0; s < NS; ++s)
            for (int u = S->slot_done[s]; u < S->slot_issued[s]; ++u) {
                const long long t0 = clock64();
                while (!mbar_try_wait(smem_u32(&S->full[s]), u & 1) && clock64() - t0 < kWaitCycles) {
                }
            }
        for (int b = 0; b < 2; ++b)
            for (int u = S->a_done[b]; u < S->a_issued[b]; ++u) {
                const long long t0 = clock64();
                while (!mbar_try_wait(smem_u32(&S->a_full[b]), u & 1) && clock64() - t0 < kWaitCycles) {
                }
            }
    }
    tc_fence_before();
    __syncthreads();
    // a CTA of a pair leaves only when its peer no longer arrives on its barriers, its MMAs no longer
    // read the peer's shared memory, and the pair frees its TMEM together
    if (PAIR) cluster_sync_all();
    tc_fence_after();
    if (warp == 2) {
        if (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                         : "memory");
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
void free_tc_tiles(TcTiles &t)
{
    if (t.at) {
        free_tc_tiles(*t.at);
        delete t.at;
    }
    cudaFree(t.d_b);
    cudaFree(t.d_b_pair);
    cudaFree(t.d_desc);
    cudaFree(t.d_ford);
    cudaFree(t.d_D0);
    cudaFree(t.d_written);
    t = TcTiles();
}

size_t opA_bytes_for(const DevGroup &g, int prec, int n_cells, int *kpad)
{
    const int ae = atom_elems(prec);
    const int K = g.cell_alpha ? g.N * g.Q : g.P;   // node values (per-cell kernels) or coefficients
    const int kp = (K + ae - 1) / ae * ae;
    if (kpad) *kpad = kp;
    const size_t tiles = ((size_t)n_cells + kTileM - 1) / kTileM;
    return tiles * opA_tile_bytes(prec, kp);
}

size_t f32_bytes_for(const DevGroup &g, int n_cells)
{
    const size_t tiles = ((size_t)n_cells + kTileM - 1) / kTileM;
    return tiles * (size_t)g.R * kTileM * sizeof(float);
}

static uint16_t bf16_bits_rn(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);   // inf / nan
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

static float bf16_to_f(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

static uint32_t tf32_bits_rn(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return u;
    u += 0x1000u;            // round half away from zero at bit 13
    return u & 0xFFFFE000u;
}

// byte offset of element x (0 .. 32/eb - 1) of row `row` in a K-major SWIZZLE_32B k-step block
static inline size_t sw32_offset(int row, int x, int eb)
{
    const int byte = x * eb;
    const int chunk = (byte >> 4) ^ ((row >> 2) & 1);
    return (size_t)row * 32 + (chunk << 4) + (byte & 15);
}

namespace {

// Dense per-functional matrices of one contraction, already scaled for the tensor
// operands: M[(r * rows + p) * kdim + q] multiplies A column q into accumulator row p of
// functional r.  Rows come in windows of W consecutive rows (the accumulator columns of
// one functional in an N-tile); the epilogue vector of window w starts at A column
// w * p0_stride.
struct Forms {
    int R = 0, rows = 0, kdim = 0, W = 0, p0_stride = 0;
    int aofs = 0;   // A-operand column of coefficient 0 of the windows (the A column offset)
    std::vector<double> M;
    const double *row(int r, int p) const { return M.data() + ((size_t)r * rows + p) * kdim; }
    int n_win() const { return (rows + W - 1) / W; }
};

struct Ext {
    int lo, hi;
};

struct Plan {
    double cost = 1e300;
    std::vector<int> first;                 // first functional (index into ford) of every group
    std::vector<std::vector<Ext>> wext;     // [ford index][window] union of the rows' q extents
};

double tile_cost(int prec, int n, int nks)
{
    const int planes = n_planes(prec), mult = prec == GRACE_TF32 ? 1 : 3;
    const double mma = (double)nks * mult * kMmaClk;
    const double l2 = (double)nks * n * 32.0 * planes / kL2BytesPerClk;
    const double epi = kEpiBaseClk + kEpiColClk * n;
    return std::max(mma, std::max(l2, epi)) + kTileClk;
}

// dynamic program over the functional order: best[y] = cheapest cover of ford[0, y) by
// groups of consecutive functionals, each group one N-tile per non-empty window
Plan plan_forms(const Forms &F, const std::vector<int> &ford, int prec, int max_n = kMaxN)
{
    const int R = F.R, W = F.W, nw = F.n_win(), kstep = 32 / elem_bytes(prec);
    Plan pl;
    pl.wext.assign(R, std::vector<Ext>(nw, Ext{F.kdim, 0}));
    for (int x = 0; x < R; ++x)
        for (int p = 0; p < F.rows; ++p) {
            const double *Mr = F.row(ford[x], p);
            int lo = F.kdim, hi = 0;
            for (int q = 0; q < F.kdim; ++q)
                if (Mr[q] != 0.0) {
                    lo = std::min(lo, q);
                    hi = q + 1;
                }
            if (hi <= lo) continue;
            Ext &E = pl.wext[x][p / W];
            E.lo = std::min(E.lo, lo);
            E.hi = std::max(E.hi, hi);
        }
    const double inf = 1e300;
    std::vector<double> best(R + 1, inf);
    std::vector<int> from(R + 1, -1);
    best[0] = 0.0;
    const int maxf = std::min(kMaxF, std::min(kMaxN, max_n) / W);
    for (int x = 0; x < R; ++x) {
        if (best[x] >= inf) continue;
        std::vector<Ext> Un(nw, Ext{F.kdim, 0});
        std::vector<int> first_live(nw, -1);   // first functional of [x, y) with rows in the window
        for (int y = x + 1; y <= std::min(R, x + maxf); ++y) {
            double c = 0.0;
            for (int w = 0; w < nw; ++w) {
                const Ext &E = pl.wext[y - 1][w];
                if (E.hi > E.lo && first_live[w] < 0) first_live[w] = y - 1;
                Un[w].lo = std::min(Un[w].lo, E.lo);
                Un[w].hi = std::max(Un[w].hi, E.hi);
                if (Un[w].hi > Un[w].lo)
                    c += tile_cost(prec, (y - first_live[w]) * W,
                                   (Un[w].hi + kstep - 1) / kstep - Un[w].lo / kstep);
            }
            if (best[x] + c < best[y]) {
                best[y] = best[x] + c;
                from[y] = x;
            }
        }
    }
    for (int y = R; y > 0; y = from[y]) pl.first.push_back(from[y]);
    std::reverse(pl.first.begin(), pl.first.end());
    pl.cost = best[R];
    return pl;
}

// B images (SWIZZLE_32B k-step blocks, bf16 hi/lo planes or TF32) and tile descriptors of a
// plan, uploaded into out; written[r] = 1 for every functional the contraction writes
grace_status emit_tiles(const Forms &F, const Plan &pl, const std::vector<int> &ford, int prec, TcTiles &out,
                        std::vector<int> &written, bool window_major = false, bool pair_image = false)
{
    const int R = F.R, W = F.W, nw = F.n_win();
    const int eb = elem_bytes(prec), planes = n_planes(prec);
    const int kstep = 32 / eb;
    const int kps = prec == GRACE_TF32 ? 4 : 2;
    const int mult = prec == GRACE_TF32 ? 1 : 3;
    std::vector<TileDesc> tiles;
    std::vector<int> tile_win;        // window of every tile
    std::vector<double> tile_cost_v;  // cost-model cycles of every tile
    std::vector<uint8_t> B;
    written.assign(R, 0);
    long long macs = 0, mmas = 0;
    for (size_t gi = 0; gi < pl.first.size(); ++gi) {
        const int x = pl.first[gi];
        const int y = gi + 1 < pl.first.size() ? pl.first[gi + 1] : R;
        const int nf = y - x;
        const size_t first = tiles.size();
        double gcost = 0.0;
        for (int w = 0; w < nw; ++w) {
            Ext Un{F.kdim, 0};
            int fs = -1;   // functionals before the first one with rows in this window take no columns
            for (int f = x; f < y; ++f) {
                const Ext &E = pl.wext[f][w];
                if (E.hi > E.lo && fs < 0) fs = f - x;
                Un.lo = std::min(Un.lo, E.lo);
                Un.hi = std::max(Un.hi, E.hi);
            }
            if (Un.hi <= Un.lo) continue;
            const int n = (nf - fs) * W;
            TileDesc td;
            std::memset(&td, 0, sizeof(td));
            td.n = n;
            td.nf_flush = nf | (fs << 8);
            td.p0 = w * F.p0_stride;
            td.acol = td.p0 + F.aofs;
            td.ks_lo = Un.lo / kstep;
            td.ks_hi = (Un.hi + kstep - 1) / kstep;
            td.f0 = x;
            const int nks = td.ks_hi - td.ks_lo;
            td.b_off16 = (int)(B.size() / 16);
            const size_t blk = (size_t)n * 32;   // one plane of one k-step
            B.resize(B.size() + (size_t)nks * blk * planes, 0);
            uint8_t *img = B.data() + (size_t)td.b_off16 * 16;
            for (int s = 0; s < nks; ++s) {
                uint8_t *bk = img + (size_t)s * blk * planes;
                for (int f = fs; f < nf; ++f)
                    for (int c = 0; c < W; ++c) {
                        const int p = w * W + c, rowi = (f - fs) * W + c;
                        if (p >= F.rows) continue;
                        const double *Mr = F.row(ford[x + f], p);
                        for (int xx = 0; xx < kstep; ++xx) {
                            const int q = (td.ks_lo + s) * kstep + xx;
                            if (q >= F.kdim) continue;
                            const double val = Mr[q];
                            if (val == 0.0) continue;
                            const size_t off = sw32_offset(rowi, xx, eb);
                            if (prec == GRACE_TF32) {
                                const uint32_t bits = tf32_bits_rn((float)val);
                                std::memcpy(bk + off, &bits, 4);
                            } else {
                                const uint16_t hi = bf16_bits_rn((float)val);
                                const uint16_t lo = bf16_bits_rn((float)(val - (double)bf16_to_f(hi)));
                                std::memcpy(bk + off, &hi, 2);
                                std::memcpy(bk + blk + off, &lo, 2);
                            }
                        }
                    }
            }
            macs += (long long)n * nks * kstep;
            mmas += (long long)nks * mult;
            gcost += tile_cost(prec, n, nks);
            out.slot_bytes = std::max(out.slot_bytes, (int)(std::min(kps, nks) * blk * planes));
            out.max_rows = std::max(out.max_rows, n);
            tiles.push_back(td);
            tile_win.push_back(w);
            tile_cost_v.push_back(tile_cost(prec, n, nks));
        }
        if (tiles.size() > first) {
            tiles.back().nf_flush |= 1 << 16;
            out.group_tile.push_back((int)first);
            out.group_cost.push_back(gcost);
            for (int f = x; f < y; ++f) written[ford[f]] = 1;
        }
    }
    if (tiles.empty()) {
        set_error("tensor-core tiles: the coefficient tensor is empty");
        return GRACE_ERR_ARG;
    }
    if (window_major) {
        // VJP order: all tiles of coefficient window 0, then window 1, ...; the last tile of every
        // window flushes the window's partial sums; splits fall on window boundaries
        std::vector<int> idx(tiles.size());
        for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return tile_win[a] < tile_win[b]; });
        std::vector<TileDesc> sorted;
        out.group_tile.clear();
        out.group_cost.clear();
        for (size_t i = 0; i < idx.size(); ++i) {
            TileDesc td = tiles[idx[i]];
            td.nf_flush &= 0xFFFF;   // keep nf and fs, clear the flush bit
            const bool first = i == 0 || tile_win[idx[i]] != tile_win[idx[i - 1]];
            const bool last = i + 1 == idx.size() || tile_win[idx[i]] != tile_win[idx[i + 1]];
            if (first) {
                out.group_tile.push_back((int)sorted.size());
                out.group_cost.push_back(0.0);
            }
            out.group_cost.back() += tile_cost_v[idx[i]];
            if (last) td.nf_flush |= 1 << 16;
            sorted.push_back(td);
        }
        tiles.swap(sorted);
    }
    if (B.size() / 16 > (size_t)INT32_MAX) {
        set_error("tensor-core tiles: B images too large");
        return GRACE_ERR_UNSUPPORTED;
    }
    out.group_tile.push_back((int)tiles.size());
    // CTA-pair images: every tile's k-step blocks split into the halves of their rows (the N / 2
    // rows of each half start on an 8-row boundary, so the 32-byte swizzle of each row is kept),
    // each half's blocks contiguous so that a CTA copies only its own
    std::vector<uint8_t> Bp;
    if (pair_image) {
        Bp.assign(B.size(), 0);
        for (const TileDesc &td : tiles) {
            const size_t blk = (size_t)td.n * 32, half = blk / 2;
            const int nks = td.ks_hi - td.ks_lo;
            const uint8_t *src = B.data() + (size_t)td.b_off16 * 16;
            uint8_t *dst = Bp.data() + (size_t)td.b_off16 * 16;
            for (int hh = 0; hh < 2; ++hh)
                for (int s = 0; s < nks; ++s)
                    for (int pl = 0; pl < planes; ++pl)
                        std::memcpy(dst + (((size_t)hh * nks + s) * planes + pl) * half,
                                    src + ((size_t)s * planes + pl) * blk + (size_t)hh * half, half);
        }
    }
    cudaError_t e = cudaMalloc(&out.d_b, B.size());
    if (e == cudaSuccess && pair_image) e = cudaMalloc(&out.d_b_pair, Bp.size());
    if (e == cudaSuccess && pair_image) e = cudaMemcpy(out.d_b_pair, Bp.data(), Bp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&out.d_desc, tiles.size() * sizeof(TileDesc));
    if (e == cudaSuccess) e = cudaMalloc(&out.d_ford, ford.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(out.d_b, B.data(), B.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_desc, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_ford, ford.data(), ford.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_tc_tiles(out);
        return cuda_fail(e, "tensor-core tiles: upload");
    }
    out.n_tiles = (int)tiles.size();
    out.b_bytes = B.size();
    out.mac_per_cell = macs;
    out.mma_per_tile = mmas;
    out.pred_clk = pl.cost;
    out.slot_bytes = (out.slot_bytes + 1023) / 1024 * 1024;
    return GRACE_OK;
}

// The A operand stores coefficient q at column q + kofs, so that the coefficient range ends close
// to the padded K extent (every k-step block ends on a k-step boundary there).  Moves the columns
// of M ([R][P][P], coefficient q in column q) to q + kofs; with shift_rows its rows p to p + kofs
// as well.  The rows keep their place by default: the p windows stay aligned to the coefficients
// (fewer padded rows), the window of coefficients [p0, p0 + 16) is read from A columns
// [p0 + kofs, p0 + kofs + 16), and the epilogue reads zeros past the padded row.
void shift_forms(Forms &F, int P, int kofs, bool shift_rows)
{
    F.aofs = shift_rows ? 0 : kofs;
    if (kofs == 0) return;
    const int kd = P + kofs, rows = shift_rows ? P + kofs : P, r0 = shift_rows ? kofs : 0;
    std::vector<double> M((size_t)F.R * rows * kd, 0.0);
    for (int r = 0; r < F.R; ++r)
        for (int p = 0; p < P; ++p)
            std::memcpy(M.data() + ((size_t)r * rows + p + r0) * kd + kofs, F.M.data() + ((size_t)r * P + p) * P,
                        (size_t)P * sizeof(double));
    F.M.swap(M);
    F.kdim = kd;
    F.rows = rows;
}

// functionals in bin order: interface flux of bin j, then its volume terms
std::vector<int> functional_order(const DevGroup &g)
{
    std::vector<int> ford;
    for (int j = 0; j < g.N; ++j) {
        if (j < g.n_if) ford.push_back(j);
        for (int i = 1; i <= g.k; ++i) ford.push_back(g.n_if + j * g.k + i - 1);
    }
    return ford;
}

}  // namespace

// TMEM columns of one A plane in the A-in-tensor-memory form, and the accumulator width that leaves
__host__ __device__ inline int at_plane_cols(int prec, int kpad) { return kpad * elem_bytes(prec) / 4; }
inline int at_acc_cols(int prec, int kpad)
{
    return (kTmemCols - n_planes(prec) * at_plane_cols(prec, kpad)) / 2 / 16 * 16;
}

grace_status build_tc_tiles(Group &G, int prec, cudaStream_t st)
{
    TcTiles out;
    grace_status s = build_tc_tiles_from(G, G.d_T, prec, out, st, false, true);
    if (s != GRACE_OK) return s;
    // the A-in-tensor-memory form for groups whose A tile takes at most 128 TMEM columns (N <= 192)
    if (n_planes(prec) * at_plane_cols(prec, out.k_pad) <= 128) {
        TcTiles at;
        s = build_tc_tiles_from(G, G.d_T, prec, at, st, false, false, at_acc_cols(prec, out.k_pad));
        if (s != GRACE_OK) {
            free_tc_tiles(out);
            return s;
        }
        out.at = new TcTiles(at);
    }
    free_tc_tiles(G.tc[prec]);
    G.tc[prec] = out;
    return GRACE_OK;
}

// tiles of T as built (not folded: the outer and partner slots of a species' form differ)
grace_status build_species_tiles(Group &G, int prec, cudaStream_t st)
{
    TcTiles out;
    grace_status s = build_tc_tiles_from(G, G.d_T, prec, out, st, true);
    if (s != GRACE_OK) return s;
    free_tc_tiles(G.tcs[prec]);
    G.tcs[prec] = out;
    return GRACE_OK;
}

// tiles of the quadratic forms d_T ([R][P][P], FP64, device) of group G; an all-zero d_T gives
// built tiles with n_tiles = 0 (nothing to contract)
grace_status build_tc_tiles_from(const Group &G, const double *d_T, int prec, TcTiles &out, cudaStream_t st,
                                 bool unfolded_only, bool pair_image, int max_n)
{
    const DevGroup &g = G.dg;
    if (g.k > kKMax) {
        set_error("tensor-core tiles need k <= 4");
        return GRACE_ERR_UNSUPPORTED;
    }
    const int P_ = g.P, R = g.R, K1 = g.K1;
    Forms FT, FU;
    FT.R = FU.R = R;
    FT.rows = FU.rows = P_;
    FT.kdim = FU.kdim = P_;
    FT.W = FU.W = kWin;
    FT.p0_stride = FU.p0_stride = kWin;
    FT.M.resize((size_t)R * P_ * P_);
    cudaError_t e = cudaMemcpyAsync(FT.M.data(), d_T, FT.M.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core tiles: copy T");

    std::vector<double> h(g.N);
    for (int j = 0; j < g.N; ++j) h[j] = G.h_edges[j + 1] - G.h_edges[j];

    // Two representations of the same quadratic forms: T as built (u-side p, v-side q) and its
    // fold onto the upper triangle U (U[p][q] = T[p][q] + T[q][p], q > p).  Both are planned and the
    // cheaper plan under the cost model is built.  Entries are scaled by 1 / (h_bin(p) h_bin(q)).
    FU.M = FT.M;
    long long nnz_fold = 0, nnz_T = 0;
    for (int r = 0; r < R; ++r) {
        double *Ur = FU.M.data() + (size_t)r * P_ * P_;
        for (int p = 0; p < P_; ++p)
            for (int q = p + 1; q < P_; ++q) {
                Ur[(size_t)p * P_ + q] += Ur[(size_t)q * P_ + p];
                Ur[(size_t)q * P_ + p] = 0.0;
            }
    }
    for (size_t i = 0; i < FT.M.size(); ++i) {
        nnz_T += FT.M[i] != 0.0;
        nnz_fold += FU.M[i] != 0.0;
    }
    for (int r = 0; r < R; ++r)
        for (int p = 0; p < P_; ++p)
            for (int q = 0; q < P_; ++q) {
                const size_t i = ((size_t)r * P_ + p) * P_ + q;
                const double sc = 1.0 / (h[p / K1] * h[q / K1]);
                FT.M[i] *= sc;
                FU.M[i] *= sc;
            }

    const std::vector<int> ford = functional_order(g);
    if ((int)ford.size() != R) {
        set_error("tensor-core tiles: functional count mismatch");
        return GRACE_ERR_ARG;
    }
    out = TcTiles();
    const int ae = atom_elems(prec);
    out.k_pad = (P_ + ae - 1) / ae * ae;
    out.k_ofs = a_column_offset(prec, P_);
    shift_forms(FT, P_, out.k_ofs, false);
    shift_forms(FU, P_, out.k_ofs, false);
    if (nnz_T == 0) {
        out.built = 1;
        return GRACE_OK;
    }
    const Plan pT = plan_forms(FT, ford, prec, max_n);
    const Plan pU = unfolded_only ? Plan() : plan_forms(FU, ford, prec, max_n);
    const bool use_fold = !unfolded_only && pU.cost <= pT.cost;
    std::vector<int> written;
    grace_status s = emit_tiles(use_fold ? FU : FT, use_fold ? pU : pT, ford, prec, out, written, false, pair_image);
    if (s != GRACE_OK) return s;
    e = cudaMalloc(&out.d_written, R * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(out.d_written, written.data(), R * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_tc_tiles(out);
        return cuda_fail(e, "tensor-core tiles: upload");
    }
    out.nnz_fold = std::min(nnz_fold, nnz_T);
    out.folded = use_fold ? 1 : 0;
    out.built = 1;
    return GRACE_OK;
}

// Tensor-core tiles of the VJP: the symmetric S_r = T_r + T_r^T (full, scaled by
// 1 / (h_bin(p) h_bin(q))), so that the MMA gives Y[c, (r, p)] = sum_q Shat_r[p, q] ghat_q and the
// epilogue sums mu_r Y over the functionals of each 16-wide window of p (window-major order).
grace_status build_vjp_tiles(Group &G, int prec, cudaStream_t st)
{
    const DevGroup &g = G.dg;
    if (g.k > kKMax) {
        set_error("tensor-core tiles need k <= 4");
        return GRACE_ERR_UNSUPPORTED;
    }
    const int P_ = g.P, R = g.R, K1 = g.K1;
    Forms F;
    F.R = R;
    F.rows = P_;
    F.kdim = P_;
    F.W = kWin;
    F.p0_stride = kWin;
    std::vector<double> T((size_t)R * P_ * P_);
    cudaError_t e = cudaMemcpyAsync(T.data(), G.d_T, T.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "VJP tiles: copy T");
    std::vector<double> h(g.N);
    for (int j = 0; j < g.N; ++j) h[j] = G.h_edges[j + 1] - G.h_edges[j];
    F.M.resize(T.size());
    for (int r = 0; r < R; ++r)
        for (int p = 0; p < P_; ++p)
            for (int q = 0; q < P_; ++q) {
                const size_t i = ((size_t)r * P_ + p) * P_ + q, it = ((size_t)r * P_ + q) * P_ + p;
                F.M[i] = (T[i] + T[it]) / (h[p / K1] * h[q / K1]);
            }
    const std::vector<int> ford = functional_order(g);
    const int kofs = a_column_offset(prec, P_);
    shift_forms(F, P_, kofs, false);
    const Plan pl = plan_forms(F, ford, prec);
    TcTiles out;
    std::vector<int> written;
    grace_status s = emit_tiles(F, pl, ford, prec, out, written, true);
    if (s != GRACE_OK) return s;
    const int ae = atom_elems(prec);
    out.k_pad = (P_ + ae - 1) / ae * ae;
    out.k_ofs = kofs;
    out.vjp = 1;
    out.built = 1;
    free_tc_tiles(G.tcv[prec]);
    G.tcv[prec] = out;
    return GRACE_OK;
}

// Tensor-core tiles of the fixed-pair part of a per-cell kernel group.  The MMA contracts
// over the smaller node i (A = the cell's node values Ghat_i = h_bin(i) G_i), one accumulator
// row per (functional, larger node j, factor): rows [32 w, 32 w + 16) of window w hold the
// coagulation weights Cc_r[i][j] of nodes j in [16 w, 16 w + 16), rows [32 w + 16, 32 w + 32)
// the fragmentation weights Cf_r[i][j], both scaled by 1 / (h_bin(i) h_bin(j)).  The epilogue
// multiplies them by s (1 - pf_j) Ghat_j and s pf_j Ghat_j.
grace_status build_nc_tc_tiles(Group &G, int prec, cudaStream_t st)
{
    const DevGroup &g = G.dg;
    const NcTables &T = G.nc;
    if (!T.built) {
        set_error("tensor-core tiles: node-space tables not built");
        return GRACE_ERR_ORDER;
    }
    const int R = g.R, Q = g.Q, NQ = T.NQ;
    const size_t ntab = (size_t)R * NQ * NQ;
    std::vector<double> Cc(ntab), Cf(ntab), D0(NQ);
    cudaError_t e = cudaMemcpyAsync(Cc.data(), T.d_Cc, ntab * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Cf.data(), T.d_Cf, ntab * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(D0.data(), T.d_D0, NQ * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core tiles: copy node-space tables");
    std::vector<double> h(g.N);
    for (int j = 0; j < g.N; ++j) h[j] = G.h_edges[j + 1] - G.h_edges[j];

    Forms F;
    F.R = R;
    F.W = 2 * kWin;
    F.p0_stride = kWin;
    const int nw = (NQ + kWin - 1) / kWin;
    F.rows = nw * F.W;
    F.kdim = NQ;
    F.M.assign((size_t)R * F.rows * NQ, 0.0);
    double vmin = INFINITY, vmax = 0.0;
    for (int r = 0; r < R; ++r)
        for (int i = 0; i < NQ; ++i)
            for (int j = 0; j < NQ; ++j)
                for (int src = 0; src < 2; ++src) {
                    const double v = (src ? Cf : Cc)[((size_t)r * NQ + i) * NQ + j];
                    if (v == 0.0) continue;
                    const double sv = v / (h[i / Q] * h[j / Q]);
                    const int row = (j / kWin) * F.W + src * kWin + j % kWin;
                    F.M[((size_t)r * F.rows + row) * NQ + i] = sv;
                    vmin = std::min(vmin, std::fabs(sv));
                    vmax = std::max(vmax, std::fabs(sv));
                }
    // the scaled weights must be normal FP32 numbers (with room for the products)
    if (vmax > 0.0 && (vmin < 1e-30 || vmax > 1e30)) {
        set_error("tensor-core tiles: node-space weights outside the FP32 range");
        return GRACE_ERR_UNSUPPORTED;
    }
    const std::vector<int> ford = functional_order(g);
    const Plan pl = plan_forms(F, ford, prec);
    TcTiles out;
    std::vector<int> written;
    grace_status s = emit_tiles(F, pl, ford, prec, out, written);
    if (s != GRACE_OK) return s;
    const int ae = atom_elems(prec);
    out.k_pad = (NQ + ae - 1) / ae * ae;
    long long nnz = 0;
    for (size_t i = 0; i < ntab; ++i) nnz += (Cc[i] != 0.0) + (Cf[i] != 0.0);
    out.nnz_fold = nnz;
    out.folded = 1;
    out.nc = 1;
    out.n_d0 = nw * kWin;
    std::vector<float> d0f(out.n_d0, 0.f);
    for (int a = 0; a < NQ; ++a) d0f[a] = (float)D0[a];
    const double vf = g.coag_p[4], wr = g.coag_p[5];
    out.ramp_a = (float)(1.0 / (2.0 * wr * vf));
    out.ramp_b = (float)(-(1.0 - wr) / (2.0 * wr));
    e = cudaMalloc(&out.d_D0, d0f.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&out.d_written, R * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(out.d_D0, d0f.data(), d0f.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_written, written.data(), R * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_tc_tiles(out);
        return cuda_fail(e, "tensor-core tiles: node tables upload");
    }
    out.built = 1;
    free_tc_tiles(G.tc[prec]);
    G.tc[prec] = out;
    return GRACE_OK;
}

static int sm_count(int dev)
{
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Splits of the tile list (at functional-group boundaries) so that
// n_cell_tiles x n_splits work items fill the SMs evenly.
static void choose_splits(const TcTiles &t, int n_cell_tiles, int n_sm, TcParams &P)
{
    const int n_groups = (int)t.group_cost.size();
    double total = 0.0;
    for (double c : t.group_cost) total += c;
    int best_s = 1;
    double best_t = 1e300;
    for (int s = 1; s <= std::min(kMaxSplits, n_groups); ++s) {
        const long long items = (long long)n_cell_tiles * s;
        const long long rounds = (items + n_sm - 1) / n_sm;
        const double time = (double)rounds * (total / s + kItemClk);
        if (time < best_t * 0.97) {
            best_t = time;
            best_s = s;
        }
    }
    // cut where the running cost crosses multiples of total / s
    P.split[0] = 0;
    int ns = 0;
    double run = 0.0;
    for (int gi = 0; gi < n_groups && ns + 1 < best_s; ++gi) {
        run += t.group_cost[gi];
        if (run >= total * (ns + 1) / best_s && gi + 1 < n_groups) P.split[++ns] = t.group_tile[gi + 1];
    }
    P.split[++ns] = t.n_tiles;
    P.n_splits = ns;
}

// One-shot check of failure detection (grace_test_arm_wait_timeout): the next contraction launch
// of the process waits at most this many cycles and issues no B copies.
static std::atomic<long long> g_armed_wait_cycles{0};

// CTA pairs (grace_set_cta_pairs): 0 (default) never, 1 every forward contraction of at least two
// cell tiles, 2 multi-group launches only.  Measured on this part, pairs were slower in both
// places (BF16x3, 65,536 cells: 571 against 644 TFLOP/s; uneven batch: 327 against 354): halving
// each SM's table bytes does not shorten the wait for a tile's table copy.
static std::atomic<int> g_cta_pairs{0};

// the A-in-tensor-memory form for single-group forward contractions (grace_set_tc_a_in_tmem), off by
// default: measured slower on this part (BF16x3, 65,536 cells: 505 against 604 TFLOP/s; TF32 186
// against 216).  Its tiles are narrower (N <= 192: 45 tiles instead of 36) and each tile still waits
// ~880 cycles for its table copy with the 3-deep ring, as with the 2-deep one.
static std::atomic<int> g_a_in_tmem{0};

template <int PREC, int MODE, int FORM = 0>
static cudaError_t launch_prec(TcParams P, int max_rows, cudaStream_t st)
{
    constexpr int PAIR = FORM == 1 ? 1 : 0;
    constexpr bool AT = FORM == 2;
    P.wait_cycles = kWaitCycles;
    P.withhold_b = 0;
    const long long armed = g_armed_wait_cycles.exchange(0);
    if (armed > 0) {
        P.wait_cycles = armed;
        P.withhold_b = 1;
    }
    constexpr int planes = PREC == GRACE_TF32 ? 1 : 2;
    P.table_bytes = (int)((P.n_tiles * sizeof(TileDesc) + (size_t)P.R * sizeof(int) +
                           (MODE == kModeNC ? (size_t)P.n_d0 * sizeof(float) : 0) + 15) / 16 * 16);
    const size_t fixed = 1024 + (size_t)P.table_bytes + sizeof(Smem) + 64;
    const size_t a1 = (size_t)P.a_tile_bytes;
    // Shared-memory plan: B copies of up to 64 KB (4 BF16 / 8 TF32 k-steps at N = 256) in a ring of at
    // least two, fewer k-steps per copy for groups whose A tile leaves less room; two A tiles (the
    // next work item's A loads during this one) only when that still leaves a 4-deep ring.  The MMA
    // thread pays a fixed cost per copy (barrier wait, fence, commit), so few large copies beat a
    // deeper ring of small ones: measured on the 65,536-cell workload (BF16x3), two A tiles with a
    // 3-deep ring of 32 KB copies took 0.217 ms against 0.203 ms for one A tile and 2 x 64 KB (the
    // A-tile waits fell from 21k to 4k cycles per CTA, the B and per-copy time grew by 50k).
    // A CTA of a pair holds half the rows of every k-step block: its copies of up to 64 KB take 8 BF16
    // / 16 TF32 k-steps at N = 256, a whole tile of the additive workload in one copy (copies of 32 KB
    // in a 4-deep ring measured slower: the copy engine pays per copy more than per byte).
    const int rows_cta = PAIR ? max_rows / 2 : max_rows;
    auto slot_of = [&](int kps) { return (int)(((size_t)kps * rows_cta * 32 * planes + 1023) / 1024 * 1024); };
    P.acc_base = 0;
    P.acc_stride = kAccCols;
    P.at_plane_cols = 0;
    if (AT) {
        // no A tile in shared memory: ring slots of 64 KB (or the A tile, if larger) hold either the
        // item's A tile or up to kps k-steps of B; A takes the first TMEM columns, the two
        // accumulators the rest
        const int kpad = (int)(a1 / ((size_t)kTileM * elem_bytes(PREC) * planes));
        P.at_plane_cols = at_plane_cols(PREC, kpad);
        P.acc_base = planes * P.at_plane_cols;
        P.acc_stride = at_acc_cols(PREC, kpad);
        if (max_rows > P.acc_stride) return cudaErrorInvalidValue;
        P.a_bufs = 0;
        P.kps = 1;
        while (slot_of(P.kps + 1) <= std::max<size_t>(65536, a1)) ++P.kps;
        P.slot_bytes = (int)((std::max<size_t>((size_t)slot_of(P.kps), a1) + 1023) / 1024 * 1024);
        if (fixed + 2 * (size_t)P.slot_bytes > (size_t)kSmemLimit) return cudaErrorInvalidValue;
        P.n_slots = (int)std::min<size_t>(kMaxSlots, ((size_t)kSmemLimit - fixed) / P.slot_bytes);
    } else {
    P.kps = (PREC == GRACE_TF32 ? 8 : 4) * (PAIR ? 2 : 1);
    while (P.kps > 1 && fixed + a1 + 2 * (size_t)slot_of(P.kps) > (size_t)kSmemLimit) P.kps /= 2;
    P.a_bufs = fixed + 2 * a1 + 4 * (size_t)slot_of(P.kps) <= (size_t)kSmemLimit ? 2 : 1;
    P.slot_bytes = slot_of(P.kps);
    if (fixed + P.a_bufs * a1 + 2 * (size_t)P.slot_bytes > (size_t)kSmemLimit) return cudaErrorInvalidValue;
    P.n_slots = (int)std::min<size_t>(kMaxSlots, ((size_t)kSmemLimit - fixed - P.a_bufs * a1) / P.slot_bytes);
    }
    const size_t smem = fixed + P.a_bufs * a1 + (size_t)P.n_slots * P.slot_bytes;
    auto kern = contract_tc_kernel<PREC, MODE, FORM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!PAIR) {
        const int items = P.n_cell_tiles * P.n_splits;
        const int grid = std::min(items, sm_count(dev));
        kern<<<grid, kThreads, smem, st>>>(P);
        return cudaGetLastError();
    }
    // clusters of two CTAs, as many as can be resident at once (a persistent kernel: every cluster
    // loops over its share of the items)
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * (sm_count(dev) / 2));
    int max_clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (max_clusters < 1) return cudaErrorInvalidConfiguration;
    const int items = P.n_pair_tiles * P.n_splits;
    cfg.gridDim = dim3(2 * std::min(items, max_clusters));
    e = cudaLaunchKernelEx(&cfg, kern, P);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_contract_tc(const DevGroup &g, const TcTiles &t, int prec, const void *opA, int n_cells,
                               float *d_F32, int *d_err, cudaStream_t st, const float *d_cell_s)
{
    if (!t.built || n_cells <= 0) return n_cells == 0 ? cudaSuccess : cudaErrorInvalidValue;
    if (t.nc && !d_cell_s) return cudaErrorInvalidValue;
    TcParams P;
    std::memset(&P, 0, sizeof(P));
    P.tiles = (const TileDesc *)t.d_desc;
    P.ford = t.d_ford;
    P.n_tiles = t.n_tiles;
    P.B = (const uint8_t *)t.d_b;
    P.A = (const uint8_t *)opA;
    P.a_tile_bytes = (long long)opA_tile_bytes(prec, t.k_pad);
    P.n_cells = n_cells;
    P.n_cell_tiles = (n_cells + kTileM - 1) / kTileM;
    P.R = g.R;
    P.F = d_F32;
    P.err = d_err;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!t.nc && t.d_b_pair && P.n_cell_tiles >= 2 && g_cta_pairs.load() == 1) {
        P.B = (const uint8_t *)t.d_b_pair;
        P.n_pair_tiles = (P.n_cell_tiles + 1) / 2;
        choose_splits(t, P.n_pair_tiles, sm_count(dev) / 2, P);
        return prec == GRACE_TF32 ? launch_prec<GRACE_TF32, kModeF, 1>(P, t.max_rows, st)
                                  : launch_prec<GRACE_BF16X3, kModeF, 1>(P, t.max_rows, st);
    }
    if (!t.nc && t.at && t.at->built && t.at->n_tiles > 0 && g_a_in_tmem.load()) {
        const TcTiles &ta = *t.at;
        P.tiles = (const TileDesc *)ta.d_desc;
        P.ford = ta.d_ford;
        P.n_tiles = ta.n_tiles;
        P.B = (const uint8_t *)ta.d_b;
        choose_splits(ta, P.n_cell_tiles, sm_count(dev), P);
        return prec == GRACE_TF32 ? launch_prec<GRACE_TF32, kModeF, 2>(P, ta.max_rows, st)
                                  : launch_prec<GRACE_BF16X3, kModeF, 2>(P, ta.max_rows, st);
    }
    choose_splits(t, P.n_cell_tiles, sm_count(dev), P);
    if (t.nc) {
        P.D0 = t.d_D0;
        P.n_d0 = t.n_d0;
        P.cell_s = d_cell_s;
        P.ramp_a = t.ramp_a;
        P.ramp_b = t.ramp_b;
        return prec == GRACE_TF32 ? launch_prec<GRACE_TF32, kModeNC>(P, t.max_rows, st)
                                  : launch_prec<GRACE_BF16X3, kModeNC>(P, t.max_rows, st);
    }
    return prec == GRACE_TF32 ? launch_prec<GRACE_TF32, kModeF>(P, t.max_rows, st)
                              : launch_prec<GRACE_BF16X3, kModeF>(P, t.max_rows, st);
}

cudaError_t launch_contract_tc_species(const DevGroup &g, const TcTiles &t, int prec, const void *opA, int n_cells,
                                       const float *d_gsp, int n_species, float *d_F32, int *d_err, cudaStream_t st)
{
    if (!t.built || t.nc || t.vjp || n_cells <= 0 || n_species < 1 || n_species > kMaxSpeciesTc)
        return n_cells == 0 ? cudaSuccess : cudaErrorInvalidValue;
    TcParams P;
    std::memset(&P, 0, sizeof(P));
    P.tiles = (const TileDesc *)t.d_desc;
    P.ford = t.d_ford;
    P.n_tiles = t.n_tiles;
    P.B = (const uint8_t *)t.d_b;
    P.A = (const uint8_t *)opA;
    P.a_tile_bytes = (long long)opA_tile_bytes(prec, t.k_pad);
    P.n_cells = n_cells;
    P.n_cell_tiles = (n_cells + kTileM - 1) / kTileM;
    P.R = g.R;
    P.F = d_F32;
    P.err = d_err;
    P.gsp = d_gsp;
    P.gsp_kpad = t.k_pad;
    P.gsp_sstride = (long long)P.n_cell_tiles * t.k_pad * kTileM;
    P.f_sstride = (long long)P.n_cell_tiles * g.R * kTileM;
    P.n_species = n_species;
    int dev = 0;
    cudaGetDevice(&dev);
    choose_splits(t, P.n_cell_tiles, sm_count(dev), P);
    return prec == GRACE_TF32 ? launch_prec<GRACE_TF32, kModeSpecies>(P, t.max_rows, st)
                              : launch_prec<GRACE_BF16X3, kModeSpecies>(P, t.max_rows, st);
}

void free_tc_multi(TcMulti &m)
{
    cudaFree(m.d_groups);
    cudaFree(m.d_items);
    cudaFree(m.d_pair_items);
    m = TcMulti();
}

grace_status build_tc_multi(int prec, const std::vector<TcMultiPart> &parts, TcMulti &out)
{
    free_tc_multi(out);
    std::vector<TcGroupDesc> groups;
    std::vector<std::pair<double, int2>> items, pitems;
    int pair_ok = 1;
    long long max_a = 0;
    int max_rows = 0;
    for (size_t i = 0; i < parts.size(); ++i) {
        const TcMultiPart &p = parts[i];
        if (!p.t || !p.t->built || p.t->nc || p.t->vjp) {
            set_error("multi-group contraction: a part has no forward tensor-core tiles");
            return GRACE_ERR_ORDER;
        }
        TcGroupDesc g;
        std::memset(&g, 0, sizeof(g));
        g.tiles = (const TileDesc *)p.t->d_desc;
        g.ford = p.t->d_ford;
        g.B = (const uint8_t *)p.t->d_b;
        g.Bp = (const uint8_t *)p.t->d_b_pair;
        if (!g.Bp) pair_ok = 0;
        g.A = (const uint8_t *)p.opA;
        g.F = p.F32;
        g.a_tile_bytes = (long long)opA_tile_bytes(prec, p.t->k_pad);
        g.n_cells = p.n_cells;
        g.R = p.R;
        g.t0 = 0;
        g.t1 = p.t->n_tiles;
        max_a = std::max(max_a, g.a_tile_bytes);
        max_rows = std::max(max_rows, p.t->max_rows);
        const int n_ct = (p.n_cells + kTileM - 1) / kTileM;
        for (int ct = 0; ct < n_ct; ++ct) items.push_back({p.t->pred_clk, make_int2((int)i, ct)});
        for (int u = 0; u < (n_ct + 1) / 2; ++u) pitems.push_back({p.t->pred_clk, make_int2((int)i, u)});
        groups.push_back(g);
    }
    // largest items first: the round-robin assignment then approximates a balanced schedule
    auto by_cost = [](const auto &a, const auto &b) { return a.first > b.first; };
    std::stable_sort(items.begin(), items.end(), by_cost);
    std::stable_sort(pitems.begin(), pitems.end(), by_cost);
    std::vector<int2> it(items.size()), pit(pitems.size());
    for (size_t i = 0; i < items.size(); ++i) it[i] = items[i].second;
    for (size_t i = 0; i < pitems.size(); ++i) pit[i] = pitems[i].second;
    cudaError_t e = cudaMalloc(&out.d_groups, std::max<size_t>(groups.size(), 1) * sizeof(TcGroupDesc));
    if (e == cudaSuccess) e = cudaMalloc(&out.d_items, std::max<size_t>(it.size(), 1) * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&out.d_pair_items, std::max<size_t>(pit.size(), 1) * sizeof(int2));
    if (e == cudaSuccess && !pit.empty())
        e = cudaMemcpy(out.d_pair_items, pit.data(), pit.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !groups.empty())
        e = cudaMemcpy(out.d_groups, groups.data(), groups.size() * sizeof(TcGroupDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !it.empty()) e = cudaMemcpy(out.d_items, it.data(), it.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_tc_multi(out);
        return cuda_fail(e, "multi-group contraction: upload");
    }
    out.n_items = (int)it.size();
    out.n_pair_items = (int)pit.size();
    out.pair_ok = pair_ok;
    out.max_a = max_a;
    out.max_rows = max_rows;
    out.prec = prec;
    return GRACE_OK;
}

cudaError_t launch_contract_tc_multi(const TcMulti &m, int *d_err, cudaStream_t st)
{
    if (m.n_items == 0) return cudaSuccess;
    TcParams P;
    std::memset(&P, 0, sizeof(P));
    P.groups = (const TcGroupDesc *)m.d_groups;
    P.items = (const int2 *)m.d_items;
    P.n_cell_tiles = m.n_items;   // items, one split each
    P.n_splits = 1;
    P.a_tile_bytes = m.max_a;     // stride of the A buffers in shared memory
    P.err = d_err;
    if (m.pair_ok && g_cta_pairs.load() != 0) {
        // each group's tables stream once per pair of its cell tiles instead of once per tile
        P.items = (const int2 *)m.d_pair_items;
        P.n_pair_tiles = m.n_pair_items;
        return m.prec == GRACE_TF32 ? launch_prec<GRACE_TF32, kModeMulti, 1>(P, m.max_rows, st)
                                    : launch_prec<GRACE_BF16X3, kModeMulti, 1>(P, m.max_rows, st);
    }
    return m.prec == GRACE_TF32 ? launch_prec<GRACE_TF32, kModeMulti>(P, m.max_rows, st)
                                : launch_prec<GRACE_BF16X3, kModeMulti>(P, m.max_rows, st);
}

cudaError_t launch_vjp_tc(const DevGroup &g, const TcTiles &t, int prec, const void *opA, const float *d_mu32,
                          int n_cells, float *d_W32, int *d_err, cudaStream_t st)
{
    if (!t.built || !t.vjp || n_cells <= 0) return n_cells == 0 ? cudaSuccess : cudaErrorInvalidValue;
    TcParams P;
    std::memset(&P, 0, sizeof(P));
    P.tiles = (const TileDesc *)t.d_desc;
    P.ford = t.d_ford;
    P.n_tiles = t.n_tiles;
    P.B = (const uint8_t *)t.d_b;
    P.A = (const uint8_t *)opA;
    P.a_tile_bytes = (long long)opA_tile_bytes(prec, t.k_pad);
    P.n_cells = n_cells;
    P.n_cell_tiles = (n_cells + kTileM - 1) / kTileM;
    P.R = g.R;
    P.err = d_err;
    P.mu = d_mu32;
    P.W = d_W32;
    P.Pw = vjp_window_cols(g);
    int dev = 0;
    cudaGetDevice(&dev);
    choose_splits(t, P.n_cell_tiles, sm_count(dev), P);
    return prec == GRACE_TF32 ? launch_prec<GRACE_TF32, kModeVJP>(P, t.max_rows, st)
                              : launch_prec<GRACE_BF16X3, kModeVJP>(P, t.max_rows, st);
}

}  // namespace grace

namespace grace {
// the tile set a single-group forward contraction of these tiles runs (launch_contract_tc's choice for
// batches of at least two cell tiles)
const TcTiles &tc_forward_tiles(const TcTiles &t)
{
    if (!t.nc && g_cta_pairs.load() != 1 && t.at && t.at->built && t.at->n_tiles > 0 && g_a_in_tmem.load()) return *t.at;
    return t;
}
}  // namespace grace

extern "C" grace_status grace_set_tc_a_in_tmem(int enable)
{
    if (enable != 0 && enable != 1) {
        grace::set_error("grace_set_tc_a_in_tmem: enable must be 0 or 1");
        return GRACE_ERR_ARG;
    }
    grace::g_a_in_tmem.store(enable);
    return GRACE_OK;
}

extern "C" grace_status grace_set_cta_pairs(int mode)
{
    if (mode < 0 || mode > 2) {
        grace::set_error("grace_set_cta_pairs: mode must be 0, 1 or 2");
        return GRACE_ERR_ARG;
    }
    grace::g_cta_pairs.store(mode);
    return GRACE_OK;
}

extern "C" grace_status grace_test_arm_wait_timeout(long long wait_cycles)
{
    if (wait_cycles <= 0 || wait_cycles > grace::kWaitCycles) {
        grace::set_error("grace_test_arm_wait_timeout: wait_cycles must lie in [1, 4e9]");
        return GRACE_ERR_ARG;
    }
    grace::g_armed_wait_cycles.store(wait_cycles);
    return GRACE_OK;
}

namespace grace {
int tc_vjp_planes() { return kEpiSplit; }
}  // namespace grace
