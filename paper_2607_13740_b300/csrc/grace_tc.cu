// K-b: tensor-core contraction of the flux functionals on tcgen05 / TMEM.
//
// Every flux functional of a cell is a quadratic form of its coefficients,
//     F_r = sum_{p,q} T_r[p,q] g_p g_q                     (see grace_precompute.cu).
// Over a batch this is one GEMM per tile of 128 cells, factorised as
//     Y[c, (r,p)] = sum_q  ghat[c, q] * That_r[p, q]        (tcgen05.mma, FP32 in TMEM)
//     F[c, r]     = sum_p  ghat[c, p] * Y[c, (r,p)]         (epilogue, one lane per cell)
// with ghat = g * h_bin (bin-mass scaling) and That = T / (h_bin(p) h_bin(q)), so
// operands stay in a comfortable FP32/BF16 range for grids spanning 16 decades.
// The product g (x) g is never materialised: the MMA contracts T with g on one
// side and the epilogue contracts the accumulator with g on the other, which
// keeps the A operand equal to the cells' own coefficient tile.
//
// Output columns of one MMA tile are a set of up to 4 functionals x a window of
// 32 consecutive p; the epilogue holds that 32-wide window of ghat in
// registers and reuses it for every functional of the tile.  A tile's K range
// is the union of the non-zero q extents of its rows (T is block-sparse: for
// an interface flux at x_{j+1/2} the u-side rows p < 3j only couple to v-side
// columns q of bins >= j-1), so zero blocks are skipped at the MMA k-step.
//
// Operands live in global memory as ready-made shared-memory images in the
// canonical K-major SWIZZLE_128B layout (grace_tc_layout.cuh); one
// cp.async.bulk moves a cell tile's A operand or one K atom of a B tile.
//
// Warp roles (persistent, one CTA per SM, cell tiles round-robin):
//   warp 0 lane 0 : bulk-copy producer (A tile, then the B atoms of every N tile)
//   warp 1 lane 0 : MMA issuer (kind::tf32, or kind::f16 with bf16 hi/lo x3)
//   warp 2        : TMEM allocation / release
//   warps 4..7    : epilogue, TMEM lane quadrant = warp % 4, one cell per thread
// Every wait on an mbarrier is bounded; on timeout the CTA records an error in
// the device error word, stops issuing work, drains its outstanding copies and
// releases its tensor memory before returning.
#include <cstring>
#include <vector>

#include "grace_limiter.cuh"
#include "grace_tc_layout.cuh"

namespace grace {

namespace {

constexpr int kMaxFunc = 4;         // functionals per N tile
constexpr int kWin = 32;            // p window per functional
constexpr int kMaxSlots = 16;       // B ring depth (K atoms), sized at launch from free shared memory
constexpr int kAccCols = 128;       // TMEM columns per accumulator buffer
constexpr int kHalfCols = 256;      // two accumulator buffers per cell tile
constexpr int kSmemLimit = 227 * 1024;

// NT = cell tiles per CTA pass (1 or 2): TMEM columns, epilogue warps, threads
template <int NT> struct Cfg {
    static constexpr int tmem_cols = NT * kHalfCols;
    static constexpr int epi_warps = 4 * NT;     // warps 4..7: first tile, 8..11: second
    static constexpr int threads = 32 * (4 + 4 * NT);
};
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

struct TileDesc {
    long long b_off;    // byte offset of the tile's first K atom image
    int nrows;          // MMA N = nf * 32
    int nf;             // functionals in this tile
    int atom_lo;        // first K atom (global K index / atom width)
    int n_atoms;        // K atoms stored for this tile
    int ks_lo, ks_hi;   // MMA k-steps [ks_lo, ks_hi) (32 bytes of K each)
    int p0;             // first p of the window
    int flush;          // last window of its functional group: write F
    int r[kMaxFunc];    // functional ids (-1 unused)
    int bin_lo, bin_hi; // bins whose functionals belong to this tile's group
};
static_assert(sizeof(TileDesc) == 64, "TileDesc layout");

struct TcParams {
    const TileDesc *tiles;
    int n_tiles;
    const uint8_t *B;
    const uint8_t *A;
    long long a_tile_bytes;
    int n_cells;
    int n_cell_tiles;
    int R;
    float *F;
    int prec;
    int slot_bytes;       // bytes of one ring slot (max nrows x 128 x planes)
    int n_slots;          // ring depth
    int *err;
    // fused flux difference / RK stage (eq. evo, eq. RK3), used when mode != 0
    int mode;             // 0: functionals to F; 1: L[g] to gout; 2: SSP-RK3 stage update
    DevGroup G;
    const double *gn, *gs, *dt;
    double *gout;
    double ca, cb;
    int apply_limiter;
    double *mass;
    unsigned char *flags;
    uint8_t *a_next;      // A operand of gout (may alias A), or null
};

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

// bounded wait: false on timeout or when another role already aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
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

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// SWIZZLE_128B K-major shared-memory matrix descriptor (8-row groups 1024 B apart)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset
    d |= (uint64_t)1u << 46;                   // descriptor version
    d |= (uint64_t)2u << 61;                   // SWIZZLE_128B
    return d;
}

// instruction descriptor: FP32 accumulate, K-major A and B, M = 128, N = n
__device__ __forceinline__ uint32_t instr_desc(int prec, int n)
{
    const uint32_t fmt = prec == GRACE_TF32 ? 2u : 1u;   // TF32 = 2, BF16 = 1
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// ---------------------------------------------------------------- fused update
// 16-byte chunk of one cell's row of the next-stage A operand, filled in k order
struct OpChunk {
    int c;
    uint32_t w[4], lo[4];
};

__device__ __forceinline__ void chunk_flush(const OpChunk &ch, const TcParams &P, uint8_t *tile, int row)
{
    if (ch.c < 0) return;
    if (P.prec == GRACE_TF32) {
        *reinterpret_cast<uint4 *>(tile + swz_offset(kTileM, row, 4 * ch.c, 4)) = make_uint4(ch.w[0], ch.w[1], ch.w[2], ch.w[3]);
    } else {
        const size_t off = swz_offset(kTileM, row, 8 * ch.c, 2);
        *reinterpret_cast<uint4 *>(tile + off) = make_uint4(ch.w[0], ch.w[1], ch.w[2], ch.w[3]);
        *reinterpret_cast<uint4 *>(tile + P.a_tile_bytes / 2 + off) = make_uint4(ch.lo[0], ch.lo[1], ch.lo[2], ch.lo[3]);
    }
}

__device__ __forceinline__ void set4(uint32_t *w, int e, uint32_t v)
{
    w[0] = e == 0 ? v : w[0];
    w[1] = e == 1 ? v : w[1];
    w[2] = e == 2 ? v : w[2];
    w[3] = e == 3 ? v : w[3];
}

__device__ __forceinline__ void chunk_put(OpChunk &ch, const TcParams &P, uint8_t *tile, int row, int k, float x)
{
    const int per = P.prec == GRACE_TF32 ? 4 : 8;
    const int c = k / per, e = k - c * per;
    if (c != ch.c) {
        chunk_flush(ch, P, tile, row);
        ch.c = c;
        for (int i = 0; i < 4; ++i) ch.w[i] = ch.lo[i] = 0u;
    }
    if (P.prec == GRACE_TF32) {
        set4(ch.w, e, f32_to_tf32_rna(x));
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        const int wi = e >> 1, sh = (e & 1) * 16;
        const uint32_t hm = (uint32_t)__bfloat16_as_ushort(h) << sh, lm = (uint32_t)__bfloat16_as_ushort(l) << sh;
        const uint32_t keep = (e & 1) ? 0x0000FFFFu : 0xFFFF0000u;
        uint32_t hw = 0, lw = 0;
        for (int i = 0; i < 4; ++i)
            if (i == wi) { hw = ch.w[i]; lw = ch.lo[i]; }
        set4(ch.w, wi, (hw & keep) | hm);
        set4(ch.lo, wi, (lw & keep) | lm);
    }
}

// L_j^i of eq. (evo) from the bin's functionals and, in stage mode, the SSP-RK3
// combination; the i = 0 row in FP64 (telescoping flux difference, mass), the
// i >= 1 rows in FP32.  gnb / gsb hold the bin's stage inputs (loaded ahead of
// time by the caller).  Writes gout (and the next A operand through ch).
__device__ __forceinline__ void update_bin(const TcParams &P, long long cell, int j, float Fm, float Fp,
                                           const float *V, double dtc, const double *gnb, const double *gsb,
                                           double &msum, unsigned &fl, OpChunk &ch, uint8_t *tile, int row)
{
    const DevGroup &G = P.G;
    const int k = G.k, K1 = G.K1;
    const size_t base = (size_t)cell * G.P + (size_t)j * K1;
    double v[kBinMax];
    float vf[kBinMax];
    const double L0 = ((double)Fm - (double)Fp) * G.inv_h[j];
    const float ih = G.inv_h32[j];
    if (P.mode == 1) {
        v[0] = L0;
#pragma unroll
        for (int i = 1; i < kBinMax; ++i)
            if (i <= k) {
                vf[i] = (2.f * i + 1.f) * ih * (V[i - 1] - Fp + ((i & 1) ? -Fm : Fm));
                v[i] = (double)vf[i];
            }
    } else {
        v[0] = P.ca * gnb[0] + P.cb * (gsb[0] + dtc * L0);
        const float a = (float)P.ca, b = (float)P.cb, dtf = (float)dtc;
#pragma unroll
        for (int i = 1; i < kBinMax; ++i)
            if (i <= k) {
                const float L = (2.f * i + 1.f) * ih * (V[i - 1] - Fp + ((i & 1) ? -Fm : Fm));
                vf[i] = a * (float)gnb[i] + b * ((float)gsb[i] + dtf * L);
                v[i] = (double)vf[i];
            }
        if (v[0] < 0.0) fl |= GRACE_FLAG_NEGATIVE_MEAN;
#pragma unroll
        for (int i = 0; i < kBinMax; ++i)
            if (i <= k && !isfinite(v[i])) fl |= GRACE_FLAG_NONFINITE;
        if (P.apply_limiter) {
            const unsigned f = limit_bin(v, k);
            fl |= f;
            if (f & GRACE_FLAG_LIMITED) {
#pragma unroll
                for (int i = 1; i < kBinMax; ++i)
                    if (i <= k) vf[i] = (float)v[i];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kBinMax; ++i)
        if (i <= k) P.gout[base + i] = v[i];
    if (P.a_next) {
        vf[0] = (float)v[0];
        const float h = (float)G.hbin[j];
#pragma unroll
        for (int i = 0; i < kBinMax; ++i)
            if (i <= k) chunk_put(ch, P, tile, row, j * K1 + i, vf[i] * h);
    }
    msum += G.hbin[j] * v[0];
}

// stage inputs of bin j (zeros beyond k)
__device__ __forceinline__ void load_bin(const TcParams &P, long long cell, int j, double *gnb, double *gsb)
{
    const size_t base = (size_t)cell * P.G.P + (size_t)j * P.G.K1;
#pragma unroll
    for (int i = 0; i < kBinMax; ++i) {
        const bool ok = P.mode == 2 && i <= P.G.k;
        gnb[i] = ok ? P.gn[base + i] : 0.0;
        gsb[i] = ok ? P.gs[base + i] : 0.0;
    }
}

// ---------------------------------------------------------------- kernel
struct Smem {
    uint64_t a_full, a_empty;
    uint64_t full[kMaxSlots], empty[kMaxSlots];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t mma_drain;
    uint32_t tmem_base;
    int abort_flag;
    int slot_issued[kMaxSlots];  // copies issued per slot (producer)
    int slot_done[kMaxSlots];    // copies consumed per slot (MMA)
    int a_issued, a_done;
};

__device__ __forceinline__ void fail(TcParams &P, volatile int *abort_flag, int code)
{
    if (P.err) atomicOr(P.err, code);
    *abort_flag = 1;
}

// TMEM -> registers, 32 lanes x 32 columns, no wait
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t *r)
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

// Each CTA takes NT 128-cell tiles at a time (a pair when both A tiles fit in
// shared memory): every B atom it streams feeds NT MMAs, one per cell tile, so
// B traffic per cell drops by NT.  TMEM holds NT tiles x 2 buffers x 128 columns.
template <int NT>
__global__ void __launch_bounds__(Cfg<NT>::threads, 1) contract_tc_kernel(TcParams P)
{
    constexpr int kEpiWarps = Cfg<NT>::epi_warps;
    constexpr int kTmemCols = Cfg<NT>::tmem_cols;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t a_smem = base;                                          // NT A tiles
    const uint32_t b_smem = base + (uint32_t)NT * (uint32_t)P.a_tile_bytes;   // B ring
    Smem *S = reinterpret_cast<Smem *>(gbase + NT * P.a_tile_bytes + (size_t)P.n_slots * P.slot_bytes);
    volatile int *abort_flag = &S->abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int planes = P.prec == GRACE_TF32 ? 1 : 2;
    const int NS = P.n_slots;
    const int n_pairs = (P.n_cell_tiles + NT - 1) / NT;   // CTA work items of NT tiles

    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&S->a_full), 1);
        mbar_init(smem_u32(&S->a_empty), 1 + kEpiWarps);
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&S->full[s]), 1);
            mbar_init(smem_u32(&S->empty[s]), 1);
            S->slot_issued[s] = 0;
            S->slot_done[s] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&S->acc_full[b]), 1);
            mbar_init(smem_u32(&S->acc_empty[b]), kEpiWarps);
        }
        mbar_init(smem_u32(&S->mma_drain), 1);
        S->abort_flag = 0;
        S->a_issued = S->a_done = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S->tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ producer
        int slot = 0, nuse = 0, ctl = 0;
        for (int pr = blockIdx.x; pr < n_pairs && !*abort_flag; pr += gridDim.x, ++ctl) {
            if (ctl > 0 && !mbar_wait(smem_u32(&S->a_empty), (ctl - 1) & 1, abort_flag)) {
                fail(P, abort_flag, 1);
                break;
            }
            const uint32_t abytes = (uint32_t)NT * (uint32_t)P.a_tile_bytes;   // the NT tiles are contiguous
            mbar_expect_tx(smem_u32(&S->a_full), abytes);
            bulk_g2s(a_smem, P.A + (size_t)(NT * pr) * P.a_tile_bytes, abytes, smem_u32(&S->a_full));
            S->a_issued = ctl + 1;
            for (int t = 0; t < P.n_tiles && !*abort_flag; ++t) {
                const TileDesc td = P.tiles[t];
                const uint32_t atom_bytes = (uint32_t)td.nrows * 128u * planes;
                for (int a = 0; a < td.n_atoms; ++a) {
                    const int use = nuse / NS;
                    if (use > 0 && !mbar_wait(smem_u32(&S->empty[slot]), (use - 1) & 1, abort_flag)) {
                        fail(P, abort_flag, 2);
                        break;
                    }
                    mbar_expect_tx(smem_u32(&S->full[slot]), atom_bytes);
                    bulk_g2s(b_smem + (uint32_t)slot * P.slot_bytes, P.B + td.b_off + (size_t)a * atom_bytes,
                             atom_bytes, smem_u32(&S->full[slot]));
                    S->slot_issued[slot] = use + 1;
                    ++nuse;
                    slot = nuse % NS;
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------ MMA issuer
        int slot = 0, nuse = 0, acc_use = 0, ctl = 0;
        const uint32_t a1 = a_smem + (uint32_t)P.a_tile_bytes;
        for (int pr = blockIdx.x; pr < n_pairs && !*abort_flag; pr += gridDim.x, ++ctl) {
            if (!mbar_wait(smem_u32(&S->a_full), ctl & 1, abort_flag)) {
                fail(P, abort_flag, 4);
                break;
            }
            S->a_done = ctl + 1;
            tc_fence_after();
            for (int t = 0; t < P.n_tiles && !*abort_flag; ++t) {
                const TileDesc td = P.tiles[t];
                const int buf = acc_use & 1, bu = acc_use >> 1;
                if (bu > 0 && !mbar_wait(smem_u32(&S->acc_empty[buf]), (bu - 1) & 1, abort_flag)) {
                    fail(P, abort_flag, 8);
                    break;
                }
                tc_fence_after();
                const uint32_t d0 = tmem + (uint32_t)(buf * kAccCols);
                const uint32_t d1 = d0 + (uint32_t)kHalfCols;
                const uint32_t idesc = instr_desc(P.prec, td.nrows);
                int first = 1;
                for (int a = 0; a < td.n_atoms; ++a) {
                    const int use = nuse / NS;
                    if (!mbar_wait(smem_u32(&S->full[slot]), use & 1, abort_flag)) {
                        fail(P, abort_flag, 16);
                        break;
                    }
                    S->slot_done[slot] = use + 1;
                    tc_fence_after();
                    const int atom = td.atom_lo + a;
                    const uint32_t bslot = b_smem + (uint32_t)slot * P.slot_bytes;
                    for (int kk = 0; kk < 4; ++kk) {
                        const int ks = atom * 4 + kk;
                        if (ks < td.ks_lo || ks >= td.ks_hi) continue;
                        const uint32_t a_off = (uint32_t)atom * (kTileM * 128u) + (uint32_t)kk * 32u;
                        const uint64_t bd = smem_desc(bslot + (uint32_t)kk * 32u);
                        const uint32_t acc = first ? 0u : 1u;
                        if (P.prec == GRACE_TF32) {
                            mma_tf32(d0, smem_desc(a_smem + a_off), bd, idesc, acc);
                            if (NT == 2) mma_tf32(d1, smem_desc(a1 + a_off), bd, idesc, acc);
                        } else {
                            const uint32_t lo_plane = (uint32_t)(P.a_tile_bytes / 2);
                            const uint64_t bl = smem_desc(bslot + (uint32_t)td.nrows * 128u + (uint32_t)kk * 32u);
                            mma_f16(d0, smem_desc(a_smem + a_off), bd, idesc, acc);
                            mma_f16(d0, smem_desc(a_smem + a_off), bl, idesc, 1u);
                            mma_f16(d0, smem_desc(a_smem + lo_plane + a_off), bd, idesc, 1u);
                            if (NT == 2) {
                                mma_f16(d1, smem_desc(a1 + a_off), bd, idesc, acc);
                                mma_f16(d1, smem_desc(a1 + a_off), bl, idesc, 1u);
                                mma_f16(d1, smem_desc(a1 + lo_plane + a_off), bd, idesc, 1u);
                            }
                        }
                        first = 0;
                    }
                    tc_commit(smem_u32(&S->empty[slot]));   // frees the slot once these MMAs retire
                    ++nuse;
                    slot = nuse % NS;
                }
                if (*abort_flag) break;
                if (first) {
                    fail(P, abort_flag, 64);   // tiles are built with a non-empty K range
                    break;
                }
                tc_commit(smem_u32(&S->acc_full[buf]));
                ++acc_use;
            }
            tc_commit(smem_u32(&S->a_empty));   // the A pair may be overwritten once these MMAs retire
        }
        if (*abort_flag) {
            tc_commit(smem_u32(&S->mma_drain));
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(&S->mma_drain), 0) && clock64() - t0 < kWaitCycles) {
            }
        }
    } else if (warp >= 4) {
        // ------------------------------------------------ epilogue: one thread per cell
        const int half = (warp - 4) >> 2;    // which tile of the pair
        const int q = warp & 3;              // TMEM lane quadrant (warp % 4)
        const int row = q * 32 + lane;
        const uint8_t *a_gen = gbase + (size_t)half * P.a_tile_bytes;
        const uint32_t tcol0 = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * kHalfCols);
        int acc_use = 0, ctl = 0;
        for (int pr = blockIdx.x; pr < n_pairs && !*abort_flag; pr += gridDim.x, ++ctl) {
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&S->a_full), ctl & 1, abort_flag))) {
                fail(P, abort_flag, 32);
                break;
            }
            const long long cell = (long long)(NT * pr + half) * kTileM + row;
            const bool live = cell < P.n_cells;
            float Facc[kMaxFunc] = {0.f, 0.f, 0.f, 0.f};
            // fused update state of this cell
            const double dtc = (P.mode == 2 && live) ? P.dt[cell] : 0.0;
            double msum = 0.0;
            unsigned fl = 0u;
            OpChunk ch;
            ch.c = -1;
            uint8_t *anext = P.a_next ? P.a_next + (size_t)(NT * pr + half) * P.a_tile_bytes : nullptr;
            int jnext = 0;          // next bin to update
            float Fprev = 0.f;      // F(x_{jnext - 1/2}); F(x_min) = 0
            for (int t = 0; t < P.n_tiles; ++t) {
                if (__any_sync(0xffffffffu, *abort_flag)) break;
                const TileDesc td = P.tiles[t];
                // ghat window [p0, p0 + 32) of this thread's cell from its A tile
                float gw[kWin];
                if (P.prec == GRACE_TF32) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 v = *reinterpret_cast<const float4 *>(a_gen + swz_offset(kTileM, row, td.p0 + 4 * c, 4));
                        gw[4 * c] = v.x;
                        gw[4 * c + 1] = v.y;
                        gw[4 * c + 2] = v.z;
                        gw[4 * c + 3] = v.w;
                    }
                } else {
                    const size_t lo_plane = (size_t)(P.a_tile_bytes / 2);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const size_t off = swz_offset(kTileM, row, td.p0 + 8 * c, 2);
                        const uint4 hi = *reinterpret_cast<const uint4 *>(a_gen + off);
                        const uint4 lo = *reinterpret_cast<const uint4 *>(a_gen + lo_plane + off);
                        const uint32_t hw[4] = {hi.x, hi.y, hi.z, hi.w}, lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            gw[8 * c + 2 * e] = __uint_as_float(hw[e] << 16) + __uint_as_float(lw[e] << 16);
                            gw[8 * c + 2 * e + 1] =
                                __uint_as_float(hw[e] & 0xFFFF0000u) + __uint_as_float(lw[e] & 0xFFFF0000u);
                        }
                    }
                }
                // stage inputs of the next bin to update, loaded before the accumulator wait
                double pgn[kBinMax], pgs[kBinMax];
                const bool pre = P.mode == 2 && td.flush && live && jnext <= td.bin_hi;
                if (pre) load_bin(P, cell, jnext, pgn, pgs);
                const int buf = acc_use & 1, bu = acc_use >> 1;
                if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&S->acc_full[buf]), bu & 1, abort_flag))) {
                    fail(P, abort_flag, 128);
                    break;
                }
                tc_fence_after();
                const uint32_t tcol = tcol0 + (uint32_t)(buf * kAccCols);
                for (int f = 0; f < td.nf; f += 2) {
                    uint32_t y0[kWin], y1[kWin];
                    tmem_ld32_nowait(tcol + (uint32_t)(f * kWin), y0);
                    if (f + 1 < td.nf) tmem_ld32_nowait(tcol + (uint32_t)((f + 1) * kWin), y1);
                    tmem_wait_ld();
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int c = 0; c < kWin; ++c) s0 = fmaf(gw[c], __uint_as_float(y0[c]), s0);
                    Facc[f] += s0;
                    if (f + 1 < td.nf) {
#pragma unroll
                        for (int c = 0; c < kWin; ++c) s1 = fmaf(gw[c], __uint_as_float(y1[c]), s1);
                        Facc[f + 1] += s1;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&S->acc_empty[buf]));
                ++acc_use;
                if (td.flush) {
                    if (P.mode == 0) {
                        if (live)
                            for (int f = 0; f < td.nf; ++f) P.F[cell * P.R + td.r[f]] = Facc[f];
                    } else if (live) {
                        // bins [jnext, bin_hi]: functionals of this group by (bin, i), 0 where absent
                        const int K1 = P.G.K1;
                        float Fb[kMaxFunc * (kKMax + 1)];
                        for (int e = 0; e < kMaxFunc * (kKMax + 1); ++e) Fb[e] = 0.f;
                        for (int f = 0; f < td.nf; ++f) {
                            const int r = td.r[f];
                            int jj, ii;
                            if (r < P.G.n_if) { jj = r; ii = 0; }
                            else { const int qq = r - P.G.n_if; jj = qq / P.G.k; ii = qq % P.G.k + 1; }
                            const int slot = (jj - td.bin_lo) * K1 + ii;
                            for (int e = 0; e < kMaxFunc * (kKMax + 1); ++e) Fb[e] = e == slot ? Facc[f] : Fb[e];
                        }
                        for (bool first_bin = true; jnext <= td.bin_hi; ++jnext, first_bin = false) {
                            float Fp = 0.f, V[kKMax] = {0.f, 0.f, 0.f};
                            if (jnext >= td.bin_lo) {
                                const int o = (jnext - td.bin_lo) * K1;
                                for (int e = 0; e < kMaxFunc * (kKMax + 1); ++e) {
                                    Fp = e == o ? Fb[e] : Fp;
                                    for (int i = 1; i <= kKMax; ++i) V[i - 1] = e == o + i ? Fb[e] : V[i - 1];
                                }
                            }
                            if (jnext >= P.G.n_if) Fp = 0.f;   // F(x_max) = 0 for conservative fluxes
                            if (!(pre && first_bin)) load_bin(P, cell, jnext, pgn, pgs);
                            update_bin(P, cell, jnext, Fprev, Fp, V, dtc, pgn, pgs, msum, fl, ch, anext, row);
                            Fprev = Fp;
                        }
                    }
                    for (int f = 0; f < kMaxFunc; ++f) Facc[f] = 0.f;
                }
            }
            if (P.mode != 0 && live) {
                const float V0[kKMax] = {0.f, 0.f, 0.f};
                for (; jnext < P.G.N; ++jnext) {   // bins whose functionals all vanish
                    double gnb[kBinMax], gsb[kBinMax];
                    load_bin(P, cell, jnext, gnb, gsb);
                    update_bin(P, cell, jnext, Fprev, 0.f, V0, dtc, gnb, gsb, msum, fl, ch, anext, row);
                    Fprev = 0.f;
                }
                if (anext) chunk_flush(ch, P, anext, row);
                if (P.mass) P.mass[cell] = msum;
                if (P.flags && fl) P.flags[cell] |= (unsigned char)fl;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&S->a_empty));
        }
    }

    // ---------------------------------------------------- teardown
    __syncwarp();
    if (warp == 0 && lane == 0 && *abort_flag) {
        // drain copies still in flight into this CTA's shared memory (bounded)
        for (int s = 0; s < NS; ++s)
            for (int u = S->slot_done[s]; u < S->slot_issued[s]; ++u) {
                const long long t0 = clock64();
                while (!mbar_try_wait(smem_u32(&S->full[s]), u & 1) && clock64() - t0 < kWaitCycles) {
                }
            }
        for (int u = S->a_done; u < S->a_issued; ++u) {
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(&S->a_full), u & 1) && clock64() - t0 < kWaitCycles) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
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
    size_t tiles = ((size_t)n_cells + kTileM - 1) / kTileM;
    tiles += tiles & 1;   // the contraction takes tiles in pairs; a missing partner reads zeros
    return tiles * opA_tile_bytes(prec, kp);
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

grace_status build_tc_tiles(Group &G, int prec, cudaStream_t st)
{
    const DevGroup &g = G.dg;
    if (g.k > 3) {
        set_error("tensor-core tiles need k <= 3");
        return GRACE_ERR_UNSUPPORTED;
    }
    const int P_ = g.P, R = g.R, K1 = g.K1;
    const int ae = atom_elems(prec), eb = elem_bytes(prec), planes = n_planes(prec);
    const int kstep = 32 / eb;   // elements per MMA k-step
    std::vector<double> T((size_t)R * P_ * P_);
    std::vector<int> qlo((size_t)R * P_), qhi((size_t)R * P_), pr(2 * R);
    cudaError_t e = cudaMemcpyAsync(T.data(), G.d_T, T.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(qlo.data(), G.d_qlo, qlo.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(qhi.data(), G.d_qhi, qhi.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pr.data(), G.d_prange, pr.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core tiles: copy T");

    std::vector<double> h(g.N);
    for (int j = 0; j < g.N; ++j) h[j] = G.h_edges[j + 1] - G.h_edges[j];

    // functional groups: whole bins, in bin order, up to kMaxFunc functionals each
    // (the fused update needs every functional of a bin in one group)
    std::vector<std::vector<int>> groups;
    std::vector<std::pair<int, int>> gbins;
    std::vector<int> cur;
    int cur_lo = 0;
    for (int j = 0; j < g.N; ++j) {
        std::vector<int> fj;
        if (j < g.n_if) fj.push_back(j);
        for (int i = 1; i <= g.k; ++i) fj.push_back(g.n_if + j * g.k + i - 1);
        if (fj.size() > (size_t)kMaxFunc) {
            set_error("tensor-core tiles: a bin has more functionals than a tile holds");
            return GRACE_ERR_UNSUPPORTED;
        }
        if (!cur.empty() && cur.size() + fj.size() > (size_t)kMaxFunc) {
            groups.push_back(cur);
            gbins.push_back({cur_lo, j - 1});
            cur.clear();
        }
        if (cur.empty()) cur_lo = j;
        for (int r : fj) cur.push_back(r);
    }
    if (!cur.empty()) {
        groups.push_back(cur);
        gbins.push_back({cur_lo, g.N - 1});
    }

    std::vector<TileDesc> tiles;
    std::vector<uint8_t> B;
    long long macs = 0;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const auto &grp = groups[gi];
        int plo = P_, phi = 0;
        for (int r : grp)
            if (pr[2 * r + 1] > pr[2 * r]) {
                plo = std::min(plo, pr[2 * r]);
                phi = std::max(phi, pr[2 * r + 1]);
            }
        if (phi <= plo) continue;   // all functionals of the group vanish identically
        const int nf = (int)grp.size(), nrows = nf * kWin;
        size_t first_tile = tiles.size();
        for (int w = plo / kWin; w * kWin < phi; ++w) {
            const int p0 = w * kWin;
            int q_lo = P_, q_hi = 0;
            for (int f = 0; f < nf; ++f)
                for (int c = 0; c < kWin; ++c) {
                    const int p = p0 + c;
                    if (p >= P_) continue;
                    const size_t row = (size_t)grp[f] * P_ + p;
                    if (qlo[row] < qhi[row]) {
                        q_lo = std::min(q_lo, qlo[row]);
                        q_hi = std::max(q_hi, qhi[row]);
                    }
                }
            if (q_hi <= q_lo) continue;
            TileDesc td;
            std::memset(&td, 0, sizeof(td));
            td.nrows = nrows;
            td.nf = nf;
            td.ks_lo = q_lo / kstep;
            td.ks_hi = (q_hi + kstep - 1) / kstep;
            td.atom_lo = td.ks_lo / 4;
            td.n_atoms = (td.ks_hi + 3) / 4 - td.atom_lo;
            td.p0 = p0;
            td.bin_lo = gbins[gi].first;
            td.bin_hi = gbins[gi].second;
            for (int f = 0; f < kMaxFunc; ++f) td.r[f] = f < nf ? grp[f] : -1;
            td.b_off = (long long)B.size();
            const size_t atom_plane = (size_t)nrows * 128;
            B.resize(B.size() + (size_t)td.n_atoms * atom_plane * planes, 0);
            uint8_t *img = B.data() + td.b_off;
            for (int a = 0; a < td.n_atoms; ++a) {
                uint8_t *ai = img + (size_t)a * atom_plane * planes;
                for (int f = 0; f < nf; ++f)
                    for (int c = 0; c < kWin; ++c) {
                        const int p = p0 + c, rowi = f * kWin + c;
                        if (p >= P_) continue;
                        const double *Trow = T.data() + ((size_t)grp[f] * P_ + p) * P_;
                        for (int x = 0; x < ae; ++x) {
                            const int qq = (td.atom_lo + a) * ae + x;
                            if (qq >= P_) break;
                            const double val = Trow[qq] / (h[p / K1] * h[qq / K1]);
                            const size_t off = swz_offset(nrows, rowi, x, eb);
                            if (prec == GRACE_TF32) {
                                const uint32_t bits = tf32_bits_rn((float)val);
                                std::memcpy(ai + off, &bits, 4);
                            } else {
                                const uint16_t hi = bf16_bits_rn((float)val);
                                const uint16_t lo = bf16_bits_rn((float)(val - (double)bf16_to_f(hi)));
                                std::memcpy(ai + off, &hi, 2);
                                std::memcpy(ai + atom_plane + off, &lo, 2);
                            }
                        }
                    }
            }
            macs += (long long)nrows * (td.ks_hi - td.ks_lo) * kstep;
            tiles.push_back(td);
        }
        if (tiles.size() > first_tile) tiles.back().flush = 1;
    }
    if (tiles.empty()) {
        set_error("tensor-core tiles: the coefficient tensor is empty");
        return GRACE_ERR_ARG;
    }
    TcTiles &out = G.tc[prec];
    free_tc_tiles(out);
    e = cudaMalloc(&out.d_b, B.size());
    if (e == cudaSuccess) e = cudaMalloc(&out.d_desc, tiles.size() * sizeof(TileDesc));
    if (e == cudaSuccess) e = cudaMemcpy(out.d_b, B.data(), B.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_desc, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_tc_tiles(out);
        return cuda_fail(e, "tensor-core tiles: upload");
    }
    out.n_tiles = (int)tiles.size();
    out.max_rows = 0;
    for (const TileDesc &td : tiles) out.max_rows = std::max(out.max_rows, td.nrows);
    out.k_pad = (P_ + ae - 1) / ae * ae;
    out.b_bytes = B.size();
    out.mac_per_cell = macs;
    out.built = 1;
    return GRACE_OK;
}

static int sm_count(int dev)
{
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <int NT>
static cudaError_t launch_nt(TcParams P, cudaStream_t st)
{
    const size_t fixed = 1024 + (size_t)NT * P.a_tile_bytes + sizeof(Smem) + 64;
    if (fixed + (size_t)P.slot_bytes > (size_t)kSmemLimit) return cudaErrorInvalidValue;
    P.n_slots = (int)std::min<size_t>(kMaxSlots, ((size_t)kSmemLimit - fixed) / P.slot_bytes);
    const size_t smem = fixed + (size_t)P.n_slots * P.slot_bytes;
    cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    const int items = (P.n_cell_tiles + NT - 1) / NT;
    const int grid = std::min(items, sm_count(dev));
    contract_tc_kernel<NT><<<grid, Cfg<NT>::threads, smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_contract_tc(const DevGroup &g, const TcTiles &t, int prec, const void *opA, int n_cells,
                               float *d_F32, int *d_err, cudaStream_t st, int mode, const UpdateArgs *u)
{
    if (!t.built) return cudaErrorInvalidValue;
    if (mode != 0 && !u) return cudaErrorInvalidValue;
    TcParams P;
    std::memset(&P, 0, sizeof(P));
    P.mode = mode;
    P.G = g;
    if (u) {
        P.gn = u->gn;
        P.gs = u->gs;
        P.gout = u->gout;
        P.dt = u->dt;
        P.ca = u->a;
        P.cb = u->b;
        P.apply_limiter = u->apply_limiter;
        P.mass = u->mass;
        P.flags = u->flags;
        P.a_next = (uint8_t *)u->opA;
    }
    P.tiles = (const TileDesc *)t.d_desc;
    P.n_tiles = t.n_tiles;
    P.B = (const uint8_t *)t.d_b;
    P.A = (const uint8_t *)opA;
    P.a_tile_bytes = (long long)opA_tile_bytes(prec, t.k_pad);
    P.n_cells = n_cells;
    P.n_cell_tiles = (n_cells + kTileM - 1) / kTileM;
    P.R = g.R;
    P.F = d_F32;
    P.prec = prec;
    P.slot_bytes = t.max_rows * 128 * n_planes(prec);
    P.n_slots = 0;
    P.err = d_err;
    // two cell tiles per CTA pass when both A tiles and a 4-deep B ring fit, else one
    const size_t pair_need = 1024 + 2 * (size_t)P.a_tile_bytes + sizeof(Smem) + 64 + 4 * (size_t)P.slot_bytes;
    if (pair_need <= (size_t)kSmemLimit && P.n_cell_tiles > 1) return launch_nt<2>(P, st);
    return launch_nt<1>(P, st);
}

}  // namespace grace
