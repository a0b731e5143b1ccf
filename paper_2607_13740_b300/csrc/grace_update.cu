// K-c: fused flux difference, SSP-RK3 stage update, scaling limiter, mass and flags.
//
// One warp per cell, one lane per bin.  Lane j reads the cell's flux
// functionals F(x_{j-1/2}), F(x_{j+1/2}) and the volume terms of bin j,
// forms L_j^i of eq. (evo), combines it with the stage inputs as in eq.
// (RK3), optionally applies the scaling limiter of eqs. (recon)/(gamma) to the
// result (the reconstruction that opens the next step), writes the bin, and
// adds h_j g_j^0 to the cell's mass (warp-shuffle reduction, FP64).  The
// i = 0 row only ever sees F(x_{j-1/2}) - F(x_{j+1/2}), so the sum of h_j L_j^0
// telescopes and the mass is conserved to round-off whatever precision the
// functionals came from.
#include "grace_convert.cuh"
#include "grace_limiter.cuh"
#include "grace_tc_layout.cuh"

namespace grace {

namespace {

constexpr int kB = kKMax + 1;

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned warp_or(unsigned v)
{
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// asynchronous global -> shared copies of 4 or 8 bytes (a thread issues all of its copies
// before waiting, so a block has its whole input in flight at once)
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Writes one cell's new coefficients, staged in shared memory, to the FP64 state
// (coalesced) and, if requested, to the cell's row of the tensor-core A operand
// as whole 16-byte chunks (TF32: 4 values, BF16: 8 hi + 8 lo values per chunk).
__device__ __forceinline__ void write_row(const DevGroup &G, const double *row, long long cell, double *gout,
                                          void *opA, int prec, int kpad, int lane)
{
    const int P = G.P;
    if (gout)
        for (int i = lane; i < P; i += 32) gout[(size_t)cell * P + i] = row[i];
    if (!opA) return;
    const long long tile = cell / kTileM;
    const int r = (int)(cell - tile * kTileM);
    char *t = (char *)opA + (size_t)tile * opA_tile_bytes(prec, kpad);
    if (prec == GRACE_TF32) {
        for (int c = lane; c * 4 < P; c += 32) {
            uint32_t w[4];
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * c + e;
                w[e] = k < P ? f32_to_tf32_rna((float)(row[k] * G.hbin[k / G.K1])) : 0u;
            }
            *reinterpret_cast<uint4 *>(t + swz_offset(kTileM, r, 4 * c, 4)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        const size_t plane = (size_t)kTileM * kpad * 2;
        for (int c = lane; c * 8 < P; c += 32) {
            uint32_t hi[4], lo[4];
            for (int e = 0; e < 4; ++e) {
                uint32_t h2[2], l2[2];
                for (int u = 0; u < 2; ++u) {
                    const int k = 8 * c + 2 * e + u;
                    const double v = k < P ? row[k] * G.hbin[k / G.K1] : 0.0;
                    const __nv_bfloat16 h = __double2bfloat16(v);
                    const __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
                    h2[u] = (uint32_t)__bfloat16_as_ushort(h);
                    l2[u] = (uint32_t)__bfloat16_as_ushort(l);
                }
                hi[e] = h2[0] | (h2[1] << 16);
                lo[e] = l2[0] | (l2[1] << 16);
            }
            const size_t off = swz_offset(kTileM, r, 8 * c, 2);
            *reinterpret_cast<uint4 *>(t + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(t + plane + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

// The plain path: FP64 functionals in the [cell][functional] layout, everything
// in FP64.  One warp per cell; the new row is staged in shared memory and
// written out coalesced.
__global__ void __launch_bounds__(256) update_kernel(DevGroup G, UpdateArgs A, int n_cells)
{
    extern __shared__ double rows[];
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const int N = G.N, k = G.k, K1 = G.K1, R = G.R, P = G.P;
    double *row = rows + (size_t)(threadIdx.x >> 5) * P;
    const double *F = A.F + cell * R;
    const bool step = A.dt != nullptr;
    const double dt = step ? A.dt[cell] : 0.0;
    double msum = 0.0;
    unsigned fl = 0u;
    for (int j = lane; j < N; j += 32) {
        const double Fm = j == 0 ? 0.0 : F[j - 1];             // F(x_{j-1/2}), F(x_min) = 0
        const double Fp = j < G.n_if ? F[j] : 0.0;             // F(x_{j+1/2}), 0 at x_max (cons.)
        const size_t base = (size_t)cell * P + (size_t)j * K1;
        double v[kB];
        const double ih = G.inv_h[j];
        const double L0 = (Fm - Fp) * ih;
        v[0] = step ? A.a * A.gn[base] + A.b * (A.gs[base] + dt * L0) : L0;
        for (int i = 1; i <= k; ++i) {
            const double V = F[G.n_if + j * k + i - 1];
            const double L = (2.0 * i + 1.0) * ih * (V - Fp + ((i & 1) ? -Fm : Fm));
            v[i] = step ? A.a * A.gn[base + i] + A.b * (A.gs[base + i] + dt * L) : L;
        }
        if (step) {
            // eq. (dt) for this stage's forward-Euler update of the mean
            if (L0 < 0.0 && fma(dt, L0, A.gs[base]) <= 0.0) fl |= GRACE_FLAG_CFL;
            if (v[0] < 0.0) fl |= GRACE_FLAG_NEGATIVE_MEAN;
            for (int i = 0; i <= k; ++i)
                if (!isfinite(v[i])) fl |= GRACE_FLAG_NONFINITE;
            if (A.apply_limiter) fl |= limit_bin(v, k);
        }
        for (int i = 0; i <= k; ++i) row[j * K1 + i] = v[i];
        if (A.mass) msum += G.hbin[j] * v[0];
    }
    __syncwarp();
    write_row(G, row, cell, A.gout, A.opA, A.opA_prec, A.opA_kpad, lane);
    if (A.mass) {
        msum = warp_sum(msum);
        if (lane == 0) A.mass[cell] = msum;
    }
    if (A.flags) {
        fl = warp_or(fl);
        if (lane == 0 && fl) A.flags[cell] |= (unsigned char)fl;
    }
}

__global__ void __launch_bounds__(256) limit_kernel(DevGroup G, double *g, int n_cells, unsigned char *flags,
                                                     void *opA, int prec, int kpad)
{
    extern __shared__ double rows[];
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const int k = G.k, K1 = G.K1, P = G.P;
    double *row = rows + (size_t)(threadIdx.x >> 5) * P;
    for (int i = lane; i < P; i += 32) row[i] = g[(size_t)cell * P + i];
    __syncwarp();
    unsigned fl = 0u, changed = 0u;
    for (int j = lane; j < G.N; j += 32) {
        double *v = row + j * K1;
        if (G.limiter) {
            const unsigned f = limit_bin(v, k);
            if (f & GRACE_FLAG_LIMITED) changed = 1u;
            fl |= f;
        }
    }
    __syncwarp();
    changed = warp_or(changed);
    write_row(G, row, cell, changed ? g : nullptr, opA, prec, kpad, lane);
    if (flags) {
        fl = warp_or(fl);
        if (lane == 0 && fl) flags[cell] |= (unsigned char)fl;
    }
}

// ---------------------------------------------------------------------------
// K-c for the tensor path.  LPC lanes per cell (8, 16 or 32), lane l taking bins
// l, l + LPC, ...  Each block first copies its cells' functionals (from the
// contraction's [tile][functional][row] layout) into shared memory with cp.async;
// with compact stage inputs and a compact result it copies the stage inputs too,
// so every load of the block is in flight at once.  Otherwise the stage inputs
// are read bin by bin.  A compact result is written by each lane directly; an
// FP64 row and the A-operand row are assembled in shared memory and written out
// coalesced.  Only the mean row (i = 0: flux difference, stage combination, the
// eq. (dt) test, mass) uses FP64 arithmetic; the higher modes, the limiter and
// all conversions run on the FP32 and integer pipes.
//   MODE_RHS   : gout = L[g]                            (F32 required)
//   MODE_STAGE : gout = a gn + b (gs + dt L[gs]), then the limiter when asked
//   MODE_LIMIT : g = limit(g) (when asked) and the next A operand (no F32)
// In every mode the A operand of the result (ghat = g h_bin, TF32 or BF16 hi/lo)
// is written when A.opA is set.
enum { MODE_RHS = 0, MODE_STAGE = 1, MODE_LIMIT = 2 };
constexpr int kUpdWarps = 8;
constexpr int kGroupedLpc = 16;     // lanes per cell of the grouped launch (16 cells per block)

// LPC lanes per cell (8, 16 or 32, whichever leaves fewer lanes idle for N bins);
// lane l of a cell handles bins l, l + LPC, ...
//
// State layouts: FP64 rows [cell][bin][i] (the caller's), or the compact stage
// layout used inside grace_step for the tensor forms ("mixed"): for a part of n
// cells, the means [n][N] in FP64 followed by the higher modes [n][N][k] in FP32
// (the tensor forms carry the higher modes at FP32 precision anyway).  IN_MIX /
// OUT_MIX select the layout of the stage inputs / the result.
template <int MODE, int LPC, bool IN_MIX, bool OUT_MIX>
__device__ __forceinline__ void update_tc_body(const DevGroup &G, const UpdateArgs &A, int n_cells, long long block)
{
    extern __shared__ double sm[];
    constexpr int CPB = kUpdWarps * 32 / LPC;                     // cells per block (a divisor of 128)
    // compact stage inputs and compact output: the block's stage inputs are staged in shared
    // memory (the FP64 row buffer is not needed, so a cell's region holds only its ghat row)
    constexpr bool STAGED = MODE == MODE_STAGE && IN_MIX && OUT_MIX;
    const int N = G.N, k = G.k, K1 = G.K1, P = G.P, R = G.R;
    const int slot = threadIdx.x / LPC, lane = threadIdx.x % LPC;
    const long long cell0 = block * CPB;
    const long long cell = cell0 + slot;
    const int lda = A.opA_kpad;
    const size_t cell_dbl = (STAGED ? 0 : P) + lda / 2 + 1;       // doubles per cell region
    double *row = sm + (size_t)slot * cell_dbl;                   // new coefficients of the cell
    float *arow = reinterpret_cast<float *>(row + (STAGED ? 0 : P));  // its ghat row (A operand), kpad floats
    // the block's functionals, transposed to [cell][functional]: read from the contraction's
    // [tile][functional][row] layout as CPB-float pieces of each functional's row
    float *Fs = reinterpret_cast<float *>(sm + (size_t)CPB * cell_dbl);
    // staged inputs: means of g^(s) and g^n [CPB][N] (FP64), higher modes [CPB][N][k] (FP32)
    double *St_s = sm + (size_t)CPB * cell_dbl + ((size_t)CPB * (R + 1) + 1) / 2;
    double *St_n = St_s + (size_t)CPB * N;
    float *St_sh = reinterpret_cast<float *>(St_n + (size_t)CPB * N);
    float *St_nh = St_sh + (size_t)CPB * N * k;
    const size_t nN = (size_t)n_cells * N;
    if (MODE != MODE_LIMIT) {
        const int nc = (int)min((long long)CPB, (long long)n_cells - cell0);
        if (STAGED) {
            // the block's cells are contiguous in both arrays of the compact layout
            const double *gsm = A.gs + (size_t)cell0 * N, *gnm = A.gn + (size_t)cell0 * N;
            const float *gsh = reinterpret_cast<const float *>(A.gs + nN) + (size_t)cell0 * N * k;
            const float *gnh = reinterpret_cast<const float *>(A.gn + nN) + (size_t)cell0 * N * k;
            for (int i = threadIdx.x; i < nc * N; i += 32 * kUpdWarps) {
                cp_async8(St_s + i, gsm + i);
                cp_async8(St_n + i, gnm + i);
            }
            for (int i = threadIdx.x; i < nc * N * k; i += 32 * kUpdWarps) {
                cp_async4(St_sh + i, gsh + i);
                cp_async4(St_nh + i, gnh + i);
            }
        }
        const float *Ft = A.F32 + ((size_t)(cell0 >> 7) * R) * kTileM + (cell0 & (kTileM - 1));
        for (int idx = threadIdx.x; idx < R * CPB; idx += 32 * kUpdWarps) {
            const int r = idx / CPB, c = idx - r * CPB;
            if (c < nc) cp_async4(Fs + c * (R + 1) + r, Ft + (size_t)r * kTileM + c);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    if (cell >= n_cells) return;   // whole groups of LPC lanes leave together
    const float *F = Fs + slot * (R + 1);
    // stage inputs: s = gs (MODE_STAGE), or the state to limit (MODE_LIMIT, FP64 rows in A.gs)
    const double *srcs = A.gs;
    const double *srcn = MODE == MODE_STAGE ? A.gn : srcs;
    const double dt = MODE == MODE_STAGE ? A.dt[cell] : 0.0;
    const float af = (float)A.a, bf = (float)A.b, dtf = MODE == MODE_STAGE ? d2f_fast(dt) : 0.f;
    double msum = 0.0;
    unsigned fl = 0u;
    for (int j = lane; j < N; j += LPC) {
        // inputs of bin j: means (FP64) and higher modes (FP32 values, FP64 for MODE_LIMIT)
        double s0 = 0.0, n0 = 0.0;
        float sf[kB], nf_[kB];
        double vd[kB];     // MODE_LIMIT: the FP64 higher modes
        if (MODE != MODE_RHS) {
            if (STAGED) {
                s0 = St_s[slot * N + j];
                n0 = St_n[slot * N + j];
                const float *sh = St_sh + (size_t)(slot * N + j) * k;
                const float *nh = St_nh + (size_t)(slot * N + j) * k;
#pragma unroll
                for (int i = 1; i < kB; ++i) {
                    sf[i] = i <= k ? sh[i - 1] : 0.f;
                    nf_[i] = i <= k ? nh[i - 1] : 0.f;
                    vd[i] = f2d_fast(sf[i]);
                }
            } else if (IN_MIX) {
                s0 = srcs[cell * N + j];
                n0 = srcn[cell * N + j];
                const float *sh = reinterpret_cast<const float *>(srcs + nN) + ((size_t)cell * N + j) * k;
                const float *nh = reinterpret_cast<const float *>(srcn + nN) + ((size_t)cell * N + j) * k;
#pragma unroll
                for (int i = 1; i < kB; ++i) {
                    sf[i] = i <= k ? sh[i - 1] : 0.f;
                    nf_[i] = i <= k ? nh[i - 1] : 0.f;
                    vd[i] = f2d_fast(sf[i]);
                }
            } else {
                const double *vs = srcs + (size_t)cell * P + (size_t)j * K1;
                const double *vn = srcn + (size_t)cell * P + (size_t)j * K1;
                s0 = vs[0];
                n0 = vn[0];
#pragma unroll
                for (int i = 1; i < kB; ++i) {
                    vd[i] = i <= k ? vs[i] : 0.0;
                    sf[i] = d2f_fast(vd[i]);
                    nf_[i] = i <= k ? d2f_fast(vn[i]) : 0.f;
                }
            }
        }
        double v0;
        float vf[kB];
        if (MODE == MODE_LIMIT) {
            v0 = s0;
#pragma unroll
            for (int i = 1; i < kB; ++i) vf[i] = sf[i];
        } else {
            const float Fm = j == 0 ? 0.f : F[j - 1];          // F(x_{j-1/2}), F(x_min) = 0
            const float Fp = j < G.n_if ? F[j] : 0.f;           // F(x_{j+1/2}), 0 at x_max (cons.)
            const double L0 = (f2d_fast(Fm) - f2d_fast(Fp)) * G.inv_h[j];
            if (MODE == MODE_STAGE) {
                const double euler = fma(dt, L0, s0);
                v0 = fma(A.a, n0, A.b * euler);
                // eq. (dt) for this stage's forward-Euler update of the mean; L0 < 0
                // exactly when Fm < Fp (inv_h > 0, and the FP64 difference keeps the sign)
                if (Fm < Fp && nonpositive_bits(euler)) fl |= GRACE_FLAG_CFL;
            } else {
                v0 = L0;
            }
            const float ih = G.inv_h32[j];
#pragma unroll
            for (int i = 1; i < kB; ++i) {
                vf[i] = 0.f;
                if (i <= k) {
                    const float V = F[G.n_if + j * k + i - 1];
                    const float L = (2.f * i + 1.f) * ih * (V - Fp + ((i & 1) ? -Fm : Fm));
                    vf[i] = MODE == MODE_STAGE ? af * nf_[i] + bf * (sf[i] + dtf * L) : L;
                }
            }
        }
        if (MODE == MODE_STAGE) {
            if (negative_bits(v0)) fl |= GRACE_FLAG_NEGATIVE_MEAN;
            bool nf = nonfinite_bits(v0);
#pragma unroll
            for (int i = 1; i < kB; ++i) nf = nf || (i <= k && nonfinite_bits(vf[i]));
            if (nf) fl |= GRACE_FLAG_NONFINITE;
        }
        bool changed = false;   // the limiter scaled this bin's higher modes
        if (MODE != MODE_RHS && A.apply_limiter && k > 0) {
            // FP32 limiter on the bin rescaled to a mean in [1, 2); the exact FP64
            // limiter only for a mean <= 0, subnormal or not finite
            const int e0 = scaled_exponent(v0);
            float gam = -1.f;
            if (e0 >= 0) {
                float cf[kB];
#pragma unroll
                for (int i = 1; i < kB; ++i)
                    cf[i] = i > k ? 0.f
                                  : (MODE == MODE_LIMIT && !IN_MIX ? d2f_scaled(vd[i], 1023 - e0)
                                                                   : scale_pow2(vf[i], 1023 - e0));
                gam = limiter_gamma_scaled(v0, cf, k);
            }
            if (gam < 0.f) {
                bool zero = ((unsigned long long)__double_as_longlong(v0) << 1) == 0ull;
#pragma unroll
                for (int i = 1; i < kB; ++i)
                    zero = zero && (i > k || (MODE == MODE_LIMIT ? ((unsigned long long)__double_as_longlong(vd[i]) << 1) == 0ull
                                                                 : vf[i] == 0.f));
                if (!zero) {
                    double v[kB];
                    v[0] = v0;
#pragma unroll
                    for (int i = 1; i < kB; ++i) v[i] = i <= k ? (MODE == MODE_LIMIT ? vd[i] : f2d_fast(vf[i])) : 0.0;
                    const unsigned f = limit_bin(v, k);
                    fl |= f;
                    if (f & GRACE_FLAG_LIMITED) {
                        changed = true;
#pragma unroll
                        for (int i = 1; i < kB; ++i) {
                            vd[i] = v[i];
                            vf[i] = (float)v[i];
                        }
                    }
                }
            } else if (gam < 1.f) {
                fl |= GRACE_FLAG_LIMITED;
                changed = true;
#pragma unroll
                for (int i = 1; i < kB; ++i) {
                    if (MODE == MODE_LIMIT) {
                        vd[i] *= (double)gam;
                        vf[i] = d2f_fast(vd[i]);
                    } else {
                        vf[i] *= gam;
                    }
                }
            }
            // MODE_LIMIT into the caller's FP64 rows rewrites only the bins it changed
            if (MODE == MODE_LIMIT && !OUT_MIX && changed)
#pragma unroll
                for (int i = 1; i < kB; ++i)
                    if (i <= k) A.gout[(size_t)cell * P + (size_t)j * K1 + i] = vd[i];
        }
        if (OUT_MIX) {
            // the compact layout: lane j writes its bin's mean and modes directly (coalesced)
            A.gout[cell * N + j] = v0;
            float *oh = reinterpret_cast<float *>(A.gout + nN) + ((size_t)cell * N + j) * k;
#pragma unroll
            for (int i = 1; i < kB; ++i)
                if (i <= k) oh[i - 1] = vf[i];
        } else if (MODE != MODE_LIMIT) {
            double *rj = row + j * K1;
            rj[0] = v0;
#pragma unroll
            for (int i = 1; i < kB; ++i)
                if (i <= k) rj[i] = f2d_fast(vf[i]);
        }
        if (A.opA) {
            const float h = G.h32[j];
            float *ar = arow + A.opA_kofs + j * K1;
            ar[0] = d2f_fast(v0) * h;
#pragma unroll
            for (int i = 1; i < kB; ++i)
                if (i <= k) ar[i] = vf[i] * h;
        }
        if (A.mass) msum = fma(G.hbin[j], v0, msum);
    }
    const unsigned gmask = LPC == 32 ? 0xffffffffu : (((1u << LPC) - 1u) << (threadIdx.x & (32 - LPC)));
    if (A.opA) {
        for (int e = lane; e < A.opA_kofs; e += LPC) arow[e] = 0.f;
        for (int e = A.opA_kofs + P + lane; e < lda; e += LPC) arow[e] = 0.f;
    }
    __syncwarp(gmask);
    // coalesced stores of an FP64 result row (the compact layout was written above)
    if (MODE != MODE_LIMIT && !OUT_MIX) {
        double *go = A.gout + (size_t)cell * P;
        for (int e = lane; e < P; e += LPC) go[e] = row[e];
    }
    if (A.opA) {
        const long long tile = cell / kTileM;
        const int r = (int)(cell - tile * kTileM);
        char *t = (char *)A.opA + (size_t)tile * opA_tile_bytes(A.opA_prec, lda);
        if (A.opA_prec == GRACE_TF32) {
            for (int qc = lane; qc < lda / 4; qc += LPC) {
                const float *x = arow + 4 * qc;
                *reinterpret_cast<uint4 *>(t + swz_offset(kTileM, r, 4 * qc, 4)) =
                    make_uint4(f32_to_tf32_rna(x[0]), f32_to_tf32_rna(x[1]), f32_to_tf32_rna(x[2]), f32_to_tf32_rna(x[3]));
            }
        } else {
            const size_t plane = (size_t)kTileM * lda * 2;
            for (int qc = lane; qc < lda / 8; qc += LPC) {
                const float *x = arow + 8 * qc;
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * e]), h1 = __float2bfloat16_rn(x[2 * e + 1]);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * e] - __bfloat162float(h0));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * e + 1] - __bfloat162float(h1));
                    hi[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    lo[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
                const size_t off = swz_offset(kTileM, r, 8 * qc, 2);
                *reinterpret_cast<uint4 *>(t + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4 *>(t + plane + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
        }
    }
    if (A.mass) {
        for (int o = LPC / 2; o > 0; o >>= 1) msum += __shfl_xor_sync(gmask, msum, o);
        if (lane == 0) A.mass[cell] = msum;
    }
    if (A.flags) {
        for (int o = LPC / 2; o > 0; o >>= 1) fl |= __shfl_xor_sync(gmask, fl, o);
        if (lane == 0 && fl) A.flags[cell] |= (unsigned char)fl;
    }
}

template <int MODE, int LPC, bool IN_MIX, bool OUT_MIX>
__global__ void __launch_bounds__(32 * kUpdWarps, 3) update_tc_kernel(DevGroup G, UpdateArgs A, int n_cells)
{
    update_tc_body<MODE, LPC, IN_MIX, OUT_MIX>(G, A, n_cells, blockIdx.x);
}

// K-c over the parts of a batch in one launch: block b belongs to the part with the largest
// first_block <= b; the part's descriptor is staged in shared memory
template <int MODE, bool IN_MIX, bool OUT_MIX>
__global__ void __launch_bounds__(32 * kUpdWarps, 3) update_tc_grouped_kernel(const UpdPart *__restrict__ parts,
                                                                              int n_parts)
{
    __shared__ UpdPart sp;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_parts - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (parts[mid].first_block <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        sp = parts[lo];
    }
    __syncthreads();
    update_tc_body<MODE, kGroupedLpc, IN_MIX, OUT_MIX>(sp.G, sp.A, sp.n_cells, (long long)blockIdx.x - sp.first_block);
}

__global__ void __launch_bounds__(256) mass_kernel(DevGroup G, const double *g, int n_cells, double *mass)
{
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    double s = 0.0;
    for (int j = lane; j < G.N; j += 32) s += G.hbin[j] * g[(size_t)cell * G.P + (size_t)j * G.K1];
    s = warp_sum(s);
    if (lane == 0) mass[cell] = s;
}

struct Rule16 {
    double s[16], w[16];
};

// eq. (init) with a 16-point Gauss rule per bin; one thread per (cell, bin)
__global__ void project_kernel(DevGroup G, Rule16 rule, int kind, const double *ic, int n_cells, double *g)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_cells * G.N) return;
    const long long cell = t / G.N;
    const int j = (int)(t - cell * G.N);
    const double *q = ic + cell * 4;
    const double lo = G.edges[j], hi = G.edges[j + 1];
    const double h = hi - lo, xc = 0.5 * (lo + hi);
    double acc[kB] = {0.0, 0.0, 0.0, 0.0}, P[kB];
    for (int a = 0; a < 16; ++a) {
        const double x = xc + 0.5 * h * rule.s[a];
        double val = 0.0;
        if (kind == GRACE_IC_EXP) val = q[0] * x * exp(-x / q[1]);
        else if (kind == GRACE_IC_POWERLAW) val = (x >= q[2] && x <= q[3]) ? q[0] * pow(x, q[1]) : 0.0;
        else if (kind == GRACE_IC_FIRST_BIN) val = x < G.edges[1] ? q[0] : 0.0;
        dev_legendre(G.k, rule.s[a], P, nullptr);
        for (int i = 0; i <= G.k; ++i) acc[i] += rule.w[a] * val * P[i];
    }
    for (int i = 0; i <= G.k; ++i) g[(size_t)cell * G.P + (size_t)j * G.K1 + i] = acc[i] * (2.0 * i + 1.0) * 0.5;
}

inline int warp_blocks(int n_cells) { return (int)(((long long)n_cells * 32 + 255) / 256); }

}  // namespace

cudaError_t launch_update(const DevGroup &g, const UpdateArgs &a, int n_cells, cudaStream_t st)
{
    if (!a.F) return cudaErrorInvalidValue;
    const size_t smem = (size_t)8 * g.P * sizeof(double);   // one row per warp (P > 768: above 48 KB)
    cudaError_t e = cudaFuncSetAttribute(update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    update_kernel<<<warp_blocks(n_cells), 256, smem, st>>>(g, a, n_cells);
    return cudaGetLastError();
}

// shared memory a block may opt in to on the current device
size_t update_smem_limit()
{
    static int cached[64] = {0};   // per device ordinal, read once
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess) cached[dev] = v;
    }
    // an attribute that cannot be read leaves the choice to the launch itself
    return cached[dev] ? (size_t)cached[dev] : ~(size_t)0;
}

// shared memory of update_tc_kernel: one row (P doubles; not with compact stage inputs and
// output) and one ghat row (kpad floats) per cell, then the block's functionals [cells][R + 1]
// floats, then (compact stage inputs and output) the staged inputs: 2 x [cells][N] doubles and
// 2 x [cells][N][k] floats
static size_t update_tc_smem(const DevGroup &g, const UpdateArgs &a, int lpc)
{
    const size_t cpb = (size_t)kUpdWarps * 32 / lpc;
    const bool staged = a.dt && a.F32 && a.in_mixed && a.out_mixed;
    const size_t cell_dbl = (staged ? 0 : g.P) + a.opA_kpad / 2 + 1;
    size_t bytes = (cpb * cell_dbl + (cpb * (g.R + 1) + 1) / 2) * sizeof(double);
    if (staged) bytes += cpb * g.N * (2 * sizeof(double) + 2 * sizeof(float) * g.k);
    return bytes;
}

template <int MODE, int LPC, bool IN_MIX, bool OUT_MIX>
static cudaError_t launch_update_lpc(const DevGroup &g, const UpdateArgs &a, int n_cells, cudaStream_t st)
{
    const size_t smem = update_tc_smem(g, a, LPC);
    cudaError_t e = cudaFuncSetAttribute(update_tc_kernel<MODE, LPC, IN_MIX, OUT_MIX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int per_block = kUpdWarps * 32 / LPC;
    update_tc_kernel<MODE, LPC, IN_MIX, OUT_MIX>
        <<<(n_cells + per_block - 1) / per_block, 32 * kUpdWarps, smem, st>>>(g, a, n_cells);
    return cudaGetLastError();
}

template <int MODE, bool IN_MIX, bool OUT_MIX>
static cudaError_t launch_update_mode(const DevGroup &g, const UpdateArgs &a, int n_cells, cudaStream_t st)
{
    // lanes per cell: the choice that leaves fewer lanes idle over the N bins (8 only when it idles
    // strictly fewer: measured on N = 40, 8 lanes x 5 bins take 75 us per stage vs 97 us for 16 lanes
    // x 2-3 bins at 65,536 cells); when its block's shared memory does not fit, more lanes per cell
    // (fewer cells per block)
    const int idle8 = (g.N + 7) / 8 * 8 - g.N, idle16 = (g.N + 15) / 16 * 16 - g.N;
    const int idle32 = (g.N + 31) / 32 * 32 - g.N;
    const int pref = idle8 < idle16 && idle8 < idle32 ? 8 : (idle16 <= idle32 ? 16 : 32);
    const size_t limit = update_smem_limit();
    for (int lpc = pref; lpc <= 32; lpc *= 2) {
        if (update_tc_smem(g, a, lpc) > limit) continue;
        if (lpc == 8) return launch_update_lpc<MODE, 8, IN_MIX, OUT_MIX>(g, a, n_cells, st);
        if (lpc == 16) return launch_update_lpc<MODE, 16, IN_MIX, OUT_MIX>(g, a, n_cells, st);
        return launch_update_lpc<MODE, 32, IN_MIX, OUT_MIX>(g, a, n_cells, st);
    }
    return cudaErrorInvalidValue;   // even 8 cells per block exceed the shared memory of a block
}

int update_tc_grouped_cpb() { return kUpdWarps * 32 / kGroupedLpc; }

size_t update_tc_grouped_smem(const DevGroup &g, const UpdateArgs &a) { return update_tc_smem(g, a, kGroupedLpc); }

size_t update_tc_grouped_max_smem(const DevGroup &g, int kpad)
{
    // the largest of the grouped launches: a stage with compact inputs and output (staged
    // inputs), the last stage (FP64 row buffer) and the step-start limiter
    double one = 0.0;
    float onef = 0.f;
    UpdateArgs staged, last;
    staged.dt = last.dt = &one;
    staged.F32 = last.F32 = &onef;
    staged.in_mixed = staged.out_mixed = last.in_mixed = 1;
    staged.opA_kpad = last.opA_kpad = kpad;
    return std::max(update_tc_smem(g, staged, kGroupedLpc), update_tc_smem(g, last, kGroupedLpc));
}

template <int MODE, bool IN_MIX, bool OUT_MIX>
static cudaError_t launch_grouped(const UpdPart *d_parts, int n_parts, int n_blocks, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(update_tc_grouped_kernel<MODE, IN_MIX, OUT_MIX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    update_tc_grouped_kernel<MODE, IN_MIX, OUT_MIX><<<n_blocks, 32 * kUpdWarps, smem, st>>>(d_parts, n_parts);
    return cudaGetLastError();
}

cudaError_t launch_update_tc_grouped(int mode, bool in_mixed, bool out_mixed, const UpdPart *d_parts, int n_parts,
                                     int n_blocks, size_t smem, cudaStream_t st)
{
    if (n_blocks <= 0 || n_parts <= 0) return cudaSuccess;
    if (mode == GROUPED_LIMIT && !in_mixed && out_mixed)
        return launch_grouped<MODE_LIMIT, false, true>(d_parts, n_parts, n_blocks, smem, st);
    if (mode == GROUPED_STAGE && in_mixed && out_mixed)
        return launch_grouped<MODE_STAGE, true, true>(d_parts, n_parts, n_blocks, smem, st);
    if (mode == GROUPED_STAGE && in_mixed && !out_mixed)
        return launch_grouped<MODE_STAGE, true, false>(d_parts, n_parts, n_blocks, smem, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_update_tc(const DevGroup &g, const UpdateArgs &a, int n_cells, cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    if (!a.F32 || !a.gout) return cudaErrorInvalidValue;
    if (!a.dt) return launch_update_mode<MODE_RHS, false, false>(g, a, n_cells, st);
    if (a.in_mixed && a.out_mixed) return launch_update_mode<MODE_STAGE, true, true>(g, a, n_cells, st);
    if (a.in_mixed) return launch_update_mode<MODE_STAGE, true, false>(g, a, n_cells, st);
    if (a.out_mixed) return cudaErrorInvalidValue;
    return launch_update_mode<MODE_STAGE, false, false>(g, a, n_cells, st);
}

cudaError_t launch_limit_pack(const DevGroup &g, const double *d_g, int n_cells, unsigned char *flags,
                              double *mixed_out, void *opA, int opA_prec, int opA_kpad, int opA_kofs,
                              cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    UpdateArgs a;
    a.gs = d_g;
    a.gout = mixed_out;
    a.apply_limiter = g.limiter;
    a.flags = flags;
    a.opA = opA;
    a.opA_prec = opA_prec;
    a.opA_kpad = opA_kpad;
    a.opA_kofs = opA_kofs;
    a.out_mixed = 1;
    return launch_update_mode<MODE_LIMIT, false, true>(g, a, n_cells, st);
}

cudaError_t launch_limit(const DevGroup &g, double *d_g, int n_cells, unsigned char *flags, void *opA,
                         int opA_prec, int opA_kpad, int opA_kofs, cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    if (opA) {
        // tensor path: limiter pre-test off the FP64 pipe, and the A operand
        UpdateArgs a;
        a.gs = d_g;
        a.gout = d_g;
        a.apply_limiter = g.limiter;
        a.flags = flags;
        a.opA = opA;
        a.opA_prec = opA_prec;
        a.opA_kpad = opA_kpad;
        a.opA_kofs = opA_kofs;
        return launch_update_mode<MODE_LIMIT, false, false>(g, a, n_cells, st);
    }
    const size_t smem = (size_t)8 * g.P * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(limit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    limit_kernel<<<warp_blocks(n_cells), 256, smem, st>>>(g, d_g, n_cells, flags, opA, opA_prec, opA_kpad);
    return cudaGetLastError();
}

cudaError_t launch_mass(const DevGroup &g, const double *d_g, int n_cells, double *mass, cudaStream_t st)
{
    mass_kernel<<<warp_blocks(n_cells), 256, 0, st>>>(g, d_g, n_cells, mass);
    return cudaGetLastError();
}

cudaError_t launch_project(const DevGroup &g, int ic_kind, const double *ic, int n_cells, double *d_g,
                           cudaStream_t st)
{
    Rule16 rule;
    gauss_rule(16, rule.s, rule.w);
    const long long n = (long long)n_cells * g.N;
    project_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, rule, ic_kind, ic, n_cells, d_g);
    return cudaGetLastError();
}

cudaError_t launch_pack_A(const DevGroup &g, const double *d_g, int n_cells, void *opA, int prec, int kpad,
                          int kofs, cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    UpdateArgs a;
    a.gs = d_g;            // read only: MODE_LIMIT without the limiter writes no rows
    a.opA = opA;
    a.opA_prec = prec;
    a.opA_kpad = kpad;
    a.opA_kofs = kofs;
    return launch_update_mode<MODE_LIMIT, false, false>(g, a, n_cells, st);
}

}  // namespace grace
