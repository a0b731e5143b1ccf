// a4': flux functionals of groups whose kernel has a per-cell parameter
// (non-separable: the functionals are no longer fixed quadratic forms of the
// coefficients, so no T can be precomputed).
//
// The ballistic-turbulent kernels depend on the cell's alpha_turb only through
// s = sqrt(alpha) and the fragmentation ramp pf(s D0), with D0 a function of the
// larger colliding particle alone (grace_physics.cuh):
//     K_coag = s S0(u, v) (1 - pf(s D0(max(u, v)))),   K_frag = s S0(u, v) pf(s D0(max(u, v))).
// Every flux functional is the nested Gauss sum of Sec. 3.3 / App. B over node
// pairs (u, v) of w(u, v) K(u, v) g(u) g(v) with cell-independent weights w.  The
// pairs split into
//   * fixed pairs: u and v are Gauss nodes of whole bins (shared by many
//     functionals).  With G_a = g at fixed node a (nodes in increasing size), the
//     pair's kernel factor depends on the larger node max(a, b) only, so the fixed
//     part of functional r is
//         s [ G^T Cc_r Hc + G^T Cf_r Hf ],   Hc = (1 - pf(s D0)) (.) G,  Hf = pf(s D0) (.) G,
//     with C{c,f}_r = fold(B{c,f}_r), B{c,f}_r[a][b] the summed weights x S0 of the
//     coagulation / fragmentation terms, fold(M)[i][j] = M[i][j] + M[j][i] (i < j),
//     M[i][i] on the diagonal (upper triangle, the larger node on the H side).
//     The two products are kept apart (not Hf = G - Hc) so that a vanishing
//     fragmentation probability contributes an exact zero, whatever the size of
//     the fragmentation weights;
//   * partial pairs: u or v is a node remapped onto part of a bin (the end bins of
//     the inner range, the outer bin that contains a volume point): a list of
//     entries (functional, weight x S0, D0, bins and basis values of u and v),
//     evaluated per cell.
// Both are built once per setup on the device in FP64 by the same quadrature
// walk as the T build (grace_precompute.cu); each RHS then costs a bilinear
// contraction in node space plus one cheap kernel factor per partial entry.
//
// Reduced-precision forms (TF32 / BF16x3): the fixed part runs on the tensor cores
// (grace_tc.cu, node-space tiles: the MMA contracts over the smaller node, the
// epilogue applies the ramp of the larger node), the partial entries in FP32 on
// the CUDA cores, both on bin-mass-scaled values (Ghat = h_bin G) so that the
// operands stay inside the FP32 range.
#include <algorithm>
#include <cmath>
#include <vector>

#include "grace_convert.cuh"
#include "grace_physics.cuh"
#include "grace_tc_layout.cuh"

namespace grace {

namespace {

constexpr int kNcKMax = 3;          // per-cell-kernel groups: k <= 3 (entry layouts below)
constexpr int kB = kNcKMax + 1;

struct NcEntry {
    int r;              // functional
    int kind;           // 0 coagulation factor (1 - pf), 1 fragmentation factor pf
    double w;           // quadrature weight x S0(u, v) (all cell-independent factors)
    double D0;          // D0 of the larger particle
    int bu, bv;         // bins of u and v
    double pu[kB], pv[kB];   // phi_i at u and v
};
static_assert(sizeof(NcEntry) == 96, "NcEntry layout");

// FP32 entry of the reduced-precision forms.  A coagulation entry and the fragmentation entry of
// the same node pair are merged: the pair contributes (wc + wd pf) u v with wc the coagulation
// weight and wd = w_frag - w_coag, both divided by h_bu h_bv (to be used with the
// bin-mass-scaled coefficients h_bin g), and pf = clamp(s D0r + rb, 0, 1) with D0r = D0 / (2 w v_frag)
// the ramp-scaled D0 of the larger particle.  Flags mark where u or D0 differ from the previous
// entry of the same functional, so that runs sharing them reuse u and pf.
constexpr int kNcBinBits = 14;
constexpr int kNcBinMask = (1 << kNcBinBits) - 1;
constexpr int kNcBinsMask = (1 << (2 * kNcBinBits)) - 1;
constexpr int kNcNewU = 1 << 28;
constexpr int kNcNewPf = 1 << 29;
struct NcEntryF {
    int bins;              // bu | bv << 14 | flags
    float wc, wd, D0r;
    float pu[kB], pv[kB];
};
static_assert(sizeof(NcEntryF) == 48, "NcEntryF layout");

struct NcBuild {
    double *Bc, *Bf;            // [R][NQ][NQ] fixed-pair weights (dense)
    const long long *offset;    // [R][N][N] first entry of each (r, l, m) block (pass 1)
    long long *count;           // [R][N][N] entries of each block (pass 0)
    NcEntry *entries;           // pass 1
    int pass;
};

struct Acc {
    // fixed-pair accumulators of one (r, l, m) block and the partial-entry cursor
    double c[kQMax * kQMax], f[kQMax * kQMax];
    long long n;
};

__device__ __forceinline__ void emit(const DevGroup &G, const NcBuild &B, Acc &A, long long base, int r, int kind,
                                     double w, double u, double v, int l, int m)
{
    if (B.pass == 1) {
        double S0, D0;
        dev_ballistic_split(G.coag_p, u, v, &S0, &D0);
        NcEntry e;
        e.r = r;
        e.kind = kind;
        e.w = w * S0;
        e.D0 = D0;
        e.bu = l;
        e.bv = m;
        const double *ed = G.edges;
        dev_legendre(G.k, 2.0 / (ed[l + 1] - ed[l]) * (u - 0.5 * (ed[l] + ed[l + 1])), e.pu, nullptr);
        dev_legendre(G.k, 2.0 / (ed[m + 1] - ed[m]) * (v - 0.5 * (ed[m] + ed[m + 1])), e.pv, nullptr);
        for (int i = G.k + 1; i < kB; ++i) e.pu[i] = e.pv[i] = 0.0;
        B.entries[base + A.n] = e;
    }
    ++A.n;
}

// contribution c x (flux at x) of outer bin l and inner bin m, split into fixed
// pairs and partial entries (the walk of point_block in grace_precompute.cu)
__device__ void nc_point(const DevGroup &G, const NcBuild &B, Acc &A, long long base, int r, double x, int l, int m,
                         double c, bool frag)
{
    const double *e = G.edges;
    const int Q = G.Q;
    const bool do_frag = frag && G.frag_kind != GRACE_FRAG_NONE;
    // positive flux: u in [x_min, x] (outer bin l), v in [x - u + x_min, v_max(u)] within bin m
    if (e[l] < x) {
        const double a = e[l], b = fmin(e[l + 1], x);
        const bool ufix = b == e[l + 1];
        if (b > a)
            for (int al = 0; al < Q; ++al) {
                const double u = 0.5 * (a + b) + 0.5 * (b - a) * G.gs[al];
                const double Wu = 0.5 * (b - a) * G.gw[al];
                const double lo = x - u + G.x_min, hi = dev_vmax(G, u);
                if (!(hi > lo)) continue;
                const double va = fmax(lo, e[m]), vb = fmin(hi, e[m + 1]);
                if (!(vb > va)) continue;
                const bool vfix = va == e[m] && vb == e[m + 1];
                for (int be = 0; be < Q; ++be) {
                    const double v = 0.5 * (va + vb) + 0.5 * (vb - va) * G.gs[be];
                    const double Wv = 0.5 * (vb - va) * G.gw[be];
                    const double wc = c * Wu * Wv / v;
                    const double wf = do_frag ? c * Wu * Wv * dev_mass_above(G, x, u, v) / (v * (u + v)) : 0.0;
                    if (ufix && vfix) {
                        if (B.pass == 1) {
                            double S0, D0;
                            dev_ballistic_split(G.coag_p, u, v, &S0, &D0);
                            A.c[al * Q + be] += wc * S0;
                            A.f[al * Q + be] += wf * S0;
                        }
                    } else {
                        emit(G, B, A, base, r, 0, wc, u, v, l, m);
                        if (do_frag && wf != 0.0) emit(G, B, A, base, r, 1, wf, u, v, l, m);
                    }
                }
            }
    }
    // negative fragmentation flux: u in [x, x_max], v in [x_min, v_max(u)]
    if (do_frag && e[l + 1] > x) {
        const double a = fmax(e[l], x), b = e[l + 1];
        const bool ufix = a == e[l];
        if (b > a)
            for (int al = 0; al < Q; ++al) {
                const double u = 0.5 * (a + b) + 0.5 * (b - a) * G.gs[al];
                const double Wu = 0.5 * (b - a) * G.gw[al];
                const double hi = dev_vmax(G, u);
                const double va = fmax(G.x_min, e[m]), vb = fmin(hi, e[m + 1]);
                if (!(vb > va)) continue;
                const bool vfix = va == e[m] && vb == e[m + 1];
                for (int be = 0; be < Q; ++be) {
                    const double v = 0.5 * (va + vb) + 0.5 * (vb - va) * G.gs[be];
                    const double Wv = 0.5 * (vb - va) * G.gw[be];
                    const double wf = -c * Wu * Wv * dev_mass_below(G, x, u, v) / (v * (u + v));
                    if (wf == 0.0) continue;
                    if (ufix && vfix) {
                        if (B.pass == 1) {
                            double S0, D0;
                            dev_ballistic_split(G.coag_p, u, v, &S0, &D0);
                            A.f[al * Q + be] += wf * S0;
                        }
                    } else {
                        emit(G, B, A, base, r, 1, wf, u, v, l, m);
                    }
                }
            }
    }
}

// the App. B volume term of fragmentation with a Dirac remnant (appB_block)
__device__ double nc_sub_interval(const DevGroup &G, int j, int i, double a, double b, double c0, double c1,
                                  double alpha, bool pw)
{
    if (!(b > a)) return 0.0;
    const double *e = G.edges;
    const double h = e[j + 1] - e[j], xc = 0.5 * (e[j] + e[j + 1]);
    double P[kB], dP[kB], s = 0.0;
    for (int t = 0; t < G.Q; ++t) {
        const double x = 0.5 * (a + b) + 0.5 * (b - a) * G.gs[t];
        const double W = 0.5 * (b - a) * G.gw[t];
        const double f = pw ? c0 + c1 * pow(x, 2.0 + alpha) : c0;
        dev_legendre(G.k, 2.0 / h * (x - xc), P, dP);
        s += W * f * (2.0 / h) * dP[i];
    }
    return s;
}

__device__ double nc_appB_J(const DevGroup &G, int j, int i, double u, double v)
{
    const double ja = G.edges[j], jb = G.edges[j + 1], xmin = G.x_min;
    const FragOutcome o = dev_outcome(G, u, v);
    const double top = u + v - xmin;
    double J = 0.0;
    if (o.mcut > xmin) {
        const double a2 = 2.0 + o.alpha;
        const double mc2 = pow(o.mcut, a2), xm2 = pow(xmin, a2);
        const double cA = o.mfrag / (mc2 - xm2);
        J += nc_sub_interval(G, j, i, fmax(ja, u), fmin(jb, fmin(top, o.mcut)), cA * mc2, -cA, o.alpha, true);
        J -= nc_sub_interval(G, j, i, fmax(ja, xmin), fmin(jb, u), -cA * xm2, cA, o.alpha, true);
        J += nc_sub_interval(G, j, i, fmax(ja, o.mcut), fmin(jb, u), -cA * mc2, cA, o.alpha, true);
    } else {
        J -= nc_sub_interval(G, j, i, fmax(ja, xmin), fmin(jb, u), o.mfrag, 0.0, 0.0, false);
    }
    if (o.mleft > 0.0) {
        J += nc_sub_interval(G, j, i, fmax(ja, u), fmin(jb, fmin(top, o.mleft)), o.mleft, 0.0, 0.0, false);
        if (o.mleft >= xmin) J -= nc_sub_interval(G, j, i, fmax(ja, o.mleft), fmin(jb, u), o.mleft, 0.0, 0.0, false);
    }
    return J;
}

__device__ void nc_appB(const DevGroup &G, const NcBuild &B, Acc &A, long long base, int r, int j, int i, int l,
                        int m)
{
    const double *e = G.edges;
    const int Q = G.Q;
    const double hl = e[l + 1] - e[l], xl = 0.5 * (e[l] + e[l + 1]);
    for (int al = 0; al < Q; ++al) {
        const double u = xl + 0.5 * hl * G.gs[al];
        const double Wu = 0.5 * hl * G.gw[al];
        const double hi = dev_vmax(G, u);
        const double va = fmax(G.x_min, e[m]), vb = fmin(hi, e[m + 1]);
        if (!(vb > va)) continue;
        const bool vfix = va == e[m] && vb == e[m + 1];
        for (int be = 0; be < Q; ++be) {
            const double v = 0.5 * (va + vb) + 0.5 * (vb - va) * G.gs[be];
            const double Wv = 0.5 * (vb - va) * G.gw[be];
            const double w = Wu * Wv / (v * (u + v)) * nc_appB_J(G, j, i, u, v);
            if (w == 0.0) continue;
            if (vfix) {
                if (B.pass == 1) {
                    double S0, D0;
                    dev_ballistic_split(G.coag_p, u, v, &S0, &D0);
                    A.f[al * Q + be] += w * S0;
                }
            } else {
                emit(G, B, A, base, r, 1, w, u, v, l, m);
            }
        }
    }
}

// one thread per (r, l, m) block, as in the T build: pass 0 counts partial
// entries, pass 1 writes them and the block's fixed-pair weights
__global__ void __launch_bounds__(128) nc_build_kernel(DevGroup G, NcBuild B)
{
    const int r = blockIdx.y;
    const int lm = blockIdx.x * blockDim.x + threadIdx.x;
    if (lm >= G.N * G.N || r >= G.R) return;
    const int l = lm / G.N, m = lm % G.N, Q = G.Q, NQ = G.N * G.Q;
    const size_t blk = ((size_t)r * G.N + l) * G.N + m;
    const long long base = B.pass == 1 ? B.offset[blk] : 0;
    Acc A;
    for (int t = 0; t < Q * Q; ++t) A.c[t] = A.f[t] = 0.0;
    A.n = 0;
    if (r < G.n_if) {
        nc_point(G, B, A, base, r, G.edges[r + 1], l, m, 1.0, true);
    } else {
        const int q = r - G.n_if, j = q / G.k, i = q % G.k + 1;
        const double h = G.edges[j + 1] - G.edges[j], xc = 0.5 * (G.edges[j] + G.edges[j + 1]);
        double P_[kB], dP[kB];
        for (int th = 0; th < G.Q; ++th) {
            dev_legendre(G.k, G.gs[th], P_, dP);
            nc_point(G, B, A, base, r, xc + 0.5 * h * G.gs[th], l, m, G.gw[th] * dP[i], !G.has_delta);
        }
        if (G.has_delta) nc_appB(G, B, A, base, r, j, i, l, m);
    }
    if (B.pass == 0) {
        B.count[blk] = A.n;
    } else {
        for (int al = 0; al < Q; ++al)
            for (int be = 0; be < Q; ++be) {
                const size_t o = ((size_t)r * NQ + l * Q + al) * NQ + m * Q + be;
                B.Bc[o] = A.c[al * Q + be];
                B.Bf[o] = A.f[al * Q + be];
            }
    }
}

// B <- fold(B) in place for both tables, one thread per (r, i, j > i)
__global__ void nc_fold_kernel(int R, int NQ, double *Bc, double *Bf)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)R * NQ * NQ) return;
    const int r = (int)(t / ((long long)NQ * NQ));
    const int rem = (int)(t - (long long)r * NQ * NQ), i = rem / NQ, j = rem % NQ;
    if (j <= i) return;
    double *c = Bc + (size_t)r * NQ * NQ, *f = Bf + (size_t)r * NQ * NQ;
    const size_t ij = (size_t)i * NQ + j, ji = (size_t)j * NQ + i;
    c[ij] += c[ji];
    c[ji] = 0.0;
    f[ij] += f[ji];
    f[ji] = 0.0;
}

// first / one-past-last column with a non-zero in either table, per row (r, i), and the rows' range per r
__global__ void nc_extent_kernel(int R, int NQ, const double *Qt, const double *Dt, int *qlo, int *qhi)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= R * NQ) return;
    const double *a = Qt + (size_t)row * NQ, *b = Dt + (size_t)row * NQ;
    int lo = NQ, hi = 0;
    for (int j = 0; j < NQ; ++j)
        if (a[j] != 0.0 || b[j] != 0.0) {
            if (lo == NQ) lo = j;
            hi = j + 1;
        }
    qlo[row] = lo;
    qhi[row] = hi;
}

// nodal values G = g at the fixed nodes, Hc = (1 - pf(s D0)) G and Hf = pf(s D0) G, per cell
struct NodeRule {
    double phi[kQMax * kB];   // phi_i at the Gauss node alpha: phi[alpha * kB + i]
};

__global__ void nc_nodal_kernel(DevGroup G, NodeRule rule, const double *__restrict__ D0, const double *__restrict__ g,
                                const double *__restrict__ alpha, int n_cells, double *__restrict__ Gv,
                                double *__restrict__ Hc, double *__restrict__ Hf)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int NQ = G.N * G.Q;
    if (t >= (long long)n_cells * NQ) return;
    const long long cell = t / NQ;
    const int a = (int)(t - cell * NQ), l = a / G.Q, al = a - l * G.Q;
    const double *gb = g + (size_t)cell * G.P + (size_t)l * G.K1;
    double v = 0.0;
    for (int i = 0; i <= G.k; ++i) v += gb[i] * rule.phi[al * kB + i];
    const double s = sqrt(alpha[cell]);
    const double pf = dev_pfrag(G.coag_p, s * D0[a]);
    Gv[t] = v;
    Hc[t] = (1.0 - pf) * v;
    Hf[t] = pf * v;
}

// fixed part: F[c][r] = s_c sum_i G_i sum_{j >= i} (Cc_r[i][j] Hc_j + Cf_r[i][j] Hf_j); one warp per 32
// cells and a chunk of kRChunk functionals (blockIdx.y), so that small batches still fill the GPU
constexpr int kRChunk = 8;
__global__ void __launch_bounds__(128) nc_fixed_kernel(const double *__restrict__ Cc, const double *__restrict__ Cf,
                                                       const int *__restrict__ qlo, const int *__restrict__ qhi,
                                                       int R, int NQ, const double *__restrict__ Gv,
                                                       const double *__restrict__ Hcv, const double *__restrict__ Hfv,
                                                       const double *__restrict__ alpha, int n_cells,
                                                       double *__restrict__ F)
{
    extern __shared__ double nsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const long long cell0 = ((long long)blockIdx.x * nwarps + warp) * 32;
    double *gw = nsm + (size_t)warp * NQ * 96;   // G, Hc, Hf, transposed [node][cell]
    double *hc = gw + (size_t)NQ * 32, *hf = hc + (size_t)NQ * 32;
    for (int idx = lane; idx < 32 * NQ; idx += 32) {
        const int c = idx / NQ, q = idx - c * NQ;
        const long long cell = cell0 + c;
        const bool ok = cell < n_cells;
        gw[q * 32 + c] = ok ? Gv[cell * NQ + q] : 0.0;
        hc[q * 32 + c] = ok ? Hcv[cell * NQ + q] : 0.0;
        hf[q * 32 + c] = ok ? Hfv[cell * NQ + q] : 0.0;
    }
    __syncwarp();
    const long long cell = cell0 + lane;
    const double s = cell < n_cells ? sqrt(alpha[cell]) : 0.0;
    const int r_end = min(R, (int)(blockIdx.y + 1) * kRChunk);
    for (int r = blockIdx.y * kRChunk; r < r_end; ++r) {
        double Fr = 0.0;
        for (int i = 0; i < NQ; ++i) {
            const int j0 = qlo[r * NQ + i], j1 = qhi[r * NQ + i];
            if (j0 >= j1) continue;
            const double *cr = Cc + ((size_t)r * NQ + i) * NQ, *fr = Cf + ((size_t)r * NQ + i) * NQ;
            double y = 0.0;
            for (int j = j0; j < j1; ++j) y = fma(__ldg(cr + j), hc[j * 32 + lane], fma(__ldg(fr + j), hf[j * 32 + lane], y));
            Fr = fma(gw[i * 32 + lane], y, Fr);
        }
        if (cell < n_cells) F[cell * R + r] = s * Fr;
    }
}

// partial entries of functional r (blockIdx.y) for 128 cells (one per thread); the
// entries are staged through shared memory and shared by the block's cells
__global__ void __launch_bounds__(128) nc_partial_kernel(DevGroup G, const NcEntry *__restrict__ entries,
                                                         const long long *__restrict__ seg,
                                                         const double *__restrict__ g,
                                                         const double *__restrict__ alpha, int n_cells,
                                                         double *__restrict__ F)
{
    __shared__ NcEntry es[64];
    const int r = blockIdx.y;
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = cell < n_cells;
    const double s = live ? sqrt(alpha[cell]) : 0.0;
    const double *gc = g + (size_t)(live ? cell : 0) * G.P;
    const long long e0 = seg[r], e1 = seg[r + 1];
    double acc = 0.0;
    for (long long c0 = e0; c0 < e1; c0 += 64) {
        const int n = (int)min((long long)64, e1 - c0);
        __syncthreads();
        for (int w = threadIdx.x; w < n * (int)(sizeof(NcEntry) / 8); w += blockDim.x)
            reinterpret_cast<double *>(es)[w] = reinterpret_cast<const double *>(entries + c0)[w];
        __syncthreads();
        if (live)
            for (int t = 0; t < n; ++t) {
                const NcEntry &e = es[t];
                const double *gu = gc + (size_t)e.bu * G.K1, *gv = gc + (size_t)e.bv * G.K1;
                double u = 0.0, v = 0.0;
                for (int i = 0; i <= G.k; ++i) {
                    u = fma(gu[i], e.pu[i], u);
                    v = fma(gv[i], e.pv[i], v);
                }
                const double pf = dev_pfrag(G.coag_p, s * e.D0);
                acc = fma(e.w * (e.kind ? pf : 1.0 - pf), u * v, acc);
            }
    }
    if (live) F[cell * G.R + r] += s * acc;
}

// ---------------------------------------------------------------- adjoint (FP64)
// The fixed part of functional r is s G^T M_r G with M_r[i][j] = Cc_r[i][j] (1 - pf_j) + Cf_r[i][j] pf_j
// (j >= i), G = B g the nodal values; partial entries add s w (pf or 1 - pf) (u . g) (v . g).  So
//     w = sum_r mu_r dF_r/dg = B^T gamma + (partial entries),
//     gamma_a = s sum_r mu_r [ sum_j M_r[a][j] G_j + sum_i G_i M_r[i][a] ]
//             = s sum_r mu_r [ sum_j (Cc_r[a][j] Hc_j + Cf_r[a][j] Hf_j) + (1 - pf_a) (Cc_r^T G)_a + pf_a (Cf_r^T G)_a ].

// transposed copies of both tables, one thread per (r, i, j)
__global__ void nc_transpose_kernel(int R, int NQ, const double *__restrict__ C, double *__restrict__ CT)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = (long long)NQ * NQ;
    if (t >= (long long)R * per) return;
    const long long r = t / per;
    const int i = (int)((t - r * per) / NQ), j = (int)(t - r * per - (long long)i * NQ);
    CT[r * per + (long long)j * NQ + i] = C[t];
}

// gamma[c][a] for 32 cells per warp: G, Hc, Hf and mu of the warp's cells in shared memory; for
// every node a, the sum over the functionals of its row of (Cc, Cf) against (Hc, Hf) and of its
// row of the transposed tables against G
__global__ void __launch_bounds__(32) nc_vjp_node_kernel(
    DevGroup G, const double *__restrict__ Cc, const double *__restrict__ Cf, const int *__restrict__ qlo,
    const int *__restrict__ qhi, const double *__restrict__ CcT, const double *__restrict__ CfT,
    const int *__restrict__ qloT, const int *__restrict__ qhiT, const double *__restrict__ D0, int R, int NQ,
    const double *__restrict__ Gv, const double *__restrict__ Hcv, const double *__restrict__ Hfv,
    const double *__restrict__ mu, const double *__restrict__ alpha, int n_cells, double *__restrict__ gamma)
{
    extern __shared__ double vsm[];
    const int lane = threadIdx.x & 31;
    const long long cell0 = (long long)blockIdx.x * 32;
    double *gw = vsm, *hc = gw + (size_t)NQ * 32, *hf = hc + (size_t)NQ * 32, *mw = hf + (size_t)NQ * 32;
    for (int idx = lane; idx < 32 * NQ; idx += 32) {
        const int c = idx / NQ, q = idx - c * NQ;
        const long long cell = cell0 + c;
        const bool ok = cell < n_cells;
        gw[q * 32 + c] = ok ? Gv[cell * NQ + q] : 0.0;
        hc[q * 32 + c] = ok ? Hcv[cell * NQ + q] : 0.0;
        hf[q * 32 + c] = ok ? Hfv[cell * NQ + q] : 0.0;
    }
    for (int idx = lane; idx < 32 * R; idx += 32) {
        const int c = idx / R, r = idx - c * R;
        const long long cell = cell0 + c;
        mw[r * 32 + c] = cell < n_cells ? mu[cell * R + r] : 0.0;
    }
    __syncwarp();
    const long long cell = cell0 + lane;
    const double s = cell < n_cells ? sqrt(alpha[cell]) : 0.0;
    for (int a = 0; a < NQ; ++a) {
        const double pf = dev_pfrag(G.coag_p, s * D0[a]);
        double acc = 0.0;
        for (int r = 0; r < R; ++r) {
            const double m = mw[r * 32 + lane];
            const size_t row = (size_t)r * NQ + a;
            double y = 0.0;
            for (int j = qlo[row]; j < qhi[row]; ++j)
                y = fma(__ldg(Cc + row * NQ + j), hc[j * 32 + lane], fma(__ldg(Cf + row * NQ + j), hf[j * 32 + lane], y));
            double zc = 0.0, zf = 0.0;
            for (int i = qloT[row]; i < qhiT[row]; ++i) {
                zc = fma(__ldg(CcT + row * NQ + i), gw[i * 32 + lane], zc);
                zf = fma(__ldg(CfT + row * NQ + i), gw[i * 32 + lane], zf);
            }
            acc = fma(m, y + (1.0 - pf) * zc + pf * zf, acc);
        }
        if (cell < n_cells) gamma[cell * NQ + a] = s * acc;
    }
}

// w[c][l K1 + i] = sum_alpha phi_i(s_alpha) gamma[c][l Q + alpha] (the transpose of the nodal values)
__global__ void nc_vjp_assemble_kernel(DevGroup G, NodeRule rule, const double *__restrict__ gamma, int NQ,
                                       int n_cells, double *__restrict__ w)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_cells * G.P) return;
    const long long cell = t / G.P;
    const int p = (int)(t - cell * G.P), l = p / G.K1, i = p - l * G.K1;
    double acc = 0.0;
    for (int al = 0; al < G.Q; ++al) acc = fma(rule.phi[al * kB + i], gamma[cell * NQ + (long long)l * G.Q + al], acc);
    w[t] = acc;
}

// the partial entries' part of w: one thread per cell walks every functional's entries (staged in
// shared memory for the block's 128 cells) and adds s mu_r w (pf or 1 - pf) [pu (v . g) at bin bu,
// pv (u . g) at bin bv] into its own row of w
__global__ void __launch_bounds__(128) nc_vjp_partial_kernel(DevGroup G, const NcEntry *__restrict__ entries,
                                                             const long long *__restrict__ seg,
                                                             const double *__restrict__ g,
                                                             const double *__restrict__ mu,
                                                             const double *__restrict__ alpha, int n_cells,
                                                             double *__restrict__ w)
{
    __shared__ NcEntry es[64];
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = cell < n_cells;
    const double s = live ? sqrt(alpha[cell]) : 0.0;
    const double *gc = g + (size_t)(live ? cell : 0) * G.P;
    double *wc = w + (size_t)(live ? cell : 0) * G.P;
    for (int r = 0; r < G.R; ++r) {
        const double m = live ? s * mu[cell * G.R + r] : 0.0;
        const long long e0 = seg[r], e1 = seg[r + 1];
        for (long long c0 = e0; c0 < e1; c0 += 64) {
            const int n = (int)min((long long)64, e1 - c0);
            __syncthreads();
            for (int x = threadIdx.x; x < n * (int)(sizeof(NcEntry) / 8); x += blockDim.x)
                reinterpret_cast<double *>(es)[x] = reinterpret_cast<const double *>(entries + c0)[x];
            __syncthreads();
            if (!live || m == 0.0) continue;
            for (int t = 0; t < n; ++t) {
                const NcEntry &e = es[t];
                const double *gu = gc + (size_t)e.bu * G.K1, *gv = gc + (size_t)e.bv * G.K1;
                double u = 0.0, v = 0.0;
                for (int i = 0; i <= G.k; ++i) {
                    u = fma(gu[i], e.pu[i], u);
                    v = fma(gv[i], e.pv[i], v);
                }
                const double pf = dev_pfrag(G.coag_p, s * e.D0);
                const double c = m * e.w * (e.kind ? pf : 1.0 - pf);
                double *wu = wc + (size_t)e.bu * G.K1, *wv = wc + (size_t)e.bv * G.K1;
                for (int i = 0; i <= G.k; ++i) {
                    wu[i] = fma(c * v, e.pu[i], wu[i]);
                    wv[i] = fma(c * u, e.pv[i], wv[i]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- reduced-precision forms
// Per cell tile and bin (block = (tile, bin), thread = row): the scaled coefficients
// h_l g_{l,i} in FP32 into gh ([tile][P][128]), the node values Ghat_a = sum_i h_l g_{l,i} phi_i(s_alpha)
// (node a = l Q + alpha) into the A operand, and s = sqrt(alpha_turb) per cell.
struct NodeRuleF {
    float phi[kQMax * kB];
};

__global__ void __launch_bounds__(128) nc_pack_tc_kernel(DevGroup G, NodeRuleF rule, const double *__restrict__ g,
                                                         const double *__restrict__ alpha, int n_cells, void *opA,
                                                         int prec, int kpad, float *__restrict__ gh,
                                                         float *__restrict__ cell_s)
{
    const int l = blockIdx.x % G.N;
    const long long ct = blockIdx.x / G.N;
    const int row = threadIdx.x;
    const long long cell = ct * kTileM + row;
    if (cell >= n_cells) return;
    const double h = G.hbin[l];
    const double *gb = g + (size_t)cell * G.P + (size_t)l * G.K1;
    float c[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
        c[i] = i <= G.k ? d2f_fast(h * gb[i]) : 0.f;
        if (i <= G.k) gh[((size_t)ct * G.P + (size_t)l * G.K1 + i) * kTileM + row] = c[i];
    }
    char *t = (char *)opA + (size_t)ct * opA_tile_bytes(prec, kpad);
    for (int al = 0; al < G.Q; ++al) {
        float v = 0.f;
#pragma unroll
        for (int i = 0; i < kB; ++i) v = fmaf(c[i], rule.phi[al * kB + i], v);
        const int col = l * G.Q + al;
        if (prec == GRACE_TF32) {
            *(uint32_t *)(t + swz_offset(kTileM, row, col, 4)) = f32_to_tf32_rna(v);
        } else {
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            const size_t plane = (size_t)kTileM * kpad * 2;
            *(__nv_bfloat16 *)(t + swz_offset(kTileM, row, col, 2)) = hi;
            *(__nv_bfloat16 *)(t + plane + swz_offset(kTileM, row, col, 2)) = lo;
        }
    }
    if (l == 0) cell_s[cell] = sqrtf(d2f_fast(alpha[cell]));
}

// Partial entries of functional r (blockIdx.x) in FP32, added to the contraction's output
// ([tile][functional][row]); functionals the contraction does not write are overwritten.  A block
// covers C cell tiles: thread t handles row t of each (C cells), so every entry, staged through
// shared memory, is read once per C cells (the broadcast loads, not the arithmetic, bound a
// thread-per-cell loop).  Entries come sorted by (bin of u, bin of v); a thread reloads its cells'
// two bins of coefficients only when that pair changes (coalesced: gh is cell-minor).  Within a
// run of entries with the same u the terms are summed as u * sum (wc + wd pf) v, and pf is
// recomputed only where D0 changes.
template <int K1, int C>
__global__ void __launch_bounds__(128) nc_partial_f32_kernel(int P, int R, const NcEntryF *__restrict__ entries,
                                                             const long long *__restrict__ seg,
                                                             const float *__restrict__ gh,
                                                             const float *__restrict__ cell_s,
                                                             const int *__restrict__ written, float rb,
                                                             int n_cells, float *__restrict__ F32)
{
    constexpr int kChunk = 128;
    __shared__ float4 es[kChunk * 3];
    // functional fastest in the grid: the blocks of one group of C cell tiles run together, so
    // its coefficients stay in L2 across the functionals
    const int r = blockIdx.x, row = threadIdx.x;
    const long long ct0 = (long long)blockIdx.y * C;
    const long long last_tile = (long long)(n_cells - 1) / kTileM;
    float s[C], acc[C], ru[C], u[C], pf[C], gu[C][K1], gv[C][K1];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const long long cell = (ct0 + j) * kTileM + row;
        s[j] = cell < n_cells ? cell_s[cell] : 0.f;   // 0 for rows past the batch: they add nothing
        acc[j] = ru[j] = u[j] = pf[j] = 0.f;
#pragma unroll
        for (int i = 0; i < K1; ++i) gu[j][i] = gv[j][i] = 0.f;
    }
    const long long e0 = seg[r], e1 = seg[r + 1];
    int cur = -1;
    for (long long c0 = e0; c0 < e1; c0 += kChunk) {
        const int n = (int)min((long long)kChunk, e1 - c0);
        __syncthreads();
        const float4 *src = reinterpret_cast<const float4 *>(entries + c0);
        for (int w = threadIdx.x; w < n * 3; w += blockDim.x) es[w] = src[w];
        __syncthreads();
        for (int t = 0; t < n; ++t) {
            const float4 a = es[3 * t], pv = es[3 * t + 2];
            const int bf = __float_as_int(a.x), bins = bf & kNcBinsMask;
            if (bins != cur) {
                cur = bins;
                const size_t ou = (size_t)(bins & kNcBinMask) * K1 * kTileM;
                const size_t ov = (size_t)(bins >> kNcBinBits) * K1 * kTileM;
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const float *gc = gh + (size_t)min(ct0 + j, last_tile) * P * kTileM + row;
#pragma unroll
                    for (int i = 0; i < K1; ++i) {
                        gu[j][i] = gc[ou + i * kTileM];
                        gv[j][i] = gc[ov + i * kTileM];
                    }
                }
            }
            if (bf & kNcNewU) {
                const float4 pu = es[3 * t + 1];
                const float pa[4] = {pu.x, pu.y, pu.z, pu.w};
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    acc[j] = fmaf(u[j], ru[j], acc[j]);
                    ru[j] = 0.f;
                    float x = gu[j][0] * pa[0];
#pragma unroll
                    for (int i = 1; i < K1; ++i) x = fmaf(gu[j][i], pa[i], x);
                    u[j] = x;
                }
            }
            if (bf & kNcNewPf) {
#pragma unroll
                for (int j = 0; j < C; ++j) pf[j] = __saturatef(fmaf(s[j], a.w, rb));
            }
            const float pb[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int j = 0; j < C; ++j) {
                float v = gv[j][0] * pb[0];
#pragma unroll
                for (int i = 1; i < K1; ++i) v = fmaf(gv[j][i], pb[i], v);
                ru[j] = fmaf(fmaf(a.z, pf[j], a.y), v, ru[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const long long ct = ct0 + j, cell = ct * kTileM + row;
        if (cell < n_cells) {
            float *Fo = F32 + ((size_t)ct * R + r) * kTileM + row;
            *Fo = (written[r] ? *Fo : 0.f) + s[j] * fmaf(u[j], ru[j], acc[j]);
        }
    }
}

}  // namespace

grace_status build_nc_tc_entries(Group &Gr, cudaStream_t st)
{
    NcTables &T = Gr.nc;
    if (T.d_entf) return GRACE_OK;
    const int R = Gr.dg.R;
    std::vector<NcEntry> in((size_t)T.n_entries);
    std::vector<long long> seg(R + 1);
    cudaError_t e = cudaSuccess;
    if (T.n_entries > 0)
        e = cudaMemcpyAsync(in.data(), T.d_entries, in.size() * sizeof(NcEntry), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(seg.data(), T.d_seg, (R + 1) * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "node-space FP32 entries: copy");
    std::vector<double> h(Gr.dg.N);
    for (int j = 0; j < Gr.dg.N; ++j) h[j] = Gr.h_edges[j + 1] - Gr.h_edges[j];
    std::vector<NcEntryF> out;
    out.reserve(in.size());
    std::vector<long long> segf(R + 1, 0);
    auto same_pair = [](const NcEntry &a, const NcEntry &b) {
        if (a.r != b.r || a.bu != b.bu || a.bv != b.bv || a.D0 != b.D0) return false;
        for (int i = 0; i < kB; ++i)
            if (a.pu[i] != b.pu[i] || a.pv[i] != b.pv[i]) return false;
        return true;
    };
    // ramp scale of D0: pf = clamp(s D0 / (2 w v_frag) - (1 - w) / (2 w), 0, 1)
    const double ra = 1.0 / (2.0 * Gr.dg.coag_p[5] * Gr.dg.coag_p[4]);
    bool bad = false;
    for (int r = 0; r < R; ++r) {
        const size_t first = out.size();
        for (long long t = seg[r]; t < seg[r + 1]; ++t) {
            const NcEntry &a = in[t];
            double wc = a.kind == 0 ? a.w : 0.0, wf = a.kind == 1 ? a.w : 0.0;
            if (a.kind == 0 && t + 1 < seg[r + 1] && in[t + 1].kind == 1 && same_pair(a, in[t + 1])) {
                wf = in[t + 1].w;
                ++t;
            }
            const double sc = 1.0 / (h[a.bu] * h[a.bv]);
            wc *= sc;
            wf *= sc;
            // the scaled weights must be normal FP32 numbers with room for the products (their
            // difference wd may round to zero where the two nearly agree)
            for (double w : {wc, wf})
                if (w != 0.0 && (std::fabs(w) < 1e-30 || std::fabs(w) > 1e30)) bad = true;
            NcEntryF f;
            f.bins = a.bu | (a.bv << kNcBinBits);
            f.wc = (float)wc;
            f.wd = (float)(wf - wc);
            f.D0r = (float)(ra * a.D0);
            for (int i = 0; i < kB; ++i) {
                f.pu[i] = (float)a.pu[i];
                f.pv[i] = (float)a.pv[i];
            }
            if (out.size() == first) {
                f.bins |= kNcNewU | kNcNewPf;
            } else {
                const NcEntryF &p = out.back();
                bool same_u = (p.bins & kNcBinMask) == (f.bins & kNcBinMask);
                for (int i = 0; i < kB; ++i) same_u = same_u && p.pu[i] == f.pu[i];
                if (!same_u) f.bins |= kNcNewU;
                if (p.D0r != f.D0r) f.bins |= kNcNewPf;
            }
            out.push_back(f);
        }
        segf[r + 1] = (long long)out.size();
    }
    if (bad) {
        set_error("node-space partial weights outside the FP32 range");
        return GRACE_ERR_UNSUPPORTED;
    }
    if (Gr.dg.N > kNcBinMask) {
        set_error("node-space FP32 entries: too many bins");
        return GRACE_ERR_UNSUPPORTED;
    }
    e = cudaMalloc(&T.d_entf, std::max<size_t>(out.size(), 1) * sizeof(NcEntryF));
    if (e == cudaSuccess) e = cudaMalloc(&T.d_segf, (R + 1) * sizeof(long long));
    if (e == cudaSuccess && !out.empty())
        e = cudaMemcpy(T.d_entf, out.data(), out.size() * sizeof(NcEntryF), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(T.d_segf, segf.data(), (R + 1) * sizeof(long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(T.d_entf);
        cudaFree(T.d_segf);
        T.d_entf = nullptr;
        T.d_segf = nullptr;
        return cuda_fail(e, "node-space FP32 entries: upload");
    }
    T.n_entf = (long long)out.size();
    return GRACE_OK;
}

cudaError_t launch_nc_pack_tc(const DevGroup &g, const TcTiles &t, int prec, const double *d_g, const double *d_alpha,
                              int n_cells, void *opA, float *d_gh, float *d_s, cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    if (!t.built || !t.nc) return cudaErrorInvalidValue;
    NodeRuleF rule;
    for (int al = 0; al < g.Q; ++al) {
        double P[kB];
        // Legendre values at the Gauss node s_alpha (host recurrence, eq. 2.4)
        P[0] = 1.0;
        if (g.k >= 1) P[1] = g.gs[al];
        for (int n = 1; n < g.k; ++n) P[n + 1] = ((2.0 * n + 1.0) * g.gs[al] * P[n] - n * P[n - 1]) / (n + 1.0);
        for (int i = 0; i < kB; ++i) rule.phi[al * kB + i] = i <= g.k ? (float)P[i] : 0.f;
    }
    const long long tiles = (n_cells + kTileM - 1) / kTileM;
    nc_pack_tc_kernel<<<(unsigned)(tiles * g.N), kTileM, 0, st>>>(g, rule, d_g, d_alpha, n_cells, opA, prec, t.k_pad,
                                                                   d_gh, d_s);
    return cudaGetLastError();
}

cudaError_t launch_nc_partial_tc(const DevGroup &g, const NcTables &nt, const TcTiles &t, int n_cells,
                                 const float *d_gh, const float *d_s, float *d_F32, cudaStream_t st)
{
    if (n_cells <= 0 || nt.n_entf == 0) return cudaSuccess;
    if (!nt.built || !nt.d_entf || !t.built || !t.nc) return cudaErrorInvalidValue;
    const long long tiles = (n_cells + kTileM - 1) / kTileM;
    const NcEntryF *ent = (const NcEntryF *)nt.d_entf;
    // cells per thread: 8 once the grid still covers every SM a few times, else fewer
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int C = tiles * g.R >= 8LL * 4 * n_sm ? 8 : tiles * g.R >= 4LL * 4 * n_sm ? 4 : 1;
    const dim3 grid(g.R, (unsigned)((tiles + C - 1) / C));
#define GRACE_NC_PARTIAL(K, CC)                                                                                   \
    nc_partial_f32_kernel<K, CC><<<grid, kTileM, 0, st>>>(g.P, g.R, ent, nt.d_segf, d_gh, d_s, t.d_written, t.ramp_b, \
                                                        n_cells, d_F32)
#define GRACE_NC_PARTIAL_C(K)                \
    if (C == 8) GRACE_NC_PARTIAL(K, 8);       \
    else if (C == 4) GRACE_NC_PARTIAL(K, 4);  \
    else GRACE_NC_PARTIAL(K, 1)
    switch (g.K1) {
    case 1: GRACE_NC_PARTIAL_C(1); break;
    case 2: GRACE_NC_PARTIAL_C(2); break;
    case 3: GRACE_NC_PARTIAL_C(3); break;
    case 4: GRACE_NC_PARTIAL_C(4); break;
    default: return cudaErrorInvalidValue;
    }
#undef GRACE_NC_PARTIAL_C
#undef GRACE_NC_PARTIAL
    return cudaGetLastError();
}

void free_nc_tables(NcTables &t)
{
    cudaFree(t.d_Cc);
    cudaFree(t.d_Cf);
    cudaFree(t.d_qlo);
    cudaFree(t.d_qhi);
    cudaFree(t.d_D0);
    cudaFree(t.d_entries);
    cudaFree(t.d_entf);
    cudaFree(t.d_segf);
    cudaFree(t.d_seg);
    cudaFree(t.d_CcT);
    cudaFree(t.d_CfT);
    cudaFree(t.d_qloT);
    cudaFree(t.d_qhiT);
    t = NcTables();
}

grace_status build_nc_tables(Group &Gr, cudaStream_t st)
{
    const DevGroup &g = Gr.dg;
    NcTables &T = Gr.nc;
    free_nc_tables(T);
    const int N = g.N, Q = g.Q, R = g.R, NQ = N * Q;
    T.NQ = NQ;
    const size_t ntab = (size_t)R * NQ * NQ, nblk = (size_t)R * N * N;
    long long *d_count = nullptr, *d_off = nullptr;
    cudaError_t e = cudaMalloc(&T.d_Cc, ntab * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&T.d_Cf, ntab * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&d_count, nblk * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&d_off, nblk * sizeof(long long));
    if (e != cudaSuccess) {
        cudaFree(d_count);
        cudaFree(d_off);
        free_nc_tables(T);
        cudaGetLastError();
        set_error(std::string("node-space tables: allocation: ") + cudaGetErrorString(e));
        return GRACE_ERR_NOMEM;
    }
    NcBuild B;
    B.Bc = T.d_Cc;   // folded in place afterwards
    B.Bf = T.d_Cf;
    B.count = d_count;
    B.offset = d_off;
    B.entries = nullptr;
    B.pass = 0;
    const dim3 grid((N * N + 127) / 128, R);
    nc_build_kernel<<<grid, 128, 0, st>>>(g, B);
    e = cudaGetLastError();
    std::vector<long long> cnt(nblk), off(nblk);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_count, nblk * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // entries ordered by (r, l, m): each functional's entries are contiguous
    std::vector<long long> seg(R + 1, 0);
    long long total = 0;
    for (size_t b = 0; b < nblk; ++b) {
        off[b] = total;
        total += cnt[b];
        seg[b / ((size_t)N * N) + 1] = total;
    }
    T.n_entries = total;
    if (e == cudaSuccess) e = cudaMalloc(&T.d_entries, (size_t)std::max<long long>(total, 1) * sizeof(NcEntry));
    if (e == cudaSuccess) e = cudaMalloc(&T.d_seg, (R + 1) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), nblk * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T.d_seg, seg.data(), (R + 1) * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        B.entries = (NcEntry *)T.d_entries;
        B.pass = 1;
        nc_build_kernel<<<grid, 128, 0, st>>>(g, B);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        nc_fold_kernel<<<(unsigned)((ntab + 255) / 256), 256, 0, st>>>(R, NQ, T.d_Cc, T.d_Cf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMalloc(&T.d_qlo, sizeof(int) * R * NQ);
    if (e == cudaSuccess) e = cudaMalloc(&T.d_qhi, sizeof(int) * R * NQ);
    if (e == cudaSuccess) {
        nc_extent_kernel<<<(R * NQ + 127) / 128, 128, 0, st>>>(R, NQ, T.d_Cc, T.d_Cf, T.d_qlo, T.d_qhi);
        e = cudaGetLastError();
    }
    // D0 of every fixed node (the larger particle of a fixed pair is one of them)
    std::vector<double> D0(NQ), gsv(Q);
    for (int a = 0; a < NQ; ++a) {
        const int l = a / Q, al = a % Q;
        const double lo = Gr.h_edges[l], hi = Gr.h_edges[l + 1];
        const double u = 0.5 * (lo + hi) + 0.5 * (hi - lo) * g.gs[al];
        const double pi = 3.141592653589793, rho = g.coag_p[0], sig = g.coag_p[1], cs = g.coag_p[2];
        const double au = std::cbrt(3.0 * u / (4.0 * pi * rho));
        const double stn = pi * rho * au / (2.0 * sig);
        D0[a] = cs * std::sqrt(3.0 * stn / (1.0 + stn * stn));
    }
    if (e == cudaSuccess) e = cudaMalloc(&T.d_D0, NQ * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(T.d_D0, D0.data(), NQ * sizeof(double), cudaMemcpyHostToDevice, st);
    // structural non-zeros of the two tables
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_count);
    cudaFree(d_off);
    if (e != cudaSuccess) {
        free_nc_tables(T);
        return cuda_fail(e, "node-space tables: build");
    }
    T.built = 1;
    return GRACE_OK;
}

cudaError_t launch_nc_functionals(const DevGroup &g, const NcTables &t, const double *d_g, const double *d_alpha,
                                  int n_cells, double *d_G, double *d_H, double *d_F, cudaStream_t st)
// d_G: [n][NQ] nodal values; d_H: [2][n][NQ] the coagulation- and fragmentation-weighted copies
{
    if (n_cells <= 0) return cudaSuccess;
    if (!t.built) return cudaErrorInvalidValue;
    const int NQ = t.NQ;
    NodeRule rule;
    for (int al = 0; al < g.Q; ++al) {
        double P[kB];
        // Legendre values at the Gauss node s_alpha (host recurrence, eq. 2.4)
        P[0] = 1.0;
        if (g.k >= 1) P[1] = g.gs[al];
        for (int n = 1; n < g.k; ++n) P[n + 1] = ((2.0 * n + 1.0) * g.gs[al] * P[n] - n * P[n - 1]) / (n + 1.0);
        for (int i = 0; i < kB; ++i) rule.phi[al * kB + i] = i <= g.k ? P[i] : 0.0;
    }
    const long long nn = (long long)n_cells * NQ;
    double *d_Hc = d_H, *d_Hf = d_H + nn;
    nc_nodal_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(g, rule, t.d_D0, d_g, d_alpha, n_cells, d_G, d_Hc,
                                                                   d_Hf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t per_warp = (size_t)NQ * 96 * sizeof(double);
    int wpb = (int)((200 * 1024) / per_warp);
    if (wpb > 4) wpb = 4;
    if (wpb < 1) return cudaErrorInvalidValue;
    const size_t smem = per_warp * wpb;
    e = cudaFuncSetAttribute(nc_fixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int cells_per_block = 32 * wpb;
    const dim3 fgrid((n_cells + cells_per_block - 1) / cells_per_block, (g.R + kRChunk - 1) / kRChunk);
    nc_fixed_kernel<<<fgrid, 32 * wpb, smem, st>>>(
        t.d_Cc, t.d_Cf, t.d_qlo, t.d_qhi, g.R, NQ, d_G, d_Hc, d_Hf, d_alpha, n_cells, d_F);
    e = cudaGetLastError();
    if (e != cudaSuccess || t.n_entries == 0) return e;
    const dim3 grid((n_cells + 127) / 128, g.R);
    nc_partial_kernel<<<grid, 128, 0, st>>>(g, (const NcEntry *)t.d_entries, t.d_seg, d_g, d_alpha, n_cells, d_F);
    return cudaGetLastError();
}


static NodeRule node_rule(const DevGroup &g)
{
    NodeRule rule;
    for (int al = 0; al < g.Q; ++al) {
        double P[kB];
        P[0] = 1.0;
        if (g.k >= 1) P[1] = g.gs[al];
        for (int n = 1; n < g.k; ++n) P[n + 1] = ((2.0 * n + 1.0) * g.gs[al] * P[n] - n * P[n - 1]) / (n + 1.0);
        for (int i = 0; i < kB; ++i) rule.phi[al * kB + i] = i <= g.k ? P[i] : 0.0;
    }
    return rule;
}

cudaError_t launch_nc_vjp(const DevGroup &g, NcTables &t, const double *d_g, const double *d_alpha, const double *d_mu,
                          int n_cells, double *d_G, double *d_H, double *d_gamma, double *d_w, cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    if (!t.built) return cudaErrorInvalidValue;
    const int NQ = t.NQ, R = g.R;
    cudaError_t e = cudaSuccess;
    if (!t.d_CcT) {
        const size_t nt = (size_t)R * NQ * NQ;
        e = cudaMalloc(&t.d_CcT, nt * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&t.d_CfT, nt * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&t.d_qloT, (size_t)R * NQ * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&t.d_qhiT, (size_t)R * NQ * sizeof(int));
        if (e == cudaSuccess) {
            nc_transpose_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(R, NQ, t.d_Cc, t.d_CcT);
            nc_transpose_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(R, NQ, t.d_Cf, t.d_CfT);
            nc_extent_kernel<<<(R * NQ + 127) / 128, 128, 0, st>>>(R, NQ, t.d_CcT, t.d_CfT, t.d_qloT, t.d_qhiT);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFree(t.d_CcT);
            cudaFree(t.d_CfT);
            cudaFree(t.d_qloT);
            cudaFree(t.d_qhiT);
            t.d_CcT = t.d_CfT = nullptr;
            t.d_qloT = t.d_qhiT = nullptr;
            return e;
        }
    }
    const NodeRule rule = node_rule(g);
    const long long nn = (long long)n_cells * NQ;
    double *d_Hc = d_H, *d_Hf = d_H + nn;
    nc_nodal_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(g, rule, t.d_D0, d_g, d_alpha, n_cells, d_G, d_Hc, d_Hf);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = ((size_t)3 * NQ + R) * 32 * sizeof(double);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;   // node count too large for this FP64 kernel
    e = cudaFuncSetAttribute(nc_vjp_node_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    nc_vjp_node_kernel<<<(n_cells + 31) / 32, 32, smem, st>>>(g, t.d_Cc, t.d_Cf, t.d_qlo, t.d_qhi, t.d_CcT, t.d_CfT,
                                                              t.d_qloT, t.d_qhiT, t.d_D0, R, NQ, d_G, d_Hc, d_Hf, d_mu,
                                                              d_alpha, n_cells, d_gamma);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long np = (long long)n_cells * g.P;
    nc_vjp_assemble_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(g, rule, d_gamma, NQ, n_cells, d_w);
    e = cudaGetLastError();
    if (e != cudaSuccess || t.n_entries == 0) return e;
    nc_vjp_partial_kernel<<<(n_cells + 127) / 128, 128, 0, st>>>(g, (const NcEntry *)t.d_entries, t.d_seg, d_g, d_mu,
                                                                 d_alpha, n_cells, d_w);
    return cudaGetLastError();
}

}  // namespace grace
