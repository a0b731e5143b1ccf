// Internal declarations of the GRACE-DG CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "grace.h"

namespace grace {

constexpr int kQMax = 16;   // Gauss points per quadrature piece on the device
constexpr int kKMax = 4;    // largest Legendre degree (bin minimum: closed form to k = 3, bracketed for k = 4)

// Everything a device kernel needs to know about a group, passed by value.
struct DevGroup {
    int N, k, K1, Q, P, R, n_if;
    int flux_mode, coag_kind, frag_kind, break_kind, cutoff_mode, mfrag_mode, limiter, has_delta;
    int cell_alpha;                  // ballistic alpha_turb per cell (node-space path)
    double x_min, x_max;
    double coag_p[8], frag_p[8], break_p[8];
    double beta_coag, beta_frag;     // Maxwellian probabilities (constant dv_rms)
    double gs[kQMax], gw[kQMax];     // Gauss-Legendre rule with Q points on [-1, 1]
    const double *edges;             // device, N+1 bin edges x_{j-1/2}
    const double *hbin;              // device, N bin widths h_j
    const double *inv_h;             // device, N values 1 / h_j
    const float *inv_h32;            // device, N values 1 / h_j in FP32
    const float *h32;                // device, N values h_j in FP32
};

// Tensor-core operand tiles of one group for one precision (built by precompute).
struct TcTiles {
    int built = 0;
    int n_tiles = 0;          // MMA N-tiles (functional group x p-window)
    int k_pad = 0;            // padded K extent of the A operand (elements)
    int k_ofs = 0;            // A column of coefficient 0 (a_column_offset; 0 for node-space tiles)
    int max_rows = 0;         // largest MMA N over the tiles
    int slot_bytes = 0;       // largest single B copy (bytes)
    void *d_b = nullptr;      // pre-swizzled B k-step blocks (all tiles back to back)
    void *d_b_pair = nullptr; // the same images for CTA pairs: per tile [half][k-step][plane][N / 2 rows]
                              // (forward tiles only; null elsewhere)
    TcTiles *at = nullptr;    // forward tiles of N <= 192 for the A-in-tensor-memory form (owned)
    void *d_desc = nullptr;   // per-tile descriptors
    int *d_ford = nullptr;    // functional ids in tile order
    size_t b_bytes = 0;
    long long mac_per_cell = 0;    // executed MACs per cell and RHS (tile shapes)
    long long mma_per_tile = 0;    // tcgen05.mma instructions per 128-cell tile and RHS
    long long nnz_fold = 0;        // min(non-zeros of T, of its upper-triangular fold): the MACs a cell needs
    int folded = 0;                // the tiles hold the folded tables (else T as built)
    double pred_clk = 0.0;         // cost-model SM cycles per 128-cell tile and RHS
    std::vector<int> group_tile;   // first tile of every functional group (+ end)
    std::vector<double> group_cost;   // cost-model cycles of every group
    // node-space tiles of a per-cell kernel group: the epilogue applies the fragmentation ramp
    int nc = 0;
    float *d_D0 = nullptr;         // [n_d0] D0 of every fixed node (0 past the last one)
    int n_d0 = 0;
    float ramp_a = 0.f, ramp_b = 0.f;   // pf(z) = clamp(ramp_a z + ramp_b, 0, 1), z = s D0
    int *d_written = nullptr;      // [R] 1 where the contraction writes the functional
    int vjp = 0;                   // window-major tiles of T + T^T for the VJP (launch_vjp_tc)
};

// Node-space tables of a group with a per-cell kernel parameter (grace_ncell.cu)
struct NcTables {
    int built = 0;
    int NQ = 0;                   // fixed Gauss nodes (N x Q), in increasing size
    double *d_Cc = nullptr;       // [R][NQ][NQ] upper-triangular weights of the coagulation factor
    double *d_Cf = nullptr;       // [R][NQ][NQ] upper-triangular weights of the fragmentation factor
    int *d_qlo = nullptr, *d_qhi = nullptr;   // [R*NQ] non-zero column range of each row
    double *d_D0 = nullptr;       // [NQ] D0 of each fixed node
    void *d_entries = nullptr;    // partial-pair entries, grouped by functional
    void *d_entf = nullptr;       // FP32 entries of the reduced-precision forms (coag/frag pairs merged)
    long long *d_segf = nullptr;  // [R+1] their ranges per functional
    long long n_entf = 0;
    long long *d_seg = nullptr;   // [R+1] entry ranges per functional
    long long n_entries = 0;
    // the adjoint (built on the first FP64 VJP): transposed fixed-pair tables and their extents
    double *d_CcT = nullptr, *d_CfT = nullptr;
    int *d_qloT = nullptr, *d_qhiT = nullptr;
};

// d T / d theta for one kernel parameter (central difference of the FP64 precompute)
struct ParamDeriv {
    int id = -1;                  // 0..7 coag_p, 8..15 frag_p, 16..23 break_p
    double step = 0.0;
    double *d_dT = nullptr;       // [R][P][P]
    int *d_qlo = nullptr, *d_qhi = nullptr, *d_prange = nullptr;
    TcTiles tc[3];                // tensor-form tiles of dT (built by the first tensor-form adjoint)
};

struct Group {
    grace_group_desc desc;
    DevGroup dg;
    std::vector<double> h_edges;
    double *d_edges = nullptr;
    double *d_T = nullptr;        // FP64 [R][P][P]
    int *d_qlo = nullptr;         // [R*P] first non-zero q of every row (P if empty)
    int *d_qhi = nullptr;         // [R*P] one past the last non-zero q
    int *d_prange = nullptr;      // [R][2] p range with non-empty rows
    long long nnz = 0;            // structural non-zeros of T (all rows)
    TcTiles tc[3];                // indexed by grace_precision
    TcTiles tcv[3];               // VJP tiles (built on the first tensor-form VJP / adjoint call)
    TcTiles tcs[3];               // species tiles (T unfolded; built on the first tensor-form species call)
    NcTables nc;                  // cell_alpha groups: node-space tables instead of T
    std::vector<ParamDeriv> dparams;
};

}  // namespace grace

struct grace_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<grace::Group> groups;
    int precomputed = 0;
    unsigned precision_mask = 0;
    // launch timing (grace_profile_enable)
    int profiling = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pairs[3];
    size_t ev_used = 0;
    int capturing = 0;              // a CUDA graph capture is in progress
};

namespace grace {

// The cells of one group inside a batch.  A "direct" part is a batch whose cells
// all belong to one group and sit in the caller's order: the caller's arrays
// are the part's state.  Otherwise the part gathers its cells' rows from the
// caller's packed layout into contiguous workspaces and scatters results back.
struct Part {
    int group = 0;
    int n = 0;
    bool direct = true;
    int *d_idx = nullptr;          // [n] caller cell index of each part cell
    long long *d_off = nullptr;    // [n] caller offset (doubles) of each part cell
    double *d_g = nullptr;         // [n][P] gathered state
    double *d_out = nullptr;       // [n][P] gathered output (RHS)
    double *d_dt = nullptr;        // [n]
    double *d_mass = nullptr;      // [n]
    unsigned char *d_flags = nullptr;  // [n]
    double *d_ic = nullptr;        // [n][4]
    double *d_F = nullptr;         // [n][R] functionals, FP64
    float *d_F32 = nullptr;        // [tiles][R][128] functionals from the tensor path
    double *d_g1 = nullptr, *d_g2 = nullptr;   // stage states
    double *d_mx = nullptr;        // tensor path: three stage states in the compact layout
    void *d_opA = nullptr;         // tensor-core A operand of the current stage
    double *d_alpha = nullptr;     // [n] per-cell alpha_turb (cell_alpha groups)
    double *d_G = nullptr, *d_H = nullptr;   // [n][NQ], [2][n][NQ] nodal values (cell_alpha groups)
    float *d_gh = nullptr;         // [tiles][P][128] scaled coefficients (cell_alpha groups, tensor forms)
    float *d_s = nullptr;          // [n] sqrt(alpha) in FP32 (cell_alpha groups, tensor forms)
    float *d_W32 = nullptr;        // tensor-form VJP: output planes [tc_vjp_planes()][tiles][Pw][128]
    float *d_mu32 = nullptr;       // tensor-form VJP: mu in FP32, [tiles][R][128]
    double *d_cscale = nullptr;    // tensor-form JVP / VJP: per-cell power-of-two scales
    double *d_gamma = nullptr;     // per-cell-kernel adjoint: [n][NQ] nodal gradient
    double *d_F2 = nullptr;        // per-cell-kernel JVP: [n][R] the second polarization's functionals
    double *d_eps = nullptr;       // per-cell-kernel JVP: [n] polarization scales
    size_t opA_bytes = 0;
    cudaStream_t stream = nullptr; // own stream for concurrent parts (null: the context's)
    cudaEvent_t done = nullptr;
};

}  // namespace grace

struct grace_batch {
    grace_ctx *ctx = nullptr;
    int n_cells = 0;
    std::vector<int> h_group;
    std::vector<long long> h_off;
    std::vector<grace::Part> parts;
    int *d_err = nullptr;          // device error word (bounded waits)
    double *d_adj = nullptr;       // adjoint workspace (checkpoints, stage states, adjoints)
    size_t adj_bytes = 0;
    cudaEvent_t fork = nullptr;
    // CUDA graph of one grace_step call (grace_batch_set_graph)
    int use_graph = 0;
    cudaGraphExec_t graph = nullptr;
    const void *graph_key[4] = {nullptr, nullptr, nullptr, nullptr};
    int graph_steps = -1, graph_prec = -1;
    int alpha_set = 0;             // grace_batch_cell_params was called
    // grouped tensor-form steps of batches with several groups (grace_batch_set_grouped)
    int use_grouped = 1;
    void *grouped = nullptr;       // the grouped plan (grace_batch.cu), built on first use
    void *host_io = nullptr;       // staging of grace_step_host (grace_host.cu), built on first use
    double *d_drift = nullptr;     // M_1 before / after a flagged grace_step [2][n] + per-cell
                                   // conservative-group bytes [n], built on the first flagged call
    unsigned *d_flag_or = nullptr; // grace_flags_check's reduction word
    void *hydro = nullptr;         // grace_substep workspace (grace_hydro.cu), built on first use
    void *species = nullptr;       // species workspace (grace_species.cu), built on first use
    void *implicit = nullptr;      // grace_rosenbrock_step workspace (grace_implicit.cu), built on first use
};

namespace grace {

// frees the staging of grace_step_host (waits for its copies first)
void free_host_io(grace_batch *b);
// frees the workspace of grace_substep
void free_hydro(grace_batch *b);
// frees the workspace of the species calls
void free_species(grace_batch *b);
void free_implicit(grace_batch *b);

// thread-local error detail
void set_error(const std::string &msg);
grace_status cuda_fail(cudaError_t e, const char *where);

// switches to a device for the duration of an ABI call and clears stale errors
struct Guard {
    int prev = -1;
    explicit Guard(int dev)
    {
        cudaGetLastError();
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard()
    {
        int cur;
        if (cudaGetDevice(&cur) == cudaSuccess && prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// host helpers
void gauss_rule(int Q, double *s, double *w);
DevGroup make_devgroup(const grace_group_desc &d, const double *d_edges);
int n_functionals(const grace_group_desc &d);

// kernels (launchers)
cudaError_t launch_build_T(const DevGroup &g, double *d_T, cudaStream_t st);
// dT_r/dtheta for parameter id (0..7 coag_p, 8..15 frag_p, 16..23 break_p): the same quadrature on
// dual numbers; dbeta_* the derivatives of the Maxwellian probabilities (maxwell_beta_derivs)
cudaError_t launch_build_dT(const DevGroup &g, int param_id, double dbeta_coag, double dbeta_frag, double *d_dT,
                            cudaStream_t st);
void maxwell_beta_derivs(const grace_group_desc &d, int id, double *dbeta_coag, double *dbeta_frag);
cudaError_t launch_row_extents(const DevGroup &g, const double *d_T, int *d_qlo, int *d_qhi,
                               int *d_prange, cudaStream_t st);
// functional chunks (grid y) of the FP64 contractions for a batch of n_cells
int fp64_functional_chunks(int n_cells, int R);
// species of mixed grains: F_s = sum_p gs_s[p] sum_q T[p, q] g[q], F layout [S][cells][R], S <= 4
cudaError_t launch_contract_fp64_species(const DevGroup &g, const double *d_T, const int *d_qlo, const int *d_qhi,
                                         const int *d_prange, int S, const double *d_gs, const double *d_g,
                                         int n_cells, double *d_F, cudaStream_t st);
cudaError_t launch_contract_fp64(const DevGroup &g, const double *d_T, const int *d_qlo,
                                 const int *d_qhi, const int *d_prange, const double *d_g,
                                 int n_cells, double *d_F, cudaStream_t st);

// K-c: fused flux difference (eq. evo), RK stage (eq. RK3), limiter, mass, flags.
struct UpdateArgs {
    const double *F = nullptr;     // [n][R] FP64 functionals, or
    const float *F32 = nullptr;    // [tiles][R][128] FP32 functionals (tensor path)
    const double *gn = nullptr;    // g^n
    const double *gs = nullptr;    // stage input g^(s)
    double *gout = nullptr;        // output (may alias gn)
    const double *dt = nullptr;    // [n] per-cell dt; null = write L (rhs mode)
    double a = 0.0, b = 1.0;       // gout = a gn + b (gs + dt L)
    int apply_limiter = 0;         // limit gout before writing (next step's reconstruction)
    double *mass = nullptr;        // [n] M_1 of gout, or null
    unsigned char *flags = nullptr;  // [n] OR-accumulated GRACE_FLAG_* bits, or null
    void *opA = nullptr;           // tensor-core A tiles of gout, or null
    int opA_prec = 0;              // GRACE_TF32 / GRACE_BF16X3
    int opA_kpad = 0;
    int opA_kofs = 0;              // A column of coefficient 0 (TcTiles::k_ofs)
    int in_mixed = 0;              // tensor path: gn / gs in the compact stage layout
    int out_mixed = 0;             // tensor path: gout in the compact stage layout
};
cudaError_t launch_update(const DevGroup &g, const UpdateArgs &a, int n_cells, cudaStream_t st);
// tcgen05 contraction: the flux functionals of every cell into d_F32 laid out as
// [128-cell tile][functional][row of the tile]; node-space tiles (t.nc) also need the
// per-cell s = sqrt(alpha) in FP32 (d_cell_s)
cudaError_t launch_contract_tc(const DevGroup &g, const TcTiles &t, int prec, const void *opA, int n_cells,
                               float *d_F32, int *d_err, cudaStream_t st, const float *d_cell_s = nullptr);
// K-c for the tensor path: reads d_F32 in the tile layout above
cudaError_t launch_update_tc(const DevGroup &g, const UpdateArgs &a, int n_cells, cudaStream_t st);
size_t f32_bytes_for(const DevGroup &g, int n_cells);
// K-c over many parts in one launch (uneven batches): one descriptor per part, parts ordered
// by first_block; modes: the step-start limiter (FP64 rows -> compact layout + A operand) and
// the stage update (compact in; compact or FP64 rows out)
struct UpdPart {
    DevGroup G;
    UpdateArgs A;
    int n_cells;
    int first_block;
};
enum { GROUPED_STAGE = 1, GROUPED_LIMIT = 2 };
int update_tc_grouped_cpb();
size_t update_tc_grouped_smem(const DevGroup &g, const UpdateArgs &a);
// the largest shared memory of the grouped stage-update launches for a group (A operand kpad)
size_t update_tc_grouped_max_smem(const DevGroup &g, int kpad);
// shared memory a block may opt in to on the current device
size_t update_smem_limit();
cudaError_t launch_update_tc_grouped(int mode, bool in_mixed, bool out_mixed, const UpdPart *d_parts, int n_parts,
                                     int n_blocks, size_t smem, cudaStream_t st);
// the step-start limiter of the tensor path: FP64 rows d_g -> compact stage layout + A operand
cudaError_t launch_limit_pack(const DevGroup &g, const double *d_g, int n_cells, unsigned char *flags,
                              double *mixed_out, void *opA, int opA_prec, int opA_kpad, int opA_kofs,
                              cudaStream_t st);
// bytes of one state in the compact stage layout (FP64 means, FP32 higher modes)
inline size_t mixed_bytes_for(const DevGroup &g, int n_cells)
{
    return (size_t)n_cells * g.N * (sizeof(double) + (size_t)g.k * sizeof(float));
}
cudaError_t launch_limit(const DevGroup &g, double *d_g, int n_cells, unsigned char *flags,
                         void *opA, int opA_prec, int opA_kpad, int opA_kofs, cudaStream_t st);
cudaError_t launch_mass(const DevGroup &g, const double *d_g, int n_cells, double *mass,
                        cudaStream_t st);
cudaError_t launch_project(const DevGroup &g, int ic_kind, const double *ic, int n_cells,
                           double *d_g, cudaStream_t st);
cudaError_t launch_pack_A(const DevGroup &g, const double *d_g, int n_cells, void *opA, int prec,
                          int kpad, int kofs, cudaStream_t st);

// events recorded around one launch when the context's profiling is on
struct LaunchTimer {
    grace_ctx *ctx;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchTimer(grace_ctx *c, int k, cudaStream_t s) : ctx(c), kind(k), st(s)
    {
        if (!ctx->profiling || ctx->capturing) return;
        while (ctx->ev_pool.size() < ctx->ev_used + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            ctx->ev_pool.push_back(e);
        }
        a = ctx->ev_pool[ctx->ev_used++];
        b = ctx->ev_pool[ctx->ev_used++];
        cudaEventRecord(a, st);
    }
    ~LaunchTimer()
    {
        if (!a) return;
        cudaEventRecord(b, st);
        ctx->ev_pairs[kind].push_back({a, b});
    }
};

// adjoint (grace_adjoint.cu)
cudaError_t launch_jvp_contract(const DevGroup &g, const double *T, const int *qlo, const int *qhi,
                                const int *prange, const double *a, const double *b, int n, double *F,
                                cudaStream_t st);
cudaError_t launch_vjp(const DevGroup &g, const double *T, const int *qlo, const int *qhi, const int *prange,
                       const double *gst, const double *lambda, double *mu_ws, int n, double *w, cudaStream_t st);
cudaError_t launch_limiter_vjp(const DevGroup &g, const double *gpre, double *lam, int n, cudaStream_t st);
cudaError_t launch_axpby_dt(int P, int n, double a, const double *x, double b, const double *y, const double *z,
                            const double *dt, double *out, cudaStream_t st);
cudaError_t launch_param_dot(int R, int n, const double *mu, const double *Fp, const double *dt, double w,
                             int n_params, int ip, double *dtheta, cudaStream_t st);
void free_param_derivs(Group &G);

// node-space path for per-cell kernels (grace_ncell.cu)
grace_status build_nc_tables(Group &G, cudaStream_t st);
void free_nc_tables(NcTables &t);
cudaError_t launch_nc_functionals(const DevGroup &g, const NcTables &t, const double *d_g, const double *d_alpha,
                                  int n_cells, double *d_G, double *d_H, double *d_F, cudaStream_t st);
// adjoint of the per-cell functionals (FP64): w = sum_r mu_r dF_r/dg for the functional weights mu
// ([n][R]), with the nodal workspaces of launch_nc_functionals and d_gamma ([n][NQ]); builds the
// transposed tables on first use (allocates and synchronises)
cudaError_t launch_nc_vjp(const DevGroup &g, NcTables &t, const double *d_g, const double *d_alpha, const double *d_mu,
                          int n_cells, double *d_G, double *d_H, double *d_gamma, double *d_w, cudaStream_t st);
// reduced-precision forms: FP32 partial entries (built once); per RHS the node values -> A
// operand (+ FP32 scaled coefficients, s per cell), the tcgen05 fixed part (launch_contract_tc
// with d_cell_s), then the FP32 partial part added into d_F32 ([tile][functional][row])
grace_status build_nc_tc_entries(Group &G, cudaStream_t st);
cudaError_t launch_nc_pack_tc(const DevGroup &g, const TcTiles &t, int prec, const double *d_g, const double *d_alpha,
                              int n_cells, void *opA, float *d_gh, float *d_s, cudaStream_t st);
cudaError_t launch_nc_partial_tc(const DevGroup &g, const NcTables &nt, const TcTiles &t, int n_cells,
                                 const float *d_gh, const float *d_s, float *d_F32, cudaStream_t st);

// tensor-core path
grace_status build_tc_tiles(Group &G, int prec, cudaStream_t st);
// the tile set a single-group forward contraction of t runs (t, or its A-in-tensor-memory tiles)
const TcTiles &tc_forward_tiles(const TcTiles &t);
grace_status build_tc_tiles_from(const Group &G, const double *d_T, int prec, TcTiles &out, cudaStream_t st,
                                 bool unfolded_only = false, bool pair_image = false, int max_n = 256);
// tiles of T as built (no fold) for the species contraction, into G.tcs[prec]
grace_status build_species_tiles(Group &G, int prec, cudaStream_t st);
// species of mixed grains: F_s[c, r] = sum_p ghat_{s,p} sum_q That_r[p, q] ghat_q for every species, the
// cells' total in opA (the A operand), the species' scaled coefficients in d_gsp
// ([S][cell tile][k_pad][128] FP32); F_s in the tile layout at d_F32 + s [cell tiles][R][128]
cudaError_t launch_contract_tc_species(const DevGroup &g, const TcTiles &t, int prec, const void *opA, int n_cells,
                                       const float *d_gsp, int n_species, float *d_F32, int *d_err, cudaStream_t st);
grace_status build_nc_tc_tiles(Group &G, int prec, cudaStream_t st);
grace_status build_vjp_tiles(Group &G, int prec, cudaStream_t st);
// multi-group contraction (uneven batches): the flux functionals of every part of a batch in one
// persistent launch; items (part, 128-cell tile) ordered by modelled cost
struct TcMultiPart {
    const TcTiles *t;
    const void *opA;
    float *F32;
    int n_cells, R;
};
struct TcMulti {
    void *d_groups = nullptr;
    void *d_items = nullptr;
    int n_items = 0;
    void *d_pair_items = nullptr;   // CTA pairs: (group, pair of its cell tiles)
    int n_pair_items = 0;
    int pair_ok = 0;                // every group has CTA-pair B images
    long long max_a = 0;
    int max_rows = 0;
    int prec = -1;
};
grace_status build_tc_multi(int prec, const std::vector<TcMultiPart> &parts, TcMulti &out);
cudaError_t launch_contract_tc_multi(const TcMulti &m, int *d_err, cudaStream_t st);
void free_tc_multi(TcMulti &m);
// VJP contraction: W[part][tile][Pw][128] (tc_vjp_planes() partial planes, FP32) with
// W = sum_r mu_r (Shat_r ghat) per cell, mu in the [tile][R][128] layout (FP32)
cudaError_t launch_vjp_tc(const DevGroup &g, const TcTiles &t, int prec, const void *opA, const float *d_mu32,
                          int n_cells, float *d_W32, int *d_err, cudaStream_t st);
// coefficient columns of the VJP output planes (P rounded up to the 16-wide windows)
inline int vjp_window_cols(const DevGroup &g) { return (g.P + 15) / 16 * 16; }
// partial output planes of the VJP contraction (one per epilogue warp of a TMEM lane quadrant)
int tc_vjp_planes();
void free_tc_tiles(TcTiles &t);
size_t opA_bytes_for(const DevGroup &g, int prec, int n_cells, int *kpad);


}  // namespace grace
