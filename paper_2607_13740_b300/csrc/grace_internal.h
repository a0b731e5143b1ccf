// Internal declarations of the GRACE-DG CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/grace.h"

namespace grace {

constexpr int kQMax = 16;   // Gauss points per quadrature piece on the device
constexpr int kKMax = 3;    // largest Legendre degree with an analytic limiter

// Everything a device kernel needs to know about a group, passed by value.
struct DevGroup {
    int N, k, K1, Q, P, R, n_if;
    int flux_mode, coag_kind, frag_kind, break_kind, cutoff_mode, mfrag_mode, limiter, has_delta;
    double x_min, x_max;
    double coag_p[8], frag_p[8], break_p[8];
    double beta_coag, beta_frag;     // Maxwellian probabilities (constant dv_rms)
    double gs[kQMax], gw[kQMax];     // Gauss-Legendre rule with Q points on [-1, 1]
    const double *edges;             // device, N+1 bin edges x_{j-1/2}
};

// Tensor-core operand tiles of one group for one precision (built by precompute).
struct TcTiles {
    int built = 0;
    int n_tiles = 0;          // N-tiles (bin group x p-window)
    int k_pad = 0;            // padded K extent of the A operand (elements)
    void *d_b = nullptr;      // pre-swizzled B tiles (all tiles back to back)
    void *d_desc = nullptr;   // per-tile descriptors
    size_t b_bytes = 0;
    long long mac_per_cell = 0;   // executed MACs per cell and RHS (tile shapes)
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
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pairs[2];
    size_t ev_used = 0;
};

struct grace_batch {
    grace_ctx *ctx = nullptr;
    int n_cells = 0;
    int single_group = 1;          // all cells in group 0 with the plain packed layout
    std::vector<int> h_group;
    std::vector<long long> h_off;
    // workspaces (device)
    double *d_F = nullptr;         // [n_cells][R] flux functionals, FP64
    float *d_F32 = nullptr;        // [n_cells][R] flux functionals from the tensor path
    double *d_g1 = nullptr;        // stage states
    double *d_g2 = nullptr;
    void *d_opA = nullptr;         // tensor-core A operand tiles (current stage)
    size_t opA_bytes = 0;
    unsigned char *d_flags = nullptr;
    int *d_err = nullptr;          // device error word (bounded waits)
};

namespace grace {

// thread-local error detail
void set_error(const std::string &msg);
grace_status cuda_fail(cudaError_t e, const char *where);

// host helpers
void gauss_rule(int Q, double *s, double *w);
DevGroup make_devgroup(const grace_group_desc &d, const double *d_edges);
int n_functionals(const grace_group_desc &d);

// kernels (launchers)
cudaError_t launch_build_T(const DevGroup &g, double *d_T, cudaStream_t st);
cudaError_t launch_row_extents(const DevGroup &g, const double *d_T, int *d_qlo, int *d_qhi,
                               int *d_prange, cudaStream_t st);
cudaError_t launch_contract_fp64(const DevGroup &g, const double *d_T, const int *d_qlo,
                                 const int *d_qhi, const int *d_prange, const double *d_g,
                                 int n_cells, double *d_F, cudaStream_t st);

// K-c: fused flux difference (eq. evo), RK stage (eq. RK3), limiter, mass, flags.
struct UpdateArgs {
    const double *F = nullptr;     // [n][R] FP64 functionals, or
    const float *F32 = nullptr;    // [n][R] FP32 functionals (tensor path)
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
};
cudaError_t launch_update(const DevGroup &g, const UpdateArgs &a, int n_cells, cudaStream_t st);
cudaError_t launch_limit(const DevGroup &g, double *d_g, int n_cells, unsigned char *flags,
                         void *opA, int opA_prec, int opA_kpad, cudaStream_t st);
cudaError_t launch_mass(const DevGroup &g, const double *d_g, int n_cells, double *mass,
                        cudaStream_t st);
cudaError_t launch_project(const DevGroup &g, int ic_kind, const double *ic, int n_cells,
                           double *d_g, cudaStream_t st);
cudaError_t launch_pack_A(const DevGroup &g, const double *d_g, int n_cells, void *opA, int prec,
                          int kpad, cudaStream_t st);

// tensor-core path
grace_status build_tc_tiles(Group &G, int prec, cudaStream_t st);
void free_tc_tiles(TcTiles &t);
size_t opA_bytes_for(const DevGroup &g, int prec, int n_cells, int *kpad);
cudaError_t launch_contract_tc(const DevGroup &g, const TcTiles &t, int prec, const void *opA,
                               int n_cells, float *d_F32, int *d_err, cudaStream_t st);

}  // namespace grace
