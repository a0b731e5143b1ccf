/*
 * grace.h - C ABI of the B300-native GRACE-DG hot path.
 *
 * The library evaluates the right-hand side L[g] of the DG-discretised
 * Smoluchowski equation (coagulation flux plus the conservative nonlinear
 * fragmentation flux) for the Legendre modal coefficients of every
 * logarithmic mass bin, over a batch of independent cells, and advances the
 * batch with SSP-RK3.  The method is that of Yang, Chen & Bai,
 * "GRACE-DG: A Discontinuous Galerkin Method-Based Code for General
 * Nonlinear Coagulation-Fragmentation Equations" (arXiv 2607.13740).
 *
 * Conventions for every function below:
 *   - Pointers marked "device" must point to CUDA device memory of the
 *     context's device; "host" pointers to ordinary host memory.  The caller
 *     owns every buffer it passes; the library owns its context, batch and
 *     workspaces and frees them in grace_batch_destroy / grace_destroy.
 *   - Coefficient arrays are FP64, packed cell after cell; a cell of a group
 *     with N bins and degree k holds P = N (k+1) doubles ordered bin-major,
 *     coefficient index fastest: g[c*P + j*(k+1) + i] = g_j^i of cell c.
 *     Pointers must be 16-byte aligned.
 *   - Compute calls (grace_project, grace_rhs, grace_step, grace_mass,
 *     grace_limit, grace_rhs_jvp, grace_rhs_vjp) are asynchronous on the
 *     stream bound with grace_set_stream (the legacy default stream if none)
 *     and do not synchronise.  grace_setup, grace_precompute and
 *     grace_bind_batch allocate and synchronise.
 *   - No exception or abort crosses this interface.  Every function returns a
 *     grace_status; grace_last_error() gives a human-readable detail for the
 *     calling thread.  CUDA errors map to GRACE_ERR_CUDA.
 *   - One context per host thread at a time.
 */
#ifndef GRACE_H
#define GRACE_H

#if defined(__GNUC__)
#define GRACE_API __attribute__((visibility("default")))
#else
#define GRACE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grace_ctx grace_ctx;
typedef struct grace_batch grace_batch;

typedef enum {
    GRACE_OK = 0,
    GRACE_ERR_ARG = 1,          /* invalid argument (null pointer, size, kind)        */
    GRACE_ERR_ORDER = 2,        /* call sequence violated (e.g. rhs before precompute) */
    GRACE_ERR_CUDA = 3,         /* a CUDA runtime call failed                          */
    GRACE_ERR_NOMEM = 4,        /* device or host allocation failed                    */
    GRACE_ERR_UNSUPPORTED = 5,  /* valid request the build does not implement          */
    GRACE_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up                  */
    GRACE_WARN_CELLS = 100      /* grace_flags_check: some cell has a status bit set;
                                   every result was written                           */
} grace_status;

/* arithmetic of the bulk flux contraction (Sec. 3.3 quadrature, folded into a
   coefficient tensor); everything else always runs in FP64 */
typedef enum {
    GRACE_FP64 = 0,    /* FP64 CUDA-core contraction                                */
    GRACE_TF32 = 1,    /* tcgen05 kind::tf32, FP32 accumulation in tensor memory     */
    GRACE_BF16X3 = 2   /* tcgen05 kind::f16 with bf16 hi+lo splits of both operands, */
                       /* three products hi*hi + hi*lo + lo*hi, FP32 accumulation    */
} grace_precision;

/* collision kernels: K = p0 (Sec. 4.2), p0 (x+y) (Sec. 4.3), p0 x y (Sec. 4.4);
   Maxwellian sigma * dv_rms * beta (Sec. 4.5: p0 = dv_rms, p1 = v_b for
   coagulation or v_f for fragmentation); ballistic-turbulent (library model,
   p0 rho_s, p1 Sigma_g, p2 c_s, p3 alpha_turb, p4 v_frag, p5 ramp half-width
   fraction, p6 rate scale) */
enum { GRACE_COAG_NONE = 0, GRACE_COAG_CONST = 1, GRACE_COAG_ADD = 2, GRACE_COAG_MULT = 3,
       GRACE_COAG_MAXWELL = 4, GRACE_COAG_BALLISTIC = 5 };
enum { GRACE_FRAG_NONE = 0, GRACE_FRAG_MULT = 1, GRACE_FRAG_MAXWELL = 2, GRACE_FRAG_BALLISTIC = 3 };
/* breakage: uniform binary (Sec. 4.4), power law + remnant (eq. break with
   m_frag of eq. mfrag; break_p[0] = power-law index alpha), and the delta
   b = delta(w - u - v) that turns eq. (Ffrag) into coagulation */
enum { GRACE_BREAK_UNIFORM_BINARY = 0, GRACE_BREAK_POWERLAW_REMNANT = 1, GRACE_BREAK_COAG_DELTA = 2 };
/* initial conditions for grace_project (per-cell parameters q[0..3]):
   EXP g0 = q0 x exp(-x/q1); POWERLAW g0 = q0 x^q1 on [q2, q3]; FIRST_BIN g0 = q0 in bin 0 */
enum { GRACE_IC_EXP = 0, GRACE_IC_POWERLAW = 1, GRACE_IC_FIRST_BIN = 2 };
/* flux truncation of Sec. 3.3: Delta x = -u + x_min (mass conserving) or 0 */
enum { GRACE_FLUX_CONSERVATIVE = 0, GRACE_FLUX_NONCONSERVATIVE = 1 };
/* per-cell status bits written by grace_step / grace_limit */
enum { GRACE_FLAG_NEGATIVE_MEAN = 1,  /* a cell mean g_j^0 went negative (eq. dt violated) */
       GRACE_FLAG_LIMITED = 2,        /* the scaling limiter changed a bin (eq. gamma < 1)  */
       GRACE_FLAG_NONFINITE = 4,      /* a coefficient became Inf or NaN                    */
       GRACE_FLAG_CFL = 8,            /* a stage broke eq. (dt) in a bin losing mass:
                                         L_j^0 < 0 and g_j^0 + dt L_j^0 <= 0 (one rounding)
                                         for the stage input g_j^0 */
       GRACE_FLAG_MASS_DRIFT = 16 };  /* conservative groups, cells with none of the bits
                                         above but LIMITED: M_1 = sum_j h_j g_j^0 changed over
                                         the grace_step call by more than
                                         max(1e-10, 32 n_steps 2^-53) of its value, or
                                         became NaN (eq. g0 with eq. dt kept conserves it to
                                         round-off, so the bit means a conservation failure) */

/* One (grid, order, physics) combination shared by the cells of a group. */
typedef struct {
    int n_bins;       /* N >= 2 bins on [x_min, x_max]: logarithmic (Sec. 3.1) or edges  */
    int order_k;      /* k in 0..4: Legendre degree (eq. 2.3); 0..3 with cell_alpha      */
    int quad_q;       /* Gauss points per quadrature piece; 0 means k+1 (Sec. 3.3), <= 16 */
    int flux_mode;    /* GRACE_FLUX_*                                                   */
    int coag_kind;    /* GRACE_COAG_*                                                   */
    int frag_kind;    /* GRACE_FRAG_*                                                   */
    int break_kind;   /* GRACE_BREAK_*                                                  */
    int cutoff_mode;  /* 0: power law up to m_frag (eq. break); 1: up to max(u, v)       */
    int limiter;      /* 1: scaling limiter once per step before the RK stages; 0: off  */
    int mfrag_mode;   /* 0: m_frag from eq. (mfrag); 1: destructive, m_frag = u + v      */
    double x_min, x_max;
    double coag_p[8];
    double frag_p[8];
    double break_p[8];
    int cell_alpha;   /* 1: the ballistic-turbulent kernels take alpha_turb (p3) per cell, set
                         by grace_batch_cell_params; coag_kind must be BALLISTIC, frag_kind NONE
                         or BALLISTIC with the same p0..p2, p4..p6 as coagulation; 0: per group */
    int reserved_;    /* zero */
    const double *edges;  /* host, n_bins + 1 strictly increasing finite bin edges with
                             edges[0] = x_min and edges[n_bins] = x_max, copied by grace_setup
                             (the pointer is not kept); NULL: the logarithmic grid of Sec. 3.1 */
} grace_group_desc;

GRACE_API int grace_version(void);
GRACE_API const char *grace_status_string(grace_status s);
/* detail of the last failing call on this thread ("" if none); valid until the next call */
GRACE_API const char *grace_last_error(void);

/* Creates a context on CUDA device `device` for n_groups >= 1 group
   descriptions (host array, copied).  Validates every description. */
GRACE_API grace_status grace_setup(grace_ctx **ctx, int n_groups, const grace_group_desc *groups, int device);

/* Binds the CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
   used by every later compute call of this context and its batches; NULL = legacy stream. */
GRACE_API grace_status grace_set_stream(grace_ctx *ctx, void *cuda_stream);

/* Builds, on the GPU in FP64, the coefficient tensors of every group: for each
   flux functional r (the interface fluxes F(x_{j+1/2}) of eqs. Fcoagtrun /
   Ffragtrun, and the volume integrals int_{I_j} F d_x phi_i of eq. evo, by the
   nested Gauss quadrature of Sec. 3.3 and the reordered App. B form for
   breakage with a Dirac remnant) the P x P matrix T_r with
   functional_r = sum_{p,q} T_r[p,q] g_p g_q.  precision_mask bit (1<<GRACE_TF32)
   and (1<<GRACE_BF16X3) also build the tensor-core operand tiles.  Synchronises. */
GRACE_API grace_status grace_precompute(grace_ctx *ctx, unsigned precision_mask);

/* Number of coefficients P and of flux functionals R of a group. */
GRACE_API grace_status grace_group_info(const grace_ctx *ctx, int group, int *n_coef, int *n_functionals);

/* Binds a batch of n_cells >= 1 cells; cell_group (host, may be NULL = all in
   group 0) gives each cell's group, in any order and mix.  Allocates the batch
   workspaces.  The cell layout is packed in the given order (cell c holds
   P(group(c)) doubles); grace_batch_offsets returns it.  Cells of one group
   are computed together on their own stream; a batch of one group in caller
   order works directly on the caller's arrays. */
GRACE_API grace_status grace_bind_batch(grace_ctx *ctx, int n_cells, const int *cell_group, grace_batch **batch);
/* host out[n_cells + 1]: offset (in doubles) of every cell's coefficients; out[n_cells] = total */
GRACE_API grace_status grace_batch_offsets(const grace_batch *batch, long long *out);

/* Projects per-cell initial conditions (eq. init, 16-point Gauss rule per bin).
   ic_params: device [n_cells][4] doubles; g: device output. */
GRACE_API grace_status grace_project(grace_batch *batch, int ic_kind, const double *ic_params, double *g);

/* L = L[g] (eq. evo) for every cell.  g, L: device, packed layout (L has g's layout). */
GRACE_API grace_status grace_rhs(grace_batch *batch, const double *g, double *L, int precision);

/* n_steps SSP-RK3 steps (eq. RK3), each preceded by the scaling limiter
   (eqs. recon, gamma) when the group enables it, in place on g (device).
   dt: device [n_cells] per-cell time steps.  mass (device [n_cells] or NULL)
   receives M_1 = sum_j h_j g_j^0 after the last step; flags (device
   [n_cells] or NULL) receives the OR of GRACE_FLAG_* bits over all stages,
   and the mass-drift bit from M_1 before and after the call (two extra mass
   passes; the first call with flags allocates 17 bytes per cell and
   synchronises). */
GRACE_API grace_status grace_step(grace_batch *batch, double *g, const double *dt, int n_steps, int precision,
                        double *mass, unsigned char *flags);

/* grace_step on host buffers: uploads h_g (host, the packed layout of the
   batch) and h_dt (host [n_cells]), runs n_steps steps exactly as grace_step
   (same kernels, same results bit for bit), and downloads the new state to
   h_out (host, may equal h_g), M_1 to h_mass and the status bits to h_flags
   (host [n_cells] each, or NULL).  The copies run on two streams owned by the
   batch and the steps on the bound stream; device staging is double-buffered,
   so with page-locked host buffers successive calls overlap the upload of the
   next call and the download of the previous one with the steps.  A call whose
   h_g or h_dt overlaps the previous call's h_out uploads after that download,
   so in-place and chained calls (h_out of one call as h_g of the next) need no
   wait in between.  Returns once the work is enqueued: the caller keeps h_g
   and h_dt unchanged and reads h_out, h_mass and h_flags only after
   grace_step_host_wait (synchronising the bound stream alone is not enough).  With pageable host memory the CUDA
   runtime makes the copies synchronous and nothing overlaps.  The first call
   allocates two staging copies of the batch's state (and synchronises).  With
   graph replay on (grace_batch_set_graph) every call uses one staging slot so
   the graph is reused, and calls do not overlap.  Errors: GRACE_ERR_ARG for a
   NULL h_g, h_out or h_dt or n_steps < 0, otherwise those of grace_step. */
GRACE_API grace_status grace_step_host(grace_batch *batch, const double *h_g, double *h_out, const double *h_dt,
                                       int n_steps, int precision, double *h_mass, unsigned char *h_flags);

/* Waits until every grace_step_host call of the batch has finished its copies
   (and hence its steps); the host outputs are then complete. */
GRACE_API grace_status grace_step_host_wait(grace_batch *batch);

/* The FP64 L = L[g] of grace_rhs for n_cells cells of one group, for callers
   that cannot allocate device memory: codes whose device memory belongs to
   another framework's pool allocator, and solvers calling the RHS inside a
   per-substep loop where an allocation (cudaMalloc synchronises the device)
   is not acceptable.  This call allocates nothing: its flux-functional
   workspace is a fixed 16 MiB array (2^21 doubles) inside the library, held on
   every GPU that loads the library until the process exits, so
   n_cells * n_functionals must not exceed 2^21 (GRACE_ERR_ARG otherwise; C2's
   N = 40, k = 2 group allows 17,620 cells per call).  The context must have
   been set up and precomputed beforehand (those calls do allocate).  Every
   call looks up the array's device address on the context's device (a host
   query); the first lookup on a device may load the library's device code
   there, so make the first call on a device before any stream capture.  The
   first call sets up this lookup.  All calls share the one array:
   calls whose executions overlap on the GPU (other streams, other threads)
   race and must be serialised by the caller.  g, L: device, packed layout; runs
   on the context's bound stream.  The paper has no counterpart of this call. */
GRACE_API grace_status grace_rhs_noalloc(grace_ctx *ctx, int group, int n_cells, const double *g, double *L);

/* enable != 0: grace_step records its whole launch sequence (every group of the
   batch, every step and stage) into a CUDA graph on the first call with a given
   (g, dt, mass, flags, n_steps, precision) and replays the graph on later calls
   with the same arguments.  Needs a bound non-default stream; launch timing
   (grace_profile_enable) is not recorded inside graphs. */
GRACE_API grace_status grace_batch_set_graph(grace_batch *batch, int enable);

/* enable != 0 (the default): grace_step of a batch with several groups in a tensor-core
   form runs the whole batch in a fixed number of launches per stage - one multi-group
   tcgen05 contraction over every group's cell tiles (work items ordered by modelled cost)
   and one K-c launch over all parts - instead of one launch sequence per group.  Its
   descriptors are built on the first such call (allocates and synchronises, before any
   graph capture).  enable = 0 restores the per-group launches.  Same results bit for bit. */
GRACE_API grace_status grace_batch_set_grouped(grace_batch *batch, int enable);

/* Species of mixed grains (Sec. 5.3): grains are mixtures of n_species (1..4) constituent
   species whose partial mass densities g_s share the mass grid, g = sum_s g_s.  Every flux
   integral carries the share of the products of its outer collider, so a species' rate is
   L_s = L[g_s; g]: the flux integrals of eqs. (Fcoagtrun), (Ffragtrun) and App. B with g_s in the
   outer collider's slot and g in its partner's (the library's reading; the paper states no
   equations).  sum_s L_s = L[g], and each species' mass is conserved by conservative fluxes.
   gs, Ls: device, [n_species][n_cells][P] (species-major, each species a packed state of the
   batch).  precision: GRACE_FP64 (one pass over T on the CUDA cores, the partner's row sums shared
   by the species), or GRACE_TF32 / GRACE_BF16X3 (precomputed for the group): one tcgen05 pass over
   T as built with the cells' total as the A operand, each species contracting the accumulator in
   the epilogue; the reduced-precision bars of those forms apply.  Batches of one group in caller
   order without per-cell kernel parameters (GRACE_ERR_UNSUPPORTED otherwise).  The first call
   (and the first of each tensor form) allocates a workspace and plans tiles (synchronises). */
GRACE_API grace_status grace_rhs_species(grace_batch *batch, int n_species, const double *gs, double *Ls,
                                         int precision);

/* n_steps SSP-RK3 steps (eq. RK3) of the species, in place on gs ([n_species][n_cells][P],
   device): every stage forms the total of its input, then each species' rate and stage update;
   the scaling limiter acts on each species (once per step, as grace_step).  mass (device
   [n_species][n_cells] or NULL) receives each species' M_1 after the last step; flags (device
   [n_cells] or NULL) the OR of the status bits of the cell's species, the mass-drift bit from the
   cell's total M_1.  precision, restrictions and workspace as grace_rhs_species. */
GRACE_API grace_status grace_step_species(grace_batch *batch, int n_species, double *gs, const double *dt,
                                          int n_steps, int precision, double *mass, unsigned char *flags);

/* Linearly implicit (Rosenbrock-Euler) step for stiff cells, the implicit option of the coupling
   to a hydrodynamics code (Sec. 5.2): per cell, (I - dt_c J(g)) k = dt_c L[g] with J = dL/dg at g,
   then g <- g + k (in place; g, dt device [n_cells][P] / [n_cells]).  Each cell's system is solved
   by restarted GMRES(krylov_dim) (1 .. 64 basis vectors per cycle, at most max_restarts restarts)
   whose matrix-vector products are grace_rhs_jvp in `precision` over the whole batch (one JVP per
   Krylov iteration); a cell stops when its residual is below rtol (0 < rtol < 1) of its initial
   residual ||dt_c L||.  *iterations (host, nullable) receives the Krylov iterations taken.  The
   paper gives no implicit scheme; this is the library's, on the JVP of the adjoint's tables.
   Allocates a workspace on first use; synchronises once per cycle and every 4 iterations (to stop
   when every cell has converged), so it is not captured in a CUDA graph.  Restrictions of
   grace_rhs_jvp (one group in caller order, no per-cell kernel parameters). */
GRACE_API grace_status grace_rosenbrock_step(grace_batch *batch, double *g, const double *dt, int precision,
                                             int krylov_dim, int max_restarts, double rtol, int *iterations);

/* Operator-split coupling to a hydrodynamics code (Sec. 5.2): advances every cell by its
   own interval dt_hydro[c] (device [n_cells]) in sub-steps sized by the eq. (dt)
   positivity bound.  The FP64 RHS at the start gives each cell's bound
   B_c = min over bins losing mass (L_j^0 < 0) of g_j^0 / |L_j^0| and its count
   n_c = ceil(dt_hydro_c / (cfl B_c)); the batch then takes N = min(max_c n_c,
   max_substeps) steps of grace_step in which cell c moves by dt_hydro_c / N (<= cfl B_c
   unless max_substeps capped N).  *n_sub (host, nullable) receives N.  cfl > 0, e.g. 0.5.
   Status bit 8 reports cells whose bound tightened below the step during the interval.
   Allocates a workspace on the first call; synchronises once per call (to read N), so it
   is not captured in a CUDA graph.  Errors: GRACE_ERR_ARG for a null argument, cfl <= 0 or
   max_substeps < 1, otherwise those of grace_rhs and grace_step.  The paper gives no
   algorithm for the coupling; this sub-cycling is the library's. */
GRACE_API grace_status grace_substep(grace_batch *batch, double *g, const double *dt_hydro, double cfl,
                                     int max_substeps, int precision, double *mass, unsigned char *flags,
                                     int *n_sub);

/* M_1 = sum_j h_j g_j^0 per cell (Sec. 4.1).  g, mass: device. */
GRACE_API grace_status grace_mass(grace_batch *batch, const double *g, double *mass);

/* The scaling limiter alone, in place; flags (device [n_cells] or NULL). */
GRACE_API grace_status grace_limit(grace_batch *batch, double *g, unsigned char *flags);

/* Tangent-linear RHS: Jv = (dL/dg)(g) v.  L is quadratic in g, so
   Jv = D (g^T (T_r + T_r^T) v)_r exactly.  g, v, Jv: device, packed layout.
   GRACE_FP64 evaluates that form on the CUDA cores; GRACE_TF32 / GRACE_BF16X3 use
   the exact polarization Jv = [L(g + eps v) - L(g - eps v)] / (2 eps) with two
   tensor-core contractions, eps = 2^(e_g - e_v) per cell (e_x the binary exponent
   of the cell's largest |x|); their accuracy is that of the forward form.  The
   tensor forms need the precision in grace_precompute's mask before the batch was
   bound.  Batches of one group without per-cell kernel parameters only.  The paper
   has no adjoint; this and the next three calls differentiate its scheme. */
GRACE_API grace_status grace_rhs_jvp(grace_batch *batch, const double *g, const double *v, double *Jv, int precision);

/* Adjoint RHS: w = (dL/dg)(g)^T lambda = sum_r mu_r (T_r + T_r^T) g, mu = D^T lambda.
   g, lambda, w: device.  GRACE_TF32 / GRACE_BF16X3 contract tiles of T_r + T_r^T on
   the tensor cores (built, with the call's workspaces, on the first such call of a
   batch, which then allocates and synchronises). */
GRACE_API grace_status grace_rhs_vjp(grace_batch *batch, const double *g, const double *lambda, double *w,
                                     int precision);

/* Prepares parameter gradients for grace_adjoint: for each id (0..7 coag_p[i],
   8..15 frag_p[i-8], 16..23 break_p[i-16]) builds dT_r/dtheta.  rel_step <= 0: exactly, by
   forward-mode dual numbers through the FP64 precompute (the derivatives of the kernels, of the
   breakage mass functions of eqs. (break), (inte1), (inte2) and App. B, and of the Maxwellian
   probabilities of Sec. 4.5, carried through the same quadrature sums; a clamp such as the
   fragmentation ramp contributes its one-sided derivative).  rel_step > 0: a central difference
   of the FP64 precompute with that relative step (kept for cross-checks).  Replaces any earlier
   set.  Allocates and synchronises. */
GRACE_API grace_status grace_param_grad_setup(grace_ctx *ctx, int group, int n_params, const int *param_ids,
                                              double rel_step);

/* Discrete adjoint of n_steps steps of grace_step (limiter + SSP-RK3) from g0
   with per-cell dt: given lambda_T = dJ/dg(t_end), returns lambda_0 = dJ/dg0
   and, when dtheta is not NULL, dtheta[c * n_params + i] = dJ/dtheta_i from
   cell c for the parameters of grace_param_grad_setup.  Stores a checkpoint
   every ckpt_every steps and recomputes the stage states of one segment at a
   time.  g0, dt, lambda_T, lambda_0, dtheta: device.  The workspace
   (checkpoints + one segment's stage states + adjoint vectors) is allocated on
   first use and kept with the batch; that call synchronises.  With GRACE_TF32 /
   GRACE_BF16X3 the forward sweep and its recomputation run in that tensor form and
   every stage's VJP uses grace_rhs_vjp's tensor form; the limiter and parameter terms
   stay FP64. */
GRACE_API grace_status grace_adjoint(grace_batch *batch, const double *g0, const double *dt, int n_steps,
                                     int ckpt_every, const double *lambda_T, double *lambda_0, double *dtheta,
                                     int precision);

/* Launch timing with CUDA events recorded on the bound stream around every
   contraction (kernel 0) and flux-update (kernel 1) launch of this context;
   kernel 2 covers the per-cell-kernel pieces of the reduced-precision forms
   around their contraction (node values, FP32 partial entries).
   grace_profile_read synchronises the stream, returns the summed device time
   in milliseconds and the launch count since the last read, and resets them. */
GRACE_API grace_status grace_profile_enable(grace_ctx *ctx, int enable);
GRACE_API grace_status grace_profile_read(grace_ctx *ctx, int kernel, double *total_ms, long long *launches);

/* Structural statistics of a group's coefficient tensors: the number of
   non-zero entries of all T_r (the algorithmic multiply-adds of one cell's
   RHS) and the multiply-adds the tensor-core tiles of `precision` execute
   per cell and RHS (0 if not built). */
GRACE_API grace_status grace_group_stats(const grace_ctx *ctx, int group, int precision, long long *nnz,
                                         long long *tile_macs);

/* Tensor-core tile plan of one group for precision GRACE_TF32 or GRACE_BF16X3
   (built by grace_precompute; the tile shapes are chosen by a cost model over
   the sparsity of T, see the contraction's documentation).  Writes 8 values
   (host): [0] N-tiles, [1] tcgen05.mma instructions per 128-cell tile and RHS,
   [2] executed multiply-adds per cell and RHS, [3] bytes of the B images,
   [4] cost-model SM cycles per 128-cell tile and RHS, [5] widest MMA N,
   [6] the multiply-adds a cell needs (non-zeros of T or of its symmetric fold, the
   smaller), [7] 1 when the tiles hold the folded tables, 0 when T as built.
   GRACE_ERR_ORDER when that precision was not precomputed. */
GRACE_API grace_status grace_tile_info(const grace_ctx *ctx, int group, int precision, long long *info);

/* Per-cell turbulence strength for the cells of groups with cell_alpha = 1
   (non-separable kernels: the flux functionals are no longer fixed quadratic
   forms of the coefficients, so they are evaluated from node-space tables and a
   per-cell kernel factor each RHS; FP64 only).  alpha: device, n_cells doubles in
   the batch's cell order (entries of other groups are ignored), copied.
   GRACE_ERR_ORDER from grace_rhs / grace_step on such a batch until this was called. */
GRACE_API grace_status grace_batch_cell_params(grace_batch *batch, const double *alpha);

/* OR of flags (device [n_cells], as written by grace_step / grace_limit) over
   the batch's cells, into *any (host, may be NULL).  Synchronises the bound
   stream (compute calls never do, so they report per-cell problems only
   through the flags array).  Returns GRACE_WARN_CELLS when some bit is set,
   GRACE_OK otherwise. */
GRACE_API grace_status grace_flags_check(grace_batch *batch, const unsigned char *flags, unsigned *any);

/* Reads and clears the batch's device error word: non-zero bits mean a bounded
   device-side wait inside a tensor-core launch gave up (the launch then wrote
   no results for the affected cells).  Synchronises the bound stream; returns
   GRACE_ERR_TIMEOUT when the word was non-zero. */
GRACE_API grace_status grace_batch_error(grace_batch *batch, int *code);

/* Failure-detection check: arms a one-shot fault of the next tensor-core
   contraction launched in this process (any context or batch).  That launch
   issues none of its operand-table copies, so its MMA issuer waits on a
   shared-memory barrier that nothing arrives at, and every bounded wait of
   the launch gives up after wait_cycles SM clock cycles (1 .. 4e9; the
   default limit of every other launch is 4e9, about 2 s) instead of the
   default.  The kernel then takes its normal abort path: it records the
   failure in the batch's device error word, drains its copies in flight,
   frees its tensor memory and returns without results; grace_batch_error
   reports GRACE_ERR_TIMEOUT.  Nothing faults or hangs.  The paper has no
   counterpart of this call. */
GRACE_API grace_status grace_test_arm_wait_timeout(long long wait_cycles);

/* Selects, for the whole process, where the tensor-form (TF32, BF16X3) forward
   contractions run on CTA pairs: two SMs of a cluster share every work item,
   one tcgen05.mma covering 256 cells (cta_group::2), each SM loading half of
   every table block, so a group's tables stream once per two cell tiles.
   mode 0 (the default): never; 1: every forward contraction of at least 256
   cells; 2: multi-group launches only (uneven batches).  Both forms run the
   same tiles in the same order; on a B300 the pairs measured slower than
   single CTAs in both places, so they are off unless selected.
   Returns GRACE_ERR_ARG for other values.  The paper has no counterpart of
   this call. */
GRACE_API grace_status grace_set_cta_pairs(int mode);

/* Selects, for the whole process, whether single-group forward contractions in
   the tensor forms keep the cells' A tile in tensor memory: enable = 1, for
   groups whose A tile takes at most 128 TMEM columns (TF32 or BF16 hi + lo of
   at most 128 coefficients), with table tiles of N <= 192 and a three-deep
   ring of 64 KB table copies in shared memory; enable = 0 (the default) keeps
   A in shared memory (N <= 256, two ring slots), which measured faster on a
   B300.  CTA pairs selected with mode 1 take precedence.  Returns
   GRACE_ERR_ARG for other values.  The paper has no counterpart of this call. */
GRACE_API grace_status grace_set_tc_a_in_tmem(int enable);

/* ---------------------------------------------------------------------------
   Two-dimensional (mass x, volume v) DG (Sec. 5.3, "Toward a Multidimensional
   Treatment").  Cells I_{j,m} = I_j x I_m of logarithmic grids (x_{j-1/2} =
   x_min (x_max/x_min)^(j/n_x), likewise in v), the tensor-product Legendre basis
   phi_p(xi_j(x)) phi_q(eta_m(v)) with p, q <= order_k, and the unknown g = x f.
   The right-hand side is the Galerkin weak form of the multidimensional
   Smoluchowski equation of Sec. 5.3 tested with x phi_{j,m}^{p,q}, with additive
   merging (x = x1 + x2, v = v1 + v2), pairs whose merger leaves the grid lost,
   and the collision kernel
       K(x1, v1; x2, v2) = sum_t coef[t] x1^ax[t] x2^bx[t] v1^av[t] v2^bv[t]
   (n_terms <= 8; give a symmetric K, e.g. both orders of an asymmetric term).
   Every integral uses a Gauss rule of quad_q nodes per coordinate, split
   exactly where a merger crosses a cell edge.  Coefficient layout per cell:
   g_{j,m}^{p,q} at ((j (order_k+1) + p) n_v + m)(order_k+1) + q; n_coef =
   n_x n_v (order_k+1)^2 doubles per cell.  The state is FP64; the contraction
   runs in FP64 or, with arithmetic = 1, in FP32. */
typedef struct {
    int n_x, n_v;              /* bins in mass and in volume (1 .. 256)          */
    int order_k;               /* degree in each coordinate (0 .. 4)              */
    int quad_q;                /* Gauss nodes per coordinate and piece (1 .. 24)  */
    double x_min, x_max, v_min, v_max;
    int n_terms;               /* 1 .. 8                                          */
    double coef[8], ax[8], bx[8], av[8], bv[8];
    int arithmetic;            /* the RHS contraction: 0 FP64, 1 FP32 (CUDA cores;
                                  FP32 factor forms and sums; the state, the stage
                                  combinations of grace_mv_step and L stay FP64)  */
} grace_mv_desc;
typedef struct grace_mv grace_mv;

/* Validates the description and builds, on `device`, the 1-D factor forms of
   every kernel term (the gain forms over pairs of bins in x and in v, the loss
   factors; with arithmetic = 1 also their FP32 copies).  Allocates and
   synchronises.  GRACE_ERR_ARG for a field out of its range (arithmetic other
   than 0 or 1 included); GRACE_ERR_UNSUPPORTED when a cell's coefficient matrix
   (n_x (k+1)) x (n_v (k+1)) does not fit the per-cell stage in shared memory
   (FP32 stages take less). */
GRACE_API grace_status grace_mv_setup(grace_mv **mv, const grace_mv_desc *desc, int device);
/* Stream for the compute calls (the legacy default stream if none). */
GRACE_API grace_status grace_mv_set_stream(grace_mv *mv, void *cuda_stream);
/* L = dg/dt for n_cells independent cells; g and L device arrays of n_cells x
   n_coef doubles (must not overlap).  Asynchronous on the bound stream. */
GRACE_API grace_status grace_mv_rhs(grace_mv *mv, int n_cells, const double *g, double *L);
/* n_steps SSP-RK3 steps (eq. (RK3)) in place on g, dt: device array of n_cells
   step sizes.  No limiter (positivity is the caller's choice of dt).  Allocates
   a workspace of 3 n_cells n_coef doubles on first use or growth (synchronising
   then); otherwise asynchronous. */
GRACE_API grace_status grace_mv_step(grace_mv *mv, int n_cells, double *g, const double *dt, int n_steps);
GRACE_API void grace_mv_destroy(grace_mv *mv);

/* Measures, on `device`, the CUDA-core throughput used as roofline
   denominators: rates[0] FP64 FMA/s, rates[1] FP32 FMA/s, rates[2] FP64->FP32
   conversions/s (3 doubles, host).  Allocates and synchronises. */
GRACE_API grace_status grace_probe_rates(int device, double *rates);

/* Measures, on `device`, the dense tensor-core rate used as the roofline
   denominator of a tensor-core form: tcgen05.mma with M = 128 and N = n
   (a multiple of 16 in [16, 256]) issued back to back by one thread per SM
   from shared-memory operands, kind::tf32 (precision GRACE_TF32, K = 8) or
   kind::f16 with bf16 operands (precision GRACE_BF16X3, one product per
   instruction, K = 16).  *flops_per_s (host) = 2 M N K x instructions / s over
   the whole GPU.  Allocates and synchronises.  GRACE_ERR_TIMEOUT if the
   bounded completion wait gave up. */
GRACE_API grace_status grace_probe_mma(int device, int precision, int n, double *flops_per_s);

GRACE_API void grace_batch_destroy(grace_batch *batch);
GRACE_API void grace_destroy(grace_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GRACE_H */
