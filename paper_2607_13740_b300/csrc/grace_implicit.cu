// Linearly implicit (Rosenbrock-Euler) step for stiff cells, the implicit option of the
// operator-split coupling to a hydrodynamics code (Sec. 5.2):
//     (I - dt_c J(g)) k = dt_c L[g],   g <- g + k,   J = dL/dg at the step's start,
// one linear system of P unknowns per cell.  Each is solved by restarted GMRES(m) (Saad & Schultz's
// generalised minimal residual method: Arnoldi with modified Gram-Schmidt, Givens rotations on the
// Hessenberg matrix, the small least-squares problem solved at the end of every cycle) whose
// matrix-vector products are grace_rhs_jvp's: one JVP launch over the whole batch per Krylov
// iteration, then one warp per cell for the orthogonalisation.  Cells converge on their own: a cell
// whose residual fell below rtol of its initial residual takes no further basis vectors.
#include <algorithm>
#include <cmath>
#include <string>

#include "grace_internal.h"

namespace grace {

namespace {

struct ImplicitWs {
    int n = 0, P = 0, m = 0;
    double *L = nullptr;      // [n][P] L[g]
    double *k = nullptr;      // [n][P] solution increment
    double *V = nullptr;      // [m + 1][n][P] Krylov basis
    double *w = nullptr;      // [n][P] JVP output
    double *H = nullptr;      // [n][m + 1][m] Hessenberg matrix (rotated to upper triangular)
    double *cs = nullptr, *sn = nullptr;   // [n][m] Givens rotations
    double *s = nullptr;      // [n][m + 1] rotated right-hand side of the least-squares problem
    double *beta0 = nullptr;  // [n] initial residual norm of the step
    int *ncol = nullptr;      // [n] basis vectors taken in the current cycle
    int *active = nullptr;    // [n] 1 while the cell iterates
    int *n_active = nullptr;  // device counter of active cells
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// r = dt L - (k - dt J k) with J k in w (first cycle: k = 0, w unused), beta = ||r||, v_0 = r / beta,
// s = (beta, 0, ...); a cell whose residual is already below rtol beta0 stops
__global__ void cycle_start_kernel(int n, int P, int m, const double *__restrict__ dt, const double *__restrict__ L,
                                   const double *__restrict__ k, const double *__restrict__ w, int first, double rtol,
                                   double *__restrict__ V0, double *__restrict__ s, double *__restrict__ beta0,
                                   int *__restrict__ ncol, int *__restrict__ active, int *__restrict__ n_active)
{
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (cell >= n) return;
    const double d = dt[cell];
    const size_t o = (size_t)cell * P;
    double ss = 0.0;
    for (int q = lane; q < P; q += 32) {
        const double r = first ? d * L[o + q] : d * L[o + q] - (k[o + q] - d * w[o + q]);
        V0[o + q] = r;
        ss += r * r;
    }
    const double beta = sqrt(warp_sum(ss));
    if (first && lane == 0) beta0[cell] = beta;
    const double b0 = first ? beta : beta0[cell];
    const bool go = beta > rtol * b0 && beta > 0.0;
    const double inv = go ? 1.0 / beta : 0.0;
    for (int q = lane; q < P; q += 32) V0[o + q] *= inv;
    if (lane == 0) {
        for (int i = 0; i <= m; ++i) s[(size_t)cell * (m + 1) + i] = i == 0 ? beta : 0.0;
        ncol[cell] = 0;
        active[cell] = go ? 1 : 0;
        if (go) atomicAdd(n_active, 1);
    }
}

// one Arnoldi step for column j: w <- v_j - dt J v_j (J v_j in w), modified Gram-Schmidt against
// v_0..v_j, v_{j+1} = w / ||w||, the previous rotations and a new one applied to column j, and the
// residual |s_{j+1}| compared with rtol beta0
__global__ void arnoldi_kernel(int n, int P, int m, int j, const double *__restrict__ dt, double *__restrict__ V,
                               const double *__restrict__ w, double *__restrict__ H, double *__restrict__ cs,
                               double *__restrict__ sn, double *__restrict__ s, const double *__restrict__ beta0,
                               double rtol, int *__restrict__ ncol, int *__restrict__ active, int *__restrict__ n_active)
{
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (cell >= n || !active[cell]) return;
    const double d = dt[cell];
    const size_t o = (size_t)cell * P, vs = (size_t)n * P;
    double *vj1 = V + (size_t)(j + 1) * vs + o;
    const double *vj = V + (size_t)j * vs + o;
    for (int q = lane; q < P; q += 32) vj1[q] = vj[q] - d * w[o + q];
    __syncwarp();
    double *h = H + (size_t)cell * (m + 1) * m;   // h[i * m + j]
    for (int i = 0; i <= j; ++i) {
        const double *vi = V + (size_t)i * vs + o;
        double dot = 0.0;
        for (int q = lane; q < P; q += 32) dot += vj1[q] * vi[q];
        dot = warp_sum(dot);
        for (int q = lane; q < P; q += 32) vj1[q] -= dot * vi[q];
        __syncwarp();
        if (lane == 0) h[i * m + j] = dot;
    }
    double ss = 0.0;
    for (int q = lane; q < P; q += 32) ss += vj1[q] * vj1[q];
    const double hn = sqrt(warp_sum(ss));
    const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int q = lane; q < P; q += 32) vj1[q] *= inv;
    if (lane == 0) {
        h[(j + 1) * m + j] = hn;
        double *c = cs + (size_t)cell * m, *sv = sn + (size_t)cell * m, *sr = s + (size_t)cell * (m + 1);
        for (int i = 0; i < j; ++i) {   // earlier rotations
            const double a = h[i * m + j], b = h[(i + 1) * m + j];
            h[i * m + j] = c[i] * a + sv[i] * b;
            h[(i + 1) * m + j] = -sv[i] * a + c[i] * b;
        }
        const double a = h[j * m + j], b = h[(j + 1) * m + j];
        const double r = hypot(a, b);
        const double cj = r > 0.0 ? a / r : 1.0, sj = r > 0.0 ? b / r : 0.0;
        c[j] = cj;
        sv[j] = sj;
        h[j * m + j] = r;
        h[(j + 1) * m + j] = 0.0;
        sr[j + 1] = -sj * sr[j];
        sr[j] = cj * sr[j];
        ncol[cell] = j + 1;
        // converged, breakdown (the Krylov space is invariant) or the cycle is full
        if (fabs(sr[j + 1]) <= rtol * beta0[cell] || hn == 0.0 || j + 1 == m) {
            active[cell] = 0;
            atomicSub(n_active, 1);
        }
    }
}

// y = H^-1 s over the cell's ncol columns (back substitution), k += V y
__global__ void update_solution_kernel(int n, int P, int m, const double *__restrict__ V, const double *__restrict__ H,
                                       const double *__restrict__ s, const int *__restrict__ ncol, double *__restrict__ k)
{
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (cell >= n) return;
    const int nc = ncol[cell];
    if (nc == 0) return;
    double y[64];   // m <= 64
    const double *h = H + (size_t)cell * (m + 1) * m;
    const double *sr = s + (size_t)cell * (m + 1);
    for (int i = nc - 1; i >= 0; --i) {
        double t = sr[i];
        for (int c = i + 1; c < nc; ++c) t -= h[i * m + c] * y[c];
        y[i] = h[i * m + i] != 0.0 ? t / h[i * m + i] : 0.0;
    }
    const size_t o = (size_t)cell * P, vs = (size_t)n * P;
    for (int q = lane; q < P; q += 32) {
        double acc = k[o + q];
        for (int i = 0; i < nc; ++i) acc += y[i] * V[(size_t)i * vs + o + q];
        k[o + q] = acc;
    }
}

__global__ void add_kernel(long long n, const double *__restrict__ k, double *__restrict__ g)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) g[i] += k[i];
}

void free_implicit_ws(ImplicitWs *w)
{
    if (!w) return;
    cudaFree(w->L);
    cudaFree(w->k);
    cudaFree(w->V);
    cudaFree(w->w);
    cudaFree(w->H);
    cudaFree(w->cs);
    cudaFree(w->sn);
    cudaFree(w->s);
    cudaFree(w->beta0);
    cudaFree(w->ncol);
    cudaFree(w->active);
    cudaFree(w->n_active);
    delete w;
}

}  // namespace

void free_implicit(grace_batch *b)
{
    free_implicit_ws(static_cast<ImplicitWs *>(b->implicit));
    b->implicit = nullptr;
}

static grace_status implicit_ws(grace_batch *b, int P, int m, ImplicitWs **out)
{
    ImplicitWs *w = static_cast<ImplicitWs *>(b->implicit);
    const int n = b->n_cells;
    if (w && w->n == n && w->P == P && w->m >= m) {
        *out = w;
        return GRACE_OK;
    }
    free_implicit(b);
    w = new ImplicitWs();
    w->n = n;
    w->P = P;
    w->m = m;
    const size_t nP = (size_t)n * P;
    cudaError_t e = cudaMalloc(&w->L, nP * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->k, nP * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->V, (size_t)(m + 1) * nP * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->w, nP * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->H, (size_t)n * (m + 1) * m * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->cs, (size_t)n * m * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->sn, (size_t)n * m * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->s, (size_t)n * (m + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->beta0, (size_t)n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->ncol, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&w->active, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&w->n_active, sizeof(int));
    b->implicit = w;
    if (e != cudaSuccess) {
        free_implicit(b);
        return cuda_fail(e, "grace_rosenbrock_step: workspace");
    }
    *out = w;
    return GRACE_OK;
}

}  // namespace grace

using namespace grace;

extern "C" grace_status grace_rosenbrock_step(grace_batch *b, double *g, const double *dt, int precision,
                                              int krylov_dim, int max_restarts, double rtol, int *iterations)
{
    if (!b || !g || !dt || krylov_dim < 1 || krylov_dim > 64 || max_restarts < 0 || !(rtol > 0.0) || !(rtol < 1.0)) {
        set_error("grace_rosenbrock_step: null argument, krylov_dim outside [1, 64], max_restarts < 0 or rtol "
                  "outside (0, 1)");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    const int P = b->ctx->groups[b->parts[0].group].dg.P, n = b->n_cells, m = krylov_dim;
    ImplicitWs *w = nullptr;
    grace_status s = implicit_ws(b, P, m, &w);
    if (s != GRACE_OK) return s;
    cudaStream_t st = b->ctx->stream;
    // L[g] of the step's start (the same call a user makes; it checks the batch and the precision)
    s = grace_rhs(b, g, w->L, precision);
    if (s != GRACE_OK) return s;
    cudaError_t e = cudaMemsetAsync(w->k, 0, (size_t)n * P * sizeof(double), st);
    const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
    int total_iters = 0;
    for (int cycle = 0; cycle <= max_restarts && e == cudaSuccess; ++cycle) {
        if (cycle > 0) {
            s = grace_rhs_jvp(b, g, w->k, w->w, precision);   // J k for the restarted residual
            if (s != GRACE_OK) return s;
        }
        e = cudaMemsetAsync(w->n_active, 0, sizeof(int), st);
        if (e == cudaSuccess) {
            cycle_start_kernel<<<blocks, 256, 0, st>>>(n, P, m, dt, w->L, w->k, w->w, cycle == 0 ? 1 : 0, rtol, w->V, w->s,
                                                      w->beta0, w->ncol, w->active, w->n_active);
            e = cudaGetLastError();
        }
        int n_active = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&n_active, w->n_active, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess || n_active == 0) break;
        for (int j = 0; j < m && e == cudaSuccess; ++j) {
            const double *vj = w->V + (size_t)j * n * P;
            s = grace_rhs_jvp(b, g, vj, w->w, precision);
            if (s != GRACE_OK) return s;
            arnoldi_kernel<<<blocks, 256, 0, st>>>(n, P, m, j, dt, w->V, w->w, w->H, w->cs, w->sn, w->s, w->beta0, rtol,
                                                  w->ncol, w->active, w->n_active);
            e = cudaGetLastError();
            ++total_iters;
            // every few iterations: stop the cycle once every cell has converged
            if (e == cudaSuccess && (j % 4 == 3 || j + 1 == m)) {
                e = cudaMemcpyAsync(&n_active, w->n_active, sizeof(int), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e == cudaSuccess && n_active == 0) break;
            }
        }
        if (e == cudaSuccess) {
            update_solution_kernel<<<blocks, 256, 0, st>>>(n, P, m, w->V, w->H, w->s, w->ncol, w->k);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        const long long nP = (long long)n * P;
        add_kernel<<<(unsigned)((nP + 255) / 256), 256, 0, st>>>(nP, w->k, g);
        e = cudaGetLastError();
    }
    if (iterations) *iterations = total_iters;
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_rosenbrock_step");
}
