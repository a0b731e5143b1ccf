/*
 * Derivative build of the GRACE-DG oracle (test infrastructure only; the same rules as
 * grace_oracle.c apply: only the tests may load it).
 *
 * This file compiles grace_oracle.c a second time, as C++, with its scalar type `real` a
 * forward-mode dual number (orc_dual.h).  Every function of the oracle's path (kernels,
 * breakage mass functions, nested flux quadrature, App. B terms, eq. evo, the scaling limiter,
 * SSP-RK3) then returns, next to its value, the exact derivative of its own arithmetic with
 * respect to one seeded input: a direction in the initial state, or one physics parameter.
 * It gives the adjoint tests an exact FP64 gradient (no finite-difference step):
 *   d g(T) / d theta    and    (d g(T) / d g0) gdot.
 * The values it returns equal the plain oracle's bit for bit (the value part runs the same
 * operations in the same order).
 */
#include "orc_dual.h"

typedef dual real;
#define RV(x) ((x).v)
#define REAL_IS_ZERO(x) ((x).v == 0.0 && (x).d == 0.0)
#define ORC_API static
#define ORC_TANGENT 1

#include "grace_oracle.c"

#include <vector>

/* Parameter ids as the CUDA library's grace_param_grad_setup: 0..7 coag_p[i], 8..15 frag_p[i-8],
   16..23 break_p[i-16]; -1 seeds no parameter. */
static int seed_param(octx *c, int id)
{
    if (id < -1 || id >= 24) return -1;
    if (id < 0) return 0;
    if (id < 8) c->coag_p[id].d = 1.0;
    else if (id < 16) c->frag_p[id - 8].d = 1.0;
    else c->break_p[id - 16].d = 1.0;
    ctx_betas(c);   /* the Maxwellian probabilities depend on coag_p / frag_p */
    return 0;
}

/* L[g] and its derivative Ldot along gdot (may be NULL: zero) and along parameter param_id. */
extern "C" int orc_tangent_rhs(const orc_params *p, int n_cells, const double *g, const double *gdot, int param_id,
                               double *L, double *Ldot)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    if (seed_param(&c, param_id)) { ctx_free(&c); return -1; }
    const int P = c.P;
    #pragma omp parallel
    {
        std::vector<dual> gd(P), Ld(P);
        #pragma omp for schedule(dynamic, 1)
        for (int cell = 0; cell < n_cells; ++cell) {
            for (int i = 0; i < P; ++i)
                gd[i] = dual(g[(size_t)cell * P + i], gdot ? gdot[(size_t)cell * P + i] : 0.0);
            rhs_one(&c, gd.data(), Ld.data(), NULL);
            for (int i = 0; i < P; ++i) {
                L[(size_t)cell * P + i] = Ld[i].v;
                Ldot[(size_t)cell * P + i] = Ld[i].d;
            }
        }
    }
    ctx_free(&c);
    return 0;
}

/* n_steps of step_one (limiter + SSP-RK3) from g; g_out = g(T), gdot_out = its derivative along
   gdot (may be NULL) and parameter param_id. */
extern "C" int orc_tangent_step(const orc_params *p, int n_cells, const double *g, const double *gdot,
                                int param_id, const double *dt, int n_steps, double *g_out, double *gdot_out)
{
    octx c;
    if (ctx_init(&c, p)) return -1;
    if (seed_param(&c, param_id)) { ctx_free(&c); return -1; }
    const int P = c.P;
    #pragma omp parallel
    {
        std::vector<dual> gd(P), work(3 * (size_t)P);
        #pragma omp for schedule(dynamic, 1)
        for (int cell = 0; cell < n_cells; ++cell) {
            for (int i = 0; i < P; ++i)
                gd[i] = dual(g[(size_t)cell * P + i], gdot ? gdot[(size_t)cell * P + i] : 0.0);
            for (int s = 0; s < n_steps; ++s) step_one(&c, gd.data(), dt[cell], work.data());
            for (int i = 0; i < P; ++i) {
                g_out[(size_t)cell * P + i] = gd[i].v;
                gdot_out[(size_t)cell * P + i] = gd[i].d;
            }
        }
    }
    ctx_free(&c);
    return 0;
}
