"""Seeded synthetic workloads shared by the CUDA path, the tests and the benchmark.

This module holds configuration and random numbers only: group descriptions
(grid, order, physics kinds and parameters), per-cell initial-condition
parameters and random coefficient arrays.  It contains none of the method's
arithmetic (no quadrature, basis functions, fluxes or time stepping), so both
the CUDA library and the independent FP64 oracle can take their inputs from it.

The enumerations below are the interface values accepted by both
implementations (the C header ``include/grace.h`` declares the same numbers).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# collision kernels (Secs. 4.2-4.5)
COAG_NONE, COAG_CONST, COAG_ADD, COAG_MULT, COAG_MAXWELL, COAG_BALLISTIC = 0, 1, 2, 3, 4, 5
FRAG_NONE, FRAG_MULT, FRAG_MAXWELL, FRAG_BALLISTIC = 0, 1, 2, 3
# breakage functions: uniform binary (Sec. 4.4), power law + remnant (eq. break),
# and b = delta(w - u - v), the coagulation special case of eq. (Ffrag)
BREAK_UNIFORM_BINARY, BREAK_POWERLAW_REMNANT, BREAK_COAG_DELTA = 0, 1, 2
# initial conditions projected with eq. (init)
IC_EXP, IC_POWERLAW, IC_FIRST_BIN = 0, 1, 2
# flux truncation (Sec. 3.3): Delta x = -u + x_min, or Delta x = 0
FLUX_CONSERVATIVE, FLUX_NONCONSERVATIVE = 0, 1


@dataclasses.dataclass(frozen=True)
class GroupSpec:
    """One (grid, order, physics) combination; every cell of a group shares it."""
    n_bins: int
    order_k: int
    x_min: float
    x_max: float
    flux_mode: int = FLUX_CONSERVATIVE
    coag_kind: int = COAG_NONE
    coag_p: tuple = ()
    frag_kind: int = FRAG_NONE
    frag_p: tuple = ()
    break_kind: int = BREAK_UNIFORM_BINARY
    break_p: tuple = ()
    cutoff_mode: int = 0
    mfrag_mode: int = 0
    quad_q: int = 0
    limiter: int = 1
    cell_alpha: int = 0     # 1: the ballistic kernels take alpha_turb per cell (non-separable)
    edges: tuple = None     # n_bins + 1 bin edges from x_min to x_max, or None: the log grid

    @property
    def n_coef(self) -> int:
        return self.n_bins * (self.order_k + 1)

    def replace(self, **kw) -> "GroupSpec":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Workload:
    name: str
    spec: GroupSpec
    n_cells: int
    ic_kind: int
    ic_params: np.ndarray      # [n_cells, 4] float64
    dt: np.ndarray             # [n_cells] float64
    n_steps: int
    notes: str = ""


# --------------------------------------------------------------------------
# the paper's test problems (Sec. 4) and the large synthetic batches
# --------------------------------------------------------------------------

def constant_kernel_spec(n_bins=20, order_k=2, flux_mode=FLUX_NONCONSERVATIVE,
                         x_min=1e-4, x_max=1e6) -> GroupSpec:
    """Pure coagulation with K = 1 (Sec. 4.2)."""
    return GroupSpec(n_bins, order_k, x_min, x_max, flux_mode, COAG_CONST, (1.0,))


def single_cell_constant(flux_mode=FLUX_NONCONSERVATIVE) -> Workload:
    """One cell, K = 1, N = 20 over [1e-4, 1e6], k = 2, g0 = x exp(-x),
    SSP-RK3 with dt = 1e-2 to t = 10 (1000 steps)."""
    spec = constant_kernel_spec(20, 2, flux_mode)
    return Workload("single_cell_constant_N20_k2", spec, 1, IC_EXP,
                    np.array([[1.0, 1.0, 0.0, 0.0]]), np.array([1e-2]), 1000)


def shard(wl: Workload, rank: int, world: int) -> Workload:
    """Rank ``rank``'s contiguous share of a workload's cells (weak scaling: the global batch
    is world x the per-rank batch; shares are disjoint and cover it)."""
    if world < 1 or not 0 <= rank < world or wl.n_cells % world:
        raise ValueError("shard: rank outside [0, world) or cells not divisible by world")
    m = wl.n_cells // world
    lo, hi = rank * m, (rank + 1) * m
    return Workload(f"{wl.name}_shard{rank}of{world}", wl.spec, m, wl.ic_kind, wl.ic_params[lo:hi].copy(),
                    wl.dt[lo:hi].copy(), wl.n_steps, wl.notes)


def additive_spec(n_bins=40, order_k=2, x_min=1e-6, x_max=1e10) -> GroupSpec:
    """Pure coagulation with K = x + y (Sec. 4.3), conservative fluxes."""
    return GroupSpec(n_bins, order_k, x_min, x_max, FLUX_CONSERVATIVE, COAG_ADD, (1.0,))


def batched_additive(n_cells=65536, seed=1002, n_bins=40, order_k=2, n_steps=100) -> Workload:
    """Batched coagulation: K = x + y, N = 40 over [1e-6, 1e10], k = 2.
    Per cell g0 = A x exp(-x / x0), A ~ lognormal(0, 0.5), x0 ~ loguniform[1e-3, 1];
    dt_c = 0.02 / M_c with M_c = A x0^2 the cell's total mass, so 100 steps
    reach M_c t = 2."""
    rng = np.random.default_rng(seed)
    A = rng.lognormal(0.0, 0.5, n_cells)
    x0 = np.exp(rng.uniform(math.log(1e-3), math.log(1.0), n_cells))
    ic = np.zeros((n_cells, 4))
    ic[:, 0] = A
    ic[:, 1] = x0
    dt = 0.02 / (A * x0 * x0)
    return Workload(f"batched_additive_{n_cells}cells_N{n_bins}_k{order_k}",
                    additive_spec(n_bins, order_k), n_cells, IC_EXP, ic, dt, n_steps,
                    "A~lognormal(0,0.5), x0~loguniform[1e-3,1], dt=0.02/(A x0^2)")


def pure_fragmentation_spec(n_bins=20, order_k=2, x_min=1e-6, x_max=1e3,
                            flux_mode=FLUX_NONCONSERVATIVE) -> GroupSpec:
    """Pure fragmentation, K_frag = x y with uniform binary breakage (Sec. 4.4)."""
    return GroupSpec(n_bins, order_k, x_min, x_max, flux_mode, COAG_NONE, (),
                     FRAG_MULT, (1.0,), BREAK_UNIFORM_BINARY, ())


def coupled_toy_spec(n_bins=20, order_k=2, flux_mode=FLUX_NONCONSERVATIVE,
                     x_min=1e-6, x_max=1e3, alpha=-1.83) -> GroupSpec:
    """Coupled aggregation-breakage toy model (Sec. 4.5): Maxwellian relative
    velocities with dv_rms = 0.5, v_b = 0.1, v_f = 1; power-law fragments with
    index alpha plus a remnant, m_frag from eq. (mfrag)."""
    return GroupSpec(n_bins, order_k, x_min, x_max, flux_mode,
                     COAG_MAXWELL, (0.5, 0.1), FRAG_MAXWELL, (0.5, 1.0),
                     BREAK_POWERLAW_REMNANT, (alpha,), 0, 0)


def random_coefficients(spec: GroupSpec, n_cells: int, seed: int = 7, rel_modes: float = 0.3,
                        dynamic_range: float = 3.0) -> np.ndarray:
    """Random modal coefficients: positive bin means spanning ``dynamic_range``
    decades per cell, higher modes a uniform fraction of the mean."""
    rng = np.random.default_rng(seed)
    N, k = spec.n_bins, spec.order_k
    g = np.zeros((n_cells, N, k + 1))
    g[:, :, 0] = 10.0 ** rng.uniform(-dynamic_range, 0.0, (n_cells, N))
    if k >= 1:
        g[:, :, 1:] = g[:, :, :1] * rng.uniform(-rel_modes, rel_modes, (n_cells, N, k)) / np.arange(1, k + 1)
    return g.reshape(n_cells, N * (k + 1))


def uneven_batch(n_cells=100000, seed=1004, n_range=(16, 80), orders=(0, 1, 2, 3),
                 kinds=(COAG_CONST, COAG_ADD), x_min=1e-6, x_max=1e10):
    """Uneven batch: per cell N ~ U{n_range}, k ~ U{orders}, kernel kind ~ U{kinds}
    (constant or additive coagulation, conservative fluxes) and a per-cell rate
    scale s ~ lognormal(0, 0.5); ICs as in batched_additive.  A kernel scale s
    multiplies the RHS, which is the same as multiplying the cell's time step,
    so it is folded into dt.  Returns (specs, cell_group, ic_params, dt)."""
    rng = np.random.default_rng(seed)
    N = rng.integers(n_range[0], n_range[1] + 1, n_cells)
    k = rng.choice(np.asarray(orders), n_cells)
    kind = rng.choice(np.asarray(kinds), n_cells)
    s = rng.lognormal(0.0, 0.5, n_cells)
    A = rng.lognormal(0.0, 0.5, n_cells)
    x0 = np.exp(rng.uniform(math.log(1e-3), math.log(1.0), n_cells))
    keys = sorted(set(zip(N.tolist(), k.tolist(), kind.tolist())))
    index = {key: i for i, key in enumerate(keys)}
    specs = [GroupSpec(int(n), int(o), x_min, x_max, FLUX_CONSERVATIVE, int(kd), (1.0,)) for (n, o, kd) in keys]
    group = np.array([index[(a, b, c)] for a, b, c in zip(N.tolist(), k.tolist(), kind.tolist())], dtype=np.int32)
    ic = np.zeros((n_cells, 4))
    ic[:, 0] = A
    ic[:, 1] = x0
    # time scale of the cell's kernel: total mass A x0^2 (additive), number A x0 (constant)
    rate = np.where(kind == COAG_ADD, A * x0 * x0, A * x0) * s
    dt = 0.02 / rate
    return specs, group, ic, dt


# --------------------------------------------------------------------------
# disk workload: coagulation + fragmentation with a per-cell turbulence strength
# --------------------------------------------------------------------------

RHO_S, SIGMA_G, C_S, V_FRAG, RAMP_W = 1.6, 10.0, 5.0e4, 100.0, 0.2


def grain_mass(a_cm):
    """Mass of a compact grain of radius a (cm) with material density 1.6 g/cm^3."""
    return 4.0 * math.pi / 3.0 * RHO_S * a_cm ** 3


def ballistic_params(alpha=1e-3):
    """Ballistic cross section, turbulent relative velocity c_s sqrt(3 alpha St/(1+St^2))
    with St = pi rho_s a / (2 Sigma_g), linear fragmentation ramp over [0.8, 1.2] v_frag."""
    return (RHO_S, SIGMA_G, C_S, alpha, V_FRAG, RAMP_W, 1.0)


def disk_spec(n_bins=60, order_k=2, a_min=1e-4, a_max=1e2, cell_alpha=1, alpha=1e-3):
    """Coagulation + fragmentation with a per-cell alpha_turb: ballistic-turbulent kernels,
    power-law fragments with index -11/6 up to the larger collider mass, plus a remnant
    (m_frag from eq. mfrag), grains of radius a_min..a_max cm on the log grid."""
    p = ballistic_params(alpha)
    return GroupSpec(n_bins, order_k, grain_mass(a_min), grain_mass(a_max), FLUX_CONSERVATIVE,
                     COAG_BALLISTIC, p, FRAG_BALLISTIC, p, BREAK_POWERLAW_REMNANT, (-11.0 / 6.0,),
                     1, 0, 0, 1, cell_alpha)


def disk_batch(n_cells=262144, seed=1003, n_bins=60, order_k=2, rho_dust=1e-12):
    """Disk workload: per cell alpha ~ loguniform[1e-4, 1e-2]; MRN size distribution
    n(a) ~ a^-3.5, i.e. g = x n(x) ~ x^(-5/6), over the first decade of the radius grid and
    zero above, normalised to the dust density rho_dust (g/cm^3).
    Returns (spec, alpha[n_cells], ic_params[n_cells, 4]) for IC_POWERLAW."""
    rng = np.random.default_rng(seed)
    alpha = np.exp(rng.uniform(math.log(1e-4), math.log(1e-2), n_cells))
    spec = disk_spec(n_bins, order_k)
    x0, x1 = spec.x_min, grain_mass(1e-3)
    q = -5.0 / 6.0
    norm = rho_dust * (1.0 + q) / (x1 ** (1.0 + q) - x0 ** (1.0 + q))   # int_x0^x1 norm x^q dx = rho_dust
    ic = np.zeros((n_cells, 4))
    ic[:, 0] = norm
    ic[:, 1] = q
    ic[:, 2] = x0
    ic[:, 3] = x1
    return spec, alpha, ic


# ---------------------------------------------------------------- two dimensions (mass, volume)
@dataclasses.dataclass(frozen=True)
class MVSpec:
    """A two-dimensional (mass x, volume v) grid of Sec. 5.3: n_x x n_v logarithmic bins, degree k in
    each coordinate (tensor-product basis), quad_q quadrature nodes per coordinate, and the collision
    kernel K = sum_t c_t x1^ax_t x2^bx_t v1^av_t v2^bv_t given as terms (c, ax, bx, av, bv)."""
    n_x: int = 6
    n_v: int = 6
    order_k: int = 1
    x_min: float = 1e-2
    x_max: float = 1e2
    v_min: float = 1e-2
    v_max: float = 1e2
    quad_q: int = 4
    terms: tuple = ((1.0, 0.0, 0.0, 0.0, 0.0),)

    @property
    def n_coef(self) -> int:
        return self.n_x * self.n_v * (self.order_k + 1) ** 2


def mv_additive_spec(n_x=6, n_v=6, order_k=1, quad_q=4, x_min=1e-2, x_max=1e2, v_min=1e-2, v_max=1e2) -> MVSpec:
    """K = x1 + x2 (independent of the volume)."""
    return MVSpec(n_x, n_v, order_k, x_min, x_max, v_min, v_max, quad_q,
                  ((1.0, 1.0, 0.0, 0.0, 0.0), (1.0, 0.0, 1.0, 0.0, 0.0)))


def mv_mixed_spec(n_x=6, n_v=6, order_k=1, quad_q=4, x_min=1e-2, x_max=1e2, v_min=1e-2, v_max=1e2) -> MVSpec:
    """A kernel coupling both coordinates: K = 1 + 0.5 (x1 v2 + x2 v1) + 0.25 (v1^(2/3) + v2^(2/3)),
    a constant plus cross terms and a cross-section-like volume term."""
    return MVSpec(n_x, n_v, order_k, x_min, x_max, v_min, v_max, quad_q,
                  ((1.0, 0.0, 0.0, 0.0, 0.0), (0.5, 1.0, 0.0, 0.0, 1.0), (0.5, 0.0, 1.0, 1.0, 0.0),
                   (0.25, 0.0, 0.0, 2.0 / 3.0, 0.0), (0.25, 0.0, 0.0, 0.0, 2.0 / 3.0)))


def mv_random_coefficients(spec: MVSpec, n_cells: int, seed: int = 11, support=None, rel_modes: float = 0.2):
    """Seeded positive-mean random coefficients g_{j,m}^{p,q}, layout [cell][(j,p)][(m,q)]; `support`
    = (jx, jv) keeps only cells j < jx, m < jv (the rest zero)."""
    rng = np.random.default_rng(seed)
    K1 = spec.order_k + 1
    g = np.zeros((n_cells, spec.n_x, K1, spec.n_v, K1))
    g[:, :, 0, :, 0] = rng.uniform(0.2, 1.0, size=(n_cells, spec.n_x, spec.n_v))
    if K1 > 1:
        hi = rng.uniform(-rel_modes, rel_modes, size=(n_cells, spec.n_x, K1, spec.n_v, K1))
        hi[:, :, 0, :, 0] = 0.0
        g += hi * g[:, :, 0:1, :, 0:1]
    if support is not None:
        jx, jv = support
        g[:, jx:, :, :, :] = 0.0
        g[:, :, :, jv:, :] = 0.0
    return g.reshape(n_cells, spec.n_coef)


def mv_batch(n_cells=16384, seed=1005, n_x=12, n_v=12, order_k=1, quad_q=8):
    """The two-dimensional workload: n_cells independent cells of the mixed kernel on 12 x 12 bins over
    four decades in mass and volume, degree 1, 8 quadrature nodes per coordinate, random positive
    coefficients in the lower half of both coordinates (their mergers stay inside the grid), dt 1e-3
    per cell."""
    spec = mv_mixed_spec(n_x, n_v, order_k, quad_q)
    g0 = mv_random_coefficients(spec, n_cells, seed, support=(n_x // 2, n_v // 2))
    return spec, g0, np.full(n_cells, 1e-3)
