"""Pins for the oracle's whole scheme: conservation, limiter, time stepping and
convergence to the paper's analytic solutions."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npl

import oracle
from paper_2607_13740_b300 import workloads as W
import analytic as A

SPECS = {
    "const": W.constant_kernel_spec(10, 2, W.FLUX_CONSERVATIVE, 1e-3, 1e4),
    "add": W.additive_spec(10, 2, 1e-3, 1e4),
    "frag": W.pure_fragmentation_spec(10, 2, 1e-3, 1e4, flux_mode=0),
    "toy": W.coupled_toy_spec(10, 2, flux_mode=0, x_min=1e-3, x_max=1e4),
    "toy_k3_cut1": W.coupled_toy_spec(8, 3, flux_mode=0, x_min=1e-3, x_max=1e4).replace(cutoff_mode=1),
    "toy_k1": W.coupled_toy_spec(8, 1, flux_mode=0, x_min=1e-3, x_max=1e4),
}


@pytest.mark.parametrize("name", sorted(SPECS))
def test_conservative_rhs_conserves_mass(name):
    """Sec. 5.1 / eq. (g0): with Delta x = -u + x_min, sum_j h_j L_j^0 telescopes to
    F(x_min) - F(x_max) = 0."""
    spec = SPECS[name]
    o = oracle.Oracle(spec)
    h = np.diff(o.edges())
    g = W.random_coefficients(spec, 4, seed=21)
    L, S = o.rhs(g)
    k = spec.order_k
    L0 = L.reshape(4, spec.n_bins, k + 1)[:, :, 0]
    dm = (h * L0).sum(axis=1)
    assert np.all(np.abs(dm) <= 1e-14 * np.abs(h * L0).sum(axis=1))
    assert np.all(S >= np.abs(L) * (1 - 1e-12))


def test_nonconservative_mass_loss_equals_boundary_flux():
    """With Delta x = 0: sum_j h_j L_j^0 = F(x_{-1/2}) - F(x_{N-1/2}) = -F(x_max)."""
    spec = W.additive_spec(8, 2, 1e-3, 1e2).replace(flux_mode=1)
    o = oracle.Oracle(spec)
    h = np.diff(o.edges())
    g = W.random_coefficients(spec, 1, seed=22)
    L, _ = o.rhs(g)
    L0 = L.reshape(spec.n_bins, 3)[:, 0]
    F, _ = o.flux_point(g[0], [spec.x_max], 3)
    assert abs((h * L0).sum() + F[0]) < 1e-13 * abs(F[0])


def test_rhs_is_a_quadratic_form():
    """L[g] is homogeneous of degree two in the coefficients (eqs. evo, Fcoagtrun)."""
    spec = SPECS["toy"]
    o = oracle.Oracle(spec)
    g = W.random_coefficients(spec, 1, seed=23)
    L1, S1 = o.rhs(g)
    L2, _ = o.rhs(3.0 * g)
    assert np.all(np.abs(L2 - 9.0 * L1) <= 1e-13 * 9.0 * S1)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_bin_minimum_matches_dense_sampling(k):
    """The analytic minimum of sum_i g^i phi_i on [-1, 1] used by eq. (gamma)."""
    rng = np.random.default_rng(30 + k)
    xs = np.linspace(-1, 1, 200001)
    for _ in range(200):
        c = rng.normal(size=k + 1)
        ref = npl.legval(xs, c).min()
        m = oracle.bin_min(c, k)
        assert m <= ref + 1e-12
        assert m >= ref - 1e-8 * (1 + abs(ref))


def test_scaling_limiter_properties():
    """eqs. (recon), (gamma), (average): keeps g^0, makes every bin non-negative, and leaves
    non-negative polynomials untouched."""
    spec = W.GroupSpec(50, 3, 1e-2, 1e2)
    rng = np.random.default_rng(40)
    g = np.zeros((3, 50, 4))
    g[:, :, 0] = rng.uniform(0.0, 1.0, (3, 50))
    g[:, :, 1:] = g[:, :, :1] * rng.uniform(-1.5, 1.5, (3, 50, 3))
    g[0, :5, 1:] = 0.0
    g[0, 5, 0] = 0.0
    o = oracle.Oracle(spec)
    gl, flags = o.limit(g.reshape(3, -1))
    gl = gl.reshape(3, 50, 4)
    np.testing.assert_array_equal(gl[:, :, 0], g[:, :, 0])
    xs = np.linspace(-1, 1, 4001)
    for c in range(3):
        for j in range(50):
            vals = npl.legval(xs, gl[c, j])
            assert vals.min() >= -1e-13 * max(1.0, g[c, j, 0])
            if npl.legval(xs, g[c, j]).min() > 1e-12:
                np.testing.assert_array_equal(gl[c, j], g[c, j])
    assert np.all(flags & 2)


def test_constant_kernel_converges_at_order_k_plus_1():
    """Sec. 4.2: convergence to eq. (fcoagsolution); EOC (eq. eoc) approaches k + 1."""
    t_end, dt = 2.0, 1e-2
    eoc = {}
    for k in (0, 1, 2):
        errs = []
        for N in (10, 20, 40):
            spec = W.constant_kernel_spec(N, k, W.FLUX_NONCONSERVATIVE, 1e-4, 1e6)
            o = oracle.Oracle(spec)
            g0 = o.project(W.IC_EXP, [1.0, 1.0, 0, 0])
            g, m, f = o.step(g0, dt, int(round(t_end / dt)), threads=4)
            errs.append(A.e_c(g[0], o.edges(), k, lambda x: A.g_constant(x, t_end)))
        eoc[k] = np.log(errs[1] / errs[2]) / np.log(2)
        assert errs[2] < errs[1] < errs[0]
    assert eoc[0] > 0.8 and eoc[1] > 1.8 and eoc[2] > 2.6


def test_golovin_additive_kernel_solution():
    """Additive kernel K = x + y with f0 = exp(-x) against the textbook Golovin solution.
    With the paper's Q = k + 1 the error is limited by the flux quadrature (it still
    decreases with N); with more Gauss points it reaches the DG order."""
    t_end, dt = 1.0, 1e-2
    errs = {}
    for N in (20, 40):
        for Q in (0, 6):
            spec = W.GroupSpec(N, 2, 1e-4, 1e4, W.FLUX_NONCONSERVATIVE, W.COAG_ADD, (1.0,), quad_q=Q)
            o = oracle.Oracle(spec)
            g0 = o.project(W.IC_EXP, [1.0, 1.0, 0, 0])
            g, _, _ = o.step(g0, dt, int(round(t_end / dt)), threads=4)
            errs[(N, Q)] = A.e_c(g[0], o.edges(), 2, lambda x: A.g_golovin(x, t_end))
    assert errs[(40, 0)] < 1e-2 and errs[(40, 0)] < errs[(20, 0)] / 2
    assert errs[(40, 6)] < 2.5e-3 and errs[(40, 6)] < errs[(20, 6)] / 6


def test_pure_fragmentation_solution():
    """Sec. 4.4: multiplicative fragmentation kernel, uniform binary breakage,
    convergence to eq. (fragsolution)."""
    t_end, dt = 2.0, 1e-2
    errs = []
    for N in (10, 20):
        spec = W.pure_fragmentation_spec(N, 2, 1e-6, 1e3)
        o = oracle.Oracle(spec)
        g0 = o.project(W.IC_EXP, [1.0, 1.0, 0, 0])
        g, _, _ = o.step(g0, dt, int(round(t_end / dt)), threads=4)
        errs.append(A.e_c(g[0], o.edges(), 2, lambda x: A.g_pure_frag(x, t_end)))
    assert errs[1] < 6e-2 and errs[1] < errs[0] / 2.5


def test_ssp_rk3_is_third_order_in_time():
    """eq. (RK3): halving dt reduces the time error by ~8."""
    spec = W.constant_kernel_spec(8, 1, W.FLUX_CONSERVATIVE, 1e-2, 1e3).replace(limiter=0)
    o = oracle.Oracle(spec)
    g0 = o.project(W.IC_EXP, [1.0, 1.0, 0, 0])
    T = 1.0
    ref, _, _ = o.step(g0, T / 512, 512)
    errs = []
    for n in (8, 16, 32):
        g, _, _ = o.step(g0, T / n, n)
        errs.append(np.abs(g - ref).max())
    p1, p2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 2.7 < p1 < 3.4 and 2.7 < p2 < 3.4


def test_step_conserves_mass_and_batches_independently():
    """Conservative fluxes keep M_1 = sum_j h_j g_j^0 (Sec. 4.1) to round-off over a
    trajectory; cells of a batch evolve independently."""
    wl = W.batched_additive(n_cells=6, n_bins=12, order_k=2, n_steps=20)
    o = oracle.Oracle(wl.spec)
    g0 = o.project(wl.ic_kind, wl.ic_params)
    m0 = o.mass(g0)
    g, m, f = o.step(g0, wl.dt, wl.n_steps)
    np.testing.assert_allclose(m, m0, rtol=1e-13)
    g3, _, _ = o.step(g0[3:4], wl.dt[3:4], wl.n_steps)
    np.testing.assert_array_equal(g3[0], g[3])


def test_cfl_flag_follows_eq_dt():
    """eq. (dt): a stage whose forward-Euler update would take a mean negative has broken
    the bound (flag bit 8 set whenever bit 1 is, for non-negative stage inputs); a step far
    below the bound sets no flag, although empty tail bins receive influx; a zero state has
    no flux and sets none; a dt above the first stage's bound min over bins losing mass of
    g_j^0 / |L_j^0| sets it."""
    spec = SPECS["add"]
    o = oracle.Oracle(spec)
    k = spec.order_k
    g = o.project(W.IC_EXP, [[1.0, 1.0, 0, 0]] * 3)
    _, _, f = o.step(g, 1e-9, 1)
    assert np.all((f & 9) == 0)
    _, _, f = o.step(np.zeros_like(g), 10.0, 1)
    assert np.all((f & 9) == 0)
    L, _ = o.rhs(g[:1])
    L0 = L.reshape(spec.n_bins, k + 1)[:, 0]
    g0 = g[0].reshape(spec.n_bins, k + 1)[:, 0]
    out = L0 < 0
    bound = (g0[out] / -L0[out]).min()
    _, _, f = o.step(g[:1], 1.01 * bound, 1)
    assert f[0] & 8
    for dt in (0.3 * bound, 3.0 * bound, 30.0 * bound):
        _, _, f = o.step(g, dt, 2)
        assert np.all((f & 1) == 0) or np.all(f[(f & 1) != 0] & 8)
    _, _, f = o.step(g[:1], 30.0 * bound, 1)
    assert f[0] & 1 and f[0] & 8


def test_mass_drift_bit():
    """eq. (g0): a conservative group keeps M_1 to round-off while eq. (dt) holds, so a normal
    call sets no drift bit (16); a non-conservative group loses mass through x_max by design and
    is not tested; a call whose state overflows is flagged non-finite (4) and not tested for
    drift."""
    spec = SPECS["add"]
    o = oracle.Oracle(spec)
    g = o.project(W.IC_EXP, [[1.0, 1.0, 0, 0]] * 2)
    _, _, f = o.step(g, 1e-3, 5)
    assert np.all((f & 16) == 0)
    _, _, f = o.step(g, 1e300, 3)
    assert np.all(f & 4) and np.all((f & 16) == 0)
    nc = W.additive_spec(8, 2, 1e-3, 1e2).replace(flux_mode=1)
    onc = oracle.Oracle(nc)
    gnc = onc.project(W.IC_EXP, [[1.0, 1.0, 0, 0]])
    m0 = onc.mass(gnc)[0]
    _, m, f = onc.step(gnc, 0.05, 20)
    assert abs(m[0] - m0) > 1e-6 * m0 and (f[0] & 16) == 0


def test_mass_drift_stays_below_the_rounding_bound():
    """eq. (g0) telescopes exactly, so with eq. (dt) kept the only change of M_1 is the
    rounding of the stage updates: at most (27.1 n + 2 N) u M_1 for n steps (u = 2^-53; the
    bound the drift bit's tolerance rests on).  Checked over 60 steps of cells whose mass moves
    across many bins, against the bound and against the bit's tolerance 32 u n (floor 1e-10)."""
    wl = W.batched_additive(n_cells=8, n_bins=16, order_k=2, n_steps=60)
    o = oracle.Oracle(wl.spec)
    g0 = o.project(wl.ic_kind, wl.ic_params)
    m0 = o.mass(g0)
    g, m, f = o.step(g0, wl.dt, wl.n_steps)
    assert np.all((f & (1 | 4 | 8 | 16)) == 0)
    u = 2.0 ** -53
    drift = np.abs(m - m0) / m0
    assert np.all(drift <= (27.1 * wl.n_steps + 2 * wl.spec.n_bins) * u)
    assert oracle.drift_tol(1) == 1e-10 and oracle.drift_tol(10 ** 6) == 32 * u * 10 ** 6
    assert np.all(drift <= oracle.drift_tol(wl.n_steps))


def test_mass_drift_bit_positive_case():
    """A planted non-conservative update (each step adds leak * M_1 to bin 0, a mistake put in
    the oracle for this test only) sets the drift bit (16) once the change over the call exceeds
    the tolerance, and not below it; cells that broke eq. (dt) (bit 8) are not tested."""
    spec = SPECS["add"]
    o = oracle.Oracle(spec)
    g = o.project(W.IC_EXP, [[1.0, 1.0, 0, 0], [2.0, 0.3, 0, 0]])
    try:
        oracle.plant_mass_leak(1e-9)
        _, _, f = o.step(g, 1e-3, 3)
        assert np.all(f & 16)
        oracle.plant_mass_leak(1e-12)
        _, _, f = o.step(g, 1e-3, 3)
        assert np.all((f & 16) == 0)
        oracle.plant_mass_leak(1e-6)
        L, _ = o.rhs(g[:1])
        L0 = L.reshape(spec.n_bins, -1)[:, 0]
        g0 = g[0].reshape(spec.n_bins, -1)[:, 0]
        bound = (g0[L0 < 0] / -L0[L0 < 0]).min()
        _, _, f = o.step(g[:1], 30.0 * bound, 1)
        assert f[0] & 8 and (f[0] & 16) == 0
    finally:
        oracle.plant_mass_leak(0.0)
    _, _, f = o.step(g, 1e-3, 3)
    assert np.all((f & 16) == 0)


def test_substep_counts_follow_the_positivity_bound():
    """Sec. 5.2 coupling: the sub-step count of a cell is the smallest n with dt_hydro / n <= cfl B,
    B the eq. (dt) bound.  Pinned by what the bound means: a forward-Euler update of the state with
    step B takes the limiting bin's mean exactly to zero and keeps every other mean >= 0, and the
    count falls by one when dt_hydro shrinks just below (n - 1) cfl B."""
    spec = SPECS["add"]
    o = oracle.Oracle(spec)
    g = o.project(W.IC_EXP, [[1.0, 1.0, 0, 0], [3.0, 0.2, 0, 0]])
    L, _ = o.rhs(g)
    K1 = spec.order_k + 1
    for c in range(2):
        m, L0 = g[c].reshape(-1, K1)[:, 0], L[c].reshape(-1, K1)[:, 0]
        # the count for dt_hydro = 1: find B from the counts at growing dt, without retyping the formula
        n1 = o.substep_counts(g[c:c + 1], 1.0, 0.5)[0]
        assert n1 >= 1
        # bracket B: the largest dt with a single sub-step at cfl = 1
        lo, hi = 0.0, 1.0
        while o.substep_counts(g[c:c + 1], hi, 1.0)[0] == 1:
            hi *= 2.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if o.substep_counts(g[c:c + 1], mid, 1.0)[0] == 1:
                lo = mid
            else:
                hi = mid
        B = lo
        euler = m + B * L0
        assert euler.min() >= -1e-12 * m.max()
        assert np.isclose(np.abs(euler[L0 < 0]).min(), 0.0, atol=1e-12 * m.max())
        n = o.substep_counts(g[c:c + 1], 7.3 * B, 0.5)[0]
        assert n == 15
        assert o.substep_counts(g[c:c + 1], 6.999 * B, 0.5)[0] == 14
