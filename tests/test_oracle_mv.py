"""Pins of the two-dimensional (mass x, volume v) oracle of Sec. 5.3 (oracle/grace_oracle_mv.c).

Each pin checks the oracle against something other than itself:
  * conservation: with every merger inside the grid (data in the lower half of both coordinates)
    the total mass sum h_j h_m L_{j,m}^{0,0} vanishes, to round-off once the quadrature has converged
    (gain and loss are evaluated with different split rules, so a wrong weight, norm or cell
    assignment in either breaks it);
  * moment equations in closed form: x and v lie in the test space for k >= 1, so with no merger
    leaving the grid the weak form must give d(int x g)/dt = (int g)^2 for K = 1, = 2 (int g)(int x g)
    for K = x1 + x2, = (int x g)^2 for K = x1 x2, and d(int v g)/dt = (int x g)(int v g) for K = x1 x2
    (the factor 1/2 of the gain, the basis norms and the v-structure all enter);
  * brute force: a Monte Carlo estimate of the four-dimensional gain and loss integrals of every
    coefficient (numpy, log-uniform samples, its own cell search and Legendre values) for a kernel
    coupling both coordinates, within six standard errors;
  * convergence of the Gauss rule with Q (exponential for these smooth integrands).
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as npl

import oracle
from paper_2607_13740_b300 import workloads as W


def _mass_rate(spec, L, o):
    ex, ev = o.edges()
    K1 = spec.order_k + 1
    Lr = L.reshape(-1, spec.n_x, K1, spec.n_v, K1)
    return (np.diff(ex)[None, :, None] * np.diff(ev)[None, None, :] * Lr[:, :, 0, :, 0]).sum(axis=(1, 2))


@pytest.mark.parametrize("make", [W.mv_additive_spec, W.mv_mixed_spec], ids=["additive", "mixed"])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_mass_is_conserved_when_no_merger_leaves_the_grid(make, k):
    spec = make(n_x=4, n_v=4, order_k=k, quad_q=10, x_min=0.1, x_max=10.0, v_min=0.1, v_max=10.0)
    o = oracle.MVOracle(spec)
    g = W.mv_random_coefficients(spec, 2, seed=5 + k, support=(2, 2))
    L = o.rhs(g)
    rate = _mass_rate(spec, L, o)
    m = o.mass(g)
    # the Q = 10 rule on bins of ratio 3.2 integrates the 1/x factors to ~1e-11
    assert np.all(np.abs(rate) <= 1e-9 * m), rate / m
    assert np.abs(L).max() > 1e-3 * np.abs(g).max()      # the operator is not trivially zero


def test_mass_leaves_only_through_the_upper_edges():
    """Data reaching the top bins: mergers beyond x_max or v_max are lost, so the mass rate is
    negative."""
    spec = W.mv_additive_spec(n_x=4, n_v=4, order_k=1, quad_q=8, x_min=0.1, x_max=10.0, v_min=0.1, v_max=10.0)
    o = oracle.MVOracle(spec)
    g = W.mv_random_coefficients(spec, 1, seed=9)
    assert _mass_rate(spec, o.rhs(g), o)[0] < -1e-6 * o.mass(g)[0]


def _moments(spec, o, g):
    """A = int g, B = int x g, C = int v g over the grid, from the coefficients (k >= 1: x and v are
    in the test space; int_j x phi_0 = x_c h, int_j x phi_1 = h^2 / 6)."""
    ex, ev = o.edges()
    K1 = spec.order_k + 1
    gr = g.reshape(-1, spec.n_x, K1, spec.n_v, K1)
    hx, hv = np.diff(ex), np.diff(ev)
    xc, vc = 0.5 * (ex[1:] + ex[:-1]), 0.5 * (ev[1:] + ev[:-1])
    w = hx[None, :, None] * hv[None, None, :]
    A = (w * gr[:, :, 0, :, 0]).sum(axis=(1, 2))
    B = (w * (xc[None, :, None] * gr[:, :, 0, :, 0] + hx[None, :, None] / 6 * gr[:, :, 1, :, 0])).sum(axis=(1, 2))
    C = (w * (vc[None, None, :] * gr[:, :, 0, :, 0] + hv[None, None, :] / 6 * gr[:, :, 0, :, 1])).sum(axis=(1, 2))
    return A, B, C


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("kernel", ["constant", "additive", "product"])
def test_moment_equations_hold_in_closed_form(kernel, k):
    """With no merger leaving the grid, the weak form tested with x and v (exact for k >= 1) gives
    the moment equations of additive merging: for K = 1, dB/dt = A^2; for K = x1 + x2,
    dB/dt = 2 A B; for K = x1 x2, dB/dt = B^2 and dC/dt = B C (A = int g is conserved)."""
    terms = {"constant": ((1.0, 0.0, 0.0, 0.0, 0.0),),
             "additive": ((1.0, 1.0, 0.0, 0.0, 0.0), (1.0, 0.0, 1.0, 0.0, 0.0)),
             "product": ((1.0, 1.0, 1.0, 0.0, 0.0),)}[kernel]
    spec = W.MVSpec(4, 4, k, 0.1, 10.0, 0.1, 10.0, 10, terms)
    o = oracle.MVOracle(spec)
    g = W.mv_random_coefficients(spec, 2, seed=61 + k, support=(2, 2))
    L = o.rhs(g)
    A, B, C = _moments(spec, o, g)
    dA, dB, dC = _moments(spec, o, L)
    assert np.all(np.abs(dA) <= 1e-9 * A)
    want_B = {"constant": A ** 2, "additive": 2 * A * B, "product": B ** 2}[kernel]
    assert np.all(np.abs(dB - want_B) <= 1e-9 * np.abs(want_B)), (dB, want_B)
    if kernel == "product":
        assert np.all(np.abs(dC - B * C) <= 1e-9 * np.abs(B * C)), (dC, B * C)


def _legendre_basis(t, k):
    return np.stack([npl.legval(t, np.eye(k + 1)[p]) for p in range(k + 1)], axis=-1)


def _g_at(spec, G, ex, ev, x, v):
    """g at points (x, v) from coefficients G [(j,p)][(m,q)] (numpy, independent of the oracle)."""
    K1 = spec.order_k + 1
    j = np.clip(np.searchsorted(ex, x, side="right") - 1, 0, spec.n_x - 1)
    m = np.clip(np.searchsorted(ev, v, side="right") - 1, 0, spec.n_v - 1)
    tx = (2 * x - ex[j] - ex[j + 1]) / (ex[j + 1] - ex[j])
    tv = (2 * v - ev[m] - ev[m + 1]) / (ev[m + 1] - ev[m])
    Px, Pv = _legendre_basis(tx, spec.order_k), _legendre_basis(tv, spec.order_k)
    Gr = G.reshape(spec.n_x, K1, spec.n_v, K1)
    C = Gr[j, :, m, :]                                   # [sample, p, q]
    return np.einsum("np,nq,npq->n", Px, Pv, C), j, m, Px, Pv


def test_brute_force_monte_carlo_of_every_coefficient():
    """A kernel coupling mass and volume: Monte Carlo of the gain and loss integrals."""
    spec = W.mv_mixed_spec(n_x=3, n_v=3, order_k=1, quad_q=12, x_min=0.1, x_max=10.0, v_min=0.1, v_max=10.0)
    o = oracle.MVOracle(spec)
    G = W.mv_random_coefficients(spec, 1, seed=33)[0]
    L = o.rhs(G[None])[0]
    ex, ev = o.edges()
    rng = np.random.default_rng(2024)
    n = 2_000_000
    lrx, lrv = np.log(spec.x_max / spec.x_min), np.log(spec.v_max / spec.v_min)
    x1 = spec.x_min * np.exp(lrx * rng.random(n))
    x2 = spec.x_min * np.exp(lrx * rng.random(n))
    v1 = spec.v_min * np.exp(lrv * rng.random(n))
    v2 = spec.v_min * np.exp(lrv * rng.random(n))
    jac = (lrx * lrv) ** 2 * x1 * x2 * v1 * v2          # d x1 dv1 dx2 dv2 of the log-uniform samples
    K = sum(c * x1 ** ax * x2 ** bx * v1 ** av * v2 ** bv for c, ax, bx, av, bv in spec.terms)
    g1, j1, m1, Px1, Pv1 = _g_at(spec, G, ex, ev, x1, v1)
    g2, _, _, _, _ = _g_at(spec, G, ex, ev, x2, v2)
    base = K * (g1 / x1) * (g2 / x2) * jac
    K1 = spec.order_k + 1
    xs, vs = x1 + x2, v1 + v2
    inside = (xs < spec.x_max) & (vs < spec.v_max)
    gj = np.clip(np.searchsorted(ex, xs, side="right") - 1, 0, spec.n_x - 1)
    gm = np.clip(np.searchsorted(ev, vs, side="right") - 1, 0, spec.n_v - 1)
    Pxs = _legendre_basis((2 * xs - ex[gj] - ex[gj + 1]) / (ex[gj + 1] - ex[gj]), spec.order_k)
    Pvs = _legendre_basis((2 * vs - ev[gm] - ev[gm + 1]) / (ev[gm + 1] - ev[gm]), spec.order_k)
    mc = np.zeros((spec.n_x, K1, spec.n_v, K1))
    err = np.zeros_like(mc)
    hx, hv = np.diff(ex), np.diff(ev)
    for j in range(spec.n_x):
        for m in range(spec.n_v):
            for p in range(K1):
                for q in range(K1):
                    norm = (2 * p + 1) * (2 * q + 1) / (hx[j] * hv[m])
                    gain = np.where(inside & (gj == j) & (gm == m), 0.5 * base * xs * Pxs[:, p] * Pvs[:, q], 0.0)
                    loss = np.where((j1 == j) & (m1 == m), base * x1 * Px1[:, p] * Pv1[:, q], 0.0)
                    s = (gain - loss) * norm
                    mc[j, p, m, q] = s.mean()
                    err[j, p, m, q] = s.std() / np.sqrt(n)
    d = np.abs(mc.reshape(-1) - L)
    assert np.all(d <= 6 * err.reshape(-1) + 1e-12 * np.abs(L).max()), (d / err.reshape(-1)).max()
    # and the estimate is informative: its errors are small against the values
    assert np.median(err.reshape(-1) / np.maximum(np.abs(L), 1e-300)) < 0.05


def test_gauss_rule_converges():
    spec_lo = W.mv_mixed_spec(n_x=3, n_v=3, order_k=1, quad_q=6, x_min=0.1, x_max=10.0, v_min=0.1, v_max=10.0)
    spec_hi = W.mv_mixed_spec(n_x=3, n_v=3, order_k=1, quad_q=12, x_min=0.1, x_max=10.0, v_min=0.1, v_max=10.0)
    g = W.mv_random_coefficients(spec_lo, 1, seed=41)
    L6 = oracle.MVOracle(spec_lo).rhs(g)
    L12 = oracle.MVOracle(spec_hi).rhs(g)
    spec_8 = W.mv_mixed_spec(n_x=3, n_v=3, order_k=1, quad_q=8, x_min=0.1, x_max=10.0, v_min=0.1, v_max=10.0)
    L8 = oracle.MVOracle(spec_8).rhs(g)
    s = np.abs(L12).max()
    e6, e8 = np.abs(L6 - L12).max() / s, np.abs(L8 - L12).max() / s
    assert e8 < e6 / 10 and e8 < 1e-6, (e6, e8)


def test_steps_conserve_mass_and_match_the_rhs():
    """SSP-RK3 (eq. (RK3)) of the weak form: mass conserved over steps while no merger can leave the
    grid (data in the lowest bin of each coordinate, three short steps), and one small step moves g
    by dt L to first order."""
    spec = W.mv_additive_spec(n_x=4, n_v=4, order_k=1, quad_q=10, x_min=0.1, x_max=10.0, v_min=0.1, v_max=10.0)
    o = oracle.MVOracle(spec)
    g = W.mv_random_coefficients(spec, 1, seed=51, support=(1, 1))
    m0 = o.mass(g)
    g3 = o.step(g, 1e-3, 3)
    assert np.abs(o.mass(g3) - m0).max() <= 1e-9 * m0.max()
    dt = 1e-4
    g1 = o.step(g, dt, 1)
    L = o.rhs(g)
    assert np.abs(g1 - g - dt * L).max() <= 1e-3 * dt * np.abs(L).max()
