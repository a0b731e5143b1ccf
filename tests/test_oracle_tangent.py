"""Pins for the oracle's forward-mode derivative build (the oracle compiled on dual numbers).

It supplies the exact FP64 gradients the adjoint tests compare with, so it is pinned to what the
mathematics fixes, independently of its own dual arithmetic: its values are the plain oracle's bit
for bit; the state derivative of the quadratic L is the polarization identity; the derivative with
respect to a parameter that scales a kernel linearly is L over that parameter; every other
parameter derivative, and the derivative of whole limited SSP-RK3 trajectories, agrees with a
central difference of the plain oracle to the difference's own truncation and rounding error."""
import numpy as np
import pytest

import oracle
from paper_2607_13740_b300 import workloads as W

TOY = W.coupled_toy_spec(8, 2, flux_mode=0, x_min=1e-3, x_max=1e4)
TOY_CUT = TOY.replace(cutoff_mode=1)
# alpha_turb = 5e-6 puts the fragmentation ramp inside the grid (both kernels and the ramp active)
BALLISTIC = W.disk_spec(n_bins=8, order_k=2, cell_alpha=0, alpha=5e-6)


def _fd(spec, name, i, h, fn):
    """Central difference of fn(spec) in parameter name[i] with step h."""
    vals = list(getattr(spec, name))
    vp, vm = list(vals), list(vals)
    vp[i] += h
    vm[i] -= h
    return (fn(spec.replace(**{name: tuple(vp)})) - fn(spec.replace(**{name: tuple(vm)}))) / (2 * h)


def test_tangent_values_equal_the_oracle():
    o = oracle.Oracle(TOY)
    g = W.random_coefficients(TOY, 6, seed=90)
    L, _ = o.rhs(g)
    Lt, _ = o.tangent_rhs(g, np.ones_like(g), param_id=9)
    np.testing.assert_array_equal(Lt, L)
    gT, _, _ = o.step(g, 0.01, 5)
    gTt, _ = o.tangent_step(g, 0.01, 5, gdot=np.ones_like(g), param_id=16)
    np.testing.assert_array_equal(gTt, gT)


@pytest.mark.parametrize("spec", [W.additive_spec(10, 2, 1e-3, 1e4), TOY, TOY_CUT, BALLISTIC],
                         ids=["add", "toy", "toy_cut", "ballistic"])
def test_state_derivative_is_the_polarization_identity(spec):
    """L is a quadratic form of g, so J(g) v = (L(g + v) - L(g - v)) / 2 exactly."""
    o = oracle.Oracle(spec)
    g = W.random_coefficients(spec, 5, seed=91)
    v = W.random_coefficients(spec, 5, seed=92) * np.random.default_rng(93).uniform(-1, 1, g.shape)
    _, dL = o.tangent_rhs(g, v)
    Lp, Sp = o.rhs(g + v)
    Lm, Sm = o.rhs(g - v)
    ref = 0.5 * (Lp - Lm)
    assert np.all(np.abs(dL - ref) <= 1e-12 * (Sp + Sm))


@pytest.mark.parametrize("spec,pid", [
    (W.additive_spec(10, 2, 1e-3, 1e4).replace(coag_p=(2.5,)), 0),
    (W.pure_fragmentation_spec(8, 2, 1e-3, 1e4, flux_mode=0).replace(frag_p=(0.7,)), 8),
], ids=["coag_scale", "frag_scale"])
def test_linear_parameter_derivative_is_L_over_the_parameter(spec, pid):
    o = oracle.Oracle(spec)
    g = W.random_coefficients(spec, 5, seed=94)
    L, S = o.rhs(g)
    _, dL = o.tangent_rhs(g, param_id=pid)
    theta = (spec.coag_p if pid < 8 else spec.frag_p)[pid % 8]
    assert np.all(np.abs(dL - L / theta) <= 1e-13 * S / theta)


@pytest.mark.parametrize("spec,name,i,pid", [
    (TOY, "frag_p", 1, 9),       # v_frag in the Maxwellian fragmentation probability
    (TOY, "frag_p", 0, 8),       # dv_rms: kernel scale and probability
    (TOY, "coag_p", 1, 1),       # v_bounce
    (TOY, "break_p", 0, 16),     # the fragment power-law index alpha (eqs. break, inte1, inte2, App. B)
    (TOY_CUT, "break_p", 0, 16),
    (BALLISTIC, "frag_p", 3, 11),   # alpha_turb in the fragmentation kernel (and its ramp)
    (BALLISTIC, "frag_p", 4, 12),   # v_frag: the ramp's edges
    (BALLISTIC, "coag_p", 0, 0),    # material density in the coagulation kernel
    (BALLISTIC, "break_p", 0, 16),  # fragment index over 18 decades of mass
], ids=["toy_vfrag", "toy_dvrms", "toy_vb", "toy_alpha", "cut_alpha", "ball_alphaturb", "ball_vfrag",
        "ball_rho", "ball_alpha"])
def test_parameter_derivative_matches_central_difference(spec, name, i, pid):
    """Central difference with a relative step of 1e-6: rounding ~ 1e-16 S / 1e-6 and truncation
    O(h^2) (the index derivative over 18 decades carries log(x)^2 ~ 1e3, so 1e-9 relative), both
    below the bar 1e-7 of the term scale over the parameter."""
    o = oracle.Oracle(spec)
    g = W.random_coefficients(spec, 4, seed=95)
    _, dL = o.tangent_rhs(g, param_id=pid)
    h = 1e-6 * abs(getattr(spec, name)[i])
    fd = _fd(spec, name, i, h, lambda s: oracle.Oracle(s).rhs(g)[0])
    _, S = o.rhs(g)
    theta = abs(getattr(spec, name)[i])
    bar = 1e-7 * S / theta
    assert np.all(np.abs(dL - fd) <= bar), np.max(np.abs(dL - fd) / bar)
    assert np.max(np.abs(dL) / bar) > 1e3      # the derivative is far above the bar somewhere


@pytest.mark.parametrize("pid,name,i", [(-1, None, None), (9, "frag_p", 1), (16, "break_p", 0)],
                         ids=["state", "vfrag", "alpha"])
def test_trajectory_derivative_matches_central_difference(pid, name, i):
    """10 limited SSP-RK3 steps of the coupled toy: the derivative of g(T) along a direction of g0
    (pid = -1) or a parameter against a central difference of the plain oracle's trajectory."""
    spec = TOY
    o = oracle.Oracle(spec)
    g0 = W.random_coefficients(spec, 3, seed=96, rel_modes=0.9)
    dt = 0.01
    _, fl = o.limit(g0)
    assert np.all(fl & 2)                       # the limiter acts on these states
    if pid < 0:
        v = W.random_coefficients(spec, 3, seed=97)
        _, dg = o.tangent_step(g0, dt, 10, gdot=v)
        h = 1e-6
        fd = (o.step(g0 + h * v, dt, 10)[0] - o.step(g0 - h * v, dt, 10)[0]) / (2 * h)
    else:
        _, dg = o.tangent_step(g0, dt, 10, param_id=pid)
        h = 1e-5 * abs(getattr(spec, name)[i])
        fd = _fd(spec, name, i, h, lambda s: oracle.Oracle(s).step(g0, dt, 10)[0])
    scale = np.abs(dg).max(axis=1, keepdims=True)
    assert np.all(np.abs(dg - fd) <= 1e-6 * scale), np.max(np.abs(dg - fd) / scale)


def test_trajectory_derivative_with_a_vanishing_tail():
    """A projected state whose top bins hold ~1e-189 (limited, with means far below any other
    bin): every derivative stays finite (quotients are differentiated without squaring a tiny
    denominator) and matches the central difference."""
    spec = TOY.replace(x_min=1e-6, x_max=1e3, n_bins=10)
    o = oracle.Oracle(spec)
    g0 = o.project(W.IC_EXP, [[1.0, 0.3, 0, 0]])
    assert g0.reshape(10, 3)[-1, 0] < 1e-150
    v = np.random.default_rng(98).uniform(-0.1, 0.1, size=g0.shape) * g0
    _, dg = o.tangent_step(g0, 0.05, 10, gdot=v)
    assert np.all(np.isfinite(dg))
    h = 1e-5
    fd = (o.step(g0 + h * v, 0.05, 10)[0] - o.step(g0 - h * v, 0.05, 10)[0]) / (2 * h)
    assert np.all(np.abs(dg - fd) <= 1e-6 * np.abs(dg).max())
