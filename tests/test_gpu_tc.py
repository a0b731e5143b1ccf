"""Parity of the tcgen05 tensor-core forms (TF32 and split BF16 x3) with the FP64 oracle.

Stated tolerances (relative to the oracle's rounding scale S of each RHS
coefficient, and for trajectories to the cell's mass M_1):
  TF32:    |L - L_oracle| <= 2e-3 S,  trajectory L1 <= 1e-3 M_1
  BF16X3:  |L - L_oracle| <= 5e-5 S,  trajectory L1 <= 2e-5 M_1
The tensor operands carry FP32's exponent range, so coefficients whose scale
is far below the cell's largest one (tail bins of exp(-x/x0) profiles, 1e-40
and smaller) are compared against a floor of 1e-24 times the cell's largest
scale instead of their own.  Mass is conserved to FP64 round-off in every form
(the i = 0 row only sees flux differences, summed in FP64).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_RHS = {grace.TF32: 2e-3, grace.BF16X3: 5e-5}
TOL_L1 = {grace.TF32: 1e-3, grace.BF16X3: 2e-5}
RANGE_FLOOR = 1e-24
FORMS = [grace.TF32, grace.BF16X3]
IDS = ["tf32", "bf16x3"]

SPECS = {
    "add_N40_k2": W.additive_spec(40, 2),
    "const_noncons_k1": W.constant_kernel_spec(16, 1, W.FLUX_NONCONSERVATIVE, 1e-4, 1e6),
    "k0": W.additive_spec(20, 0, 1e-3, 1e5),
    "k3": W.GroupSpec(12, 3, 1e-2, 1e4, 0, W.COAG_ADD, (1.0,)),
    "k4": W.GroupSpec(12, 4, 1e-2, 1e4, 0, W.COAG_ADD, (1.0,)),
    "pure_frag": W.pure_fragmentation_spec(10, 2, 1e-6, 1e3),
    "toy_remnant": W.coupled_toy_spec(10, 2, flux_mode=0),
}


def _ctx(spec):
    return grace.Context([spec], 0, precisions=(grace.FP64, grace.TF32, grace.BF16X3))


def _scaled(L, Lo, S):
    floor = RANGE_FLOOR * S.max(axis=1, keepdims=True)
    den = np.maximum(np.maximum(np.abs(Lo), S), floor)
    d = np.abs(L - Lo)
    return np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))


@pytest.mark.parametrize("form", FORMS, ids=IDS)
@pytest.mark.parametrize("name", sorted(SPECS))
def test_rhs_parity_tensor_core(name, form):
    spec = SPECS[name]
    n = 300    # three 128-cell tiles, the last one ragged
    g = W.random_coefficients(spec, n, seed=301)
    ctx = _ctx(spec)
    b = ctx.batch(n)
    L = b.rhs(torch.as_tensor(g, device=DEV), precision=form).cpu().numpy()
    assert b.device_error() == 0
    Lo, S = oracle.Oracle(spec).rhs(g)
    err = _scaled(L, Lo, S)
    assert np.isfinite(L).all()
    assert err.max() <= TOL_RHS[form], f"{name}: {err.max():.3e}"
    # mass: sum_j h_j L_j^0 telescopes to zero in FP64 (conservative fluxes)
    if spec.flux_mode == W.FLUX_CONSERVATIVE:
        h = np.diff(oracle.Oracle(spec).edges())
        L0 = L.reshape(n, spec.n_bins, spec.order_k + 1)[:, :, 0]
        assert np.all(np.abs((h * L0).sum(axis=1)) <= 1e-14 * np.abs(h * L0).sum(axis=1))


@pytest.mark.parametrize("form", FORMS, ids=IDS)
@pytest.mark.parametrize("n", [1, 127, 129, 700])
def test_small_and_ragged_batches(form, n):
    spec = SPECS["add_N40_k2"]
    g = W.random_coefficients(spec, n, seed=302)
    ctx = _ctx(spec)
    b = ctx.batch(n)
    L = b.rhs(torch.as_tensor(g, device=DEV), precision=form).cpu().numpy()
    assert b.device_error() == 0
    Lo, S = oracle.Oracle(spec).rhs(g)
    assert _scaled(L, Lo, S).max() <= TOL_RHS[form]


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_batched_additive_trajectory(form):
    """100 SSP-RK3 steps of the batched additive workload at 256 cells."""
    wl = W.batched_additive(n_cells=256)
    ctx = _ctx(wl.spec)
    b = ctx.batch(wl.n_cells)
    g = b.project(wl.ic_kind, wl.ic_params)
    g0 = g.cpu().numpy()
    m0 = b.mass(g).cpu().numpy()
    dt = torch.as_tensor(wl.dt, device=DEV)
    mass = torch.zeros(wl.n_cells, dtype=torch.float64, device=DEV)
    b.step(g, dt, wl.n_steps, precision=form, mass=mass)
    assert b.device_error() == 0
    m = mass.cpu().numpy()
    assert np.all(np.abs(m - m0) <= 1e-13 * np.abs(m0))
    o = oracle.Oracle(wl.spec)
    sample = np.arange(0, 256, 8)
    go, _, _ = o.step(g0[sample], wl.dt[sample], wl.n_steps)
    h = np.diff(o.edges())
    d = np.abs(g.cpu().numpy()[sample] - go).reshape(len(sample), 40, 3)
    l1 = (h[None, :] * d.sum(axis=2)).sum(axis=1) / np.abs(m0[sample])
    assert l1.max() <= TOL_L1[form], l1.max()


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_full_size_batch_sampled(form):
    """65,536 cells (512 tiles over every SM, several tiles per CTA)."""
    wl = W.batched_additive()
    ctx = _ctx(wl.spec)
    b = ctx.batch(wl.n_cells)
    g = b.project(wl.ic_kind, wl.ic_params)
    L = b.rhs(g, precision=form)
    assert b.device_error() == 0
    sample = np.array([0, 1, 127, 128, 18943, 18944, 40000, 65535])
    Lo, S = oracle.Oracle(wl.spec).rhs(g[sample].cpu().numpy())
    assert _scaled(L[sample].cpu().numpy(), Lo, S).max() <= TOL_RHS[form]


def test_forms_agree_with_fp64_gpu_path():
    """Reduced-precision forms against the FP64 GPU path on the same batch (all cells)."""
    spec = SPECS["add_N40_k2"]
    g = torch.as_tensor(W.random_coefficients(spec, 1000, seed=303), device=DEV)
    ctx = _ctx(spec)
    b = ctx.batch(1000)
    L64 = b.rhs(g, precision=grace.FP64)
    for form in FORMS:
        L = b.rhs(g, precision=form)
        rel = ((L - L64).abs().amax(dim=1) / L64.abs().amax(dim=1)).max().item()
        assert rel <= 50 * TOL_RHS[form], (form, rel)


@pytest.mark.parametrize("form", [grace.FP64] + FORMS, ids=["fp64"] + IDS)
def test_cfl_status_bit_against_oracle(form):
    """eq. (dt) status bit on 300 cells (two tiles and a ragged tail): cells stepped at a tenth
    of the first stage's bound keep it clear, cells at ten times the bound set it, as the
    oracle does.  FP64 compares every status bit; the tensor forms compare the eq. (dt) and
    negative-mean bits (their limiter decision is FP32)."""
    n = 300
    wl = W.batched_additive(n_cells=n)
    ctx = _ctx(wl.spec)
    b = ctx.batch(n)
    g = b.project(wl.ic_kind, wl.ic_params)
    g0 = g.cpu().numpy()
    o = oracle.Oracle(wl.spec)
    L, _ = o.rhs(g0, threads=8)
    K1 = wl.spec.order_k + 1
    L0 = L.reshape(n, -1, K1)[:, :, 0]
    m0 = g0.reshape(n, -1, K1)[:, :, 0]
    bound = np.where(L0 < 0, m0 / np.where(L0 < 0, -L0, 1.0), np.inf).min(axis=1)
    dt = np.where(np.arange(n) % 2 == 1, 10.0, 0.1) * bound
    flags = torch.zeros(n, dtype=torch.uint8, device=DEV)
    b.step(g, torch.as_tensor(dt, device=DEV), 1, precision=form, flags=flags)
    assert b.device_error() == 0
    _, _, fo = o.step(g0, dt, 1, threads=8)
    f = flags.cpu().numpy()
    assert np.all(fo[1::2] & grace.FLAG_CFL) and not np.any(fo[::2] & grace.FLAG_CFL)
    mask = 0xFF if form == grace.FP64 else grace.FLAG_CFL | grace.FLAG_NEGATIVE_MEAN
    np.testing.assert_array_equal(f & mask, fo & mask)


@pytest.mark.parametrize("form", [grace.FP64, grace.BF16X3], ids=["fp64", "bf16x3"])
def test_mass_drift_bit_and_flags_check(form):
    """Mass-drift bit (16) as the oracle sets it: clear on cells the conservative scheme keeps
    (M_1 conserved to round-off) and not tested on cells whose dt overflows the state (flagged
    non-finite, 4); grace_flags_check returns the OR of the flags and the WARN_CELLS status."""
    n = 300
    wl = W.batched_additive(n_cells=n)
    ctx = _ctx(wl.spec)
    b = ctx.batch(n)
    g = b.project(wl.ic_kind, wl.ic_params)
    g0 = g.cpu().numpy()
    dt = wl.dt.copy()
    dt[::7] = 1e300
    flags = torch.zeros(n, dtype=torch.uint8, device=DEV)
    b.step(g, torch.as_tensor(dt, device=DEV), 2, precision=form, flags=flags)
    f = flags.cpu().numpy()
    _, _, fo = oracle.Oracle(wl.spec).step(g0, dt, 2, threads=8)
    assert np.all(fo[::7] & 4) and not np.any(fo & 16)
    np.testing.assert_array_equal(f & 20, fo & 20)
    any_bits = b.flags_check(flags)
    assert any_bits == int(np.bitwise_or.reduce(f))
    clear = torch.zeros(n, dtype=torch.uint8, device=DEV)
    assert b.flags_check(clear) == 0
