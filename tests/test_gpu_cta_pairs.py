"""CTA pairs (cta_group::2) for the tensor-core contraction.

On CTA pairs one tcgen05.mma with M = 256 covers the even CTA's 128 cells and the odd CTA's 128
cells, each CTA loading half of every table block.  grace_set_cta_pairs selects them for every
forward contraction (mode 1), never (0, the default), or for multi-group launches only (2).  Both
launch forms are compared with the FP64 oracle at the tolerances of the tensor forms, on batches
with an even and an odd number of cell tiles (the last pair then has no odd tile), ragged last
tiles, several degrees, the full 65,536-cell batch sampled and uneven multi-group batches; and with
each other.  A timed-out pair launch (no table copies, bounded waits) reports the failure and
leaves the context usable.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_RHS = {grace.TF32: 2e-3, grace.BF16X3: 5e-5}
FORMS = [grace.TF32, grace.BF16X3]
IDS = ["tf32", "bf16x3"]
RANGE_FLOOR = 1e-24

SPECS = {
    "add_N40_k2": W.additive_spec(40, 2),
    "k0": W.additive_spec(20, 0, 1e-3, 1e5),
    "k4": W.GroupSpec(12, 4, 1e-2, 1e4, 0, W.COAG_ADD, (1.0,)),
    "pure_frag": W.pure_fragmentation_spec(10, 2, 1e-6, 1e3),
    "toy_remnant": W.coupled_toy_spec(10, 2, flux_mode=0),
}


@pytest.fixture(autouse=True)
def _restore_pairs():
    yield
    grace.set_cta_pairs(grace.CTA_PAIRS_NEVER)


def _scaled(L, Lo, S):
    floor = RANGE_FLOOR * S.max(axis=1, keepdims=True)
    den = np.maximum(np.maximum(np.abs(Lo), S), floor)
    d = np.abs(L - Lo)
    return np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))


def _rhs(b, g, form, pairs):
    grace.set_cta_pairs(grace.CTA_PAIRS_ALWAYS if pairs else grace.CTA_PAIRS_NEVER)
    L = b.rhs(g, precision=form).cpu().numpy()
    assert b.device_error() == 0
    return L


@pytest.mark.parametrize("form", FORMS, ids=IDS)
@pytest.mark.parametrize("name", sorted(SPECS))
@pytest.mark.parametrize("n", [256, 300, 640, 700])
def test_pairs_match_oracle_and_single_ctas(name, form, n):
    spec = SPECS[name]
    g_np = W.random_coefficients(spec, n, seed=811 + n)
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(n)
    g = torch.as_tensor(g_np, device=DEV)
    Lp = _rhs(b, g, form, True)
    Ls = _rhs(b, g, form, False)
    Lo, S = oracle.Oracle(spec).rhs(g_np)
    assert np.isfinite(Lp).all()
    ep, es = _scaled(Lp, Lo, S).max(), _scaled(Ls, Lo, S).max()
    assert ep <= TOL_RHS[form], f"pairs {ep:.3e}"
    assert es <= TOL_RHS[form], f"single {es:.3e}"
    # the same tiles in the same order: the two launches agree far inside the form's tolerance
    assert _scaled(Lp, Ls, S).max() <= TOL_RHS[form] / 10


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_pairs_full_size_odd_tile_count_sampled(form):
    """65,664 cells: 513 cell tiles (the last pair without an odd tile), every SM pair busy."""
    wl = W.batched_additive(n_cells=65664)
    ctx = grace.Context([wl.spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(wl.n_cells)
    g = b.project(wl.ic_kind, wl.ic_params)
    grace.set_cta_pairs(grace.CTA_PAIRS_ALWAYS)
    L = b.rhs(g, precision=form)
    assert b.device_error() == 0
    sample = np.array([0, 127, 128, 255, 256, 33000, 65535, 65536, 65600, 65663])
    Lo, S = oracle.Oracle(wl.spec).rhs(g[sample].cpu().numpy())
    assert _scaled(L[sample].cpu().numpy(), Lo, S).max() <= TOL_RHS[form]


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_pairs_trajectory_matches_single_ctas(form):
    """20 SSP-RK3 steps of 1,000 cells: pairs and single CTAs stay within the form's bar."""
    wl = W.batched_additive(n_cells=1000)
    ctx = grace.Context([wl.spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(wl.n_cells)
    dt = torch.as_tensor(wl.dt, device=DEV)
    out = []
    for pairs in (grace.CTA_PAIRS_ALWAYS, grace.CTA_PAIRS_NEVER):
        grace.set_cta_pairs(pairs)
        g = b.project(wl.ic_kind, wl.ic_params)
        b.step(g, dt, 20, precision=form)
        assert b.device_error() == 0
        out.append(g.cpu().numpy())
    m = np.abs(b.mass(torch.as_tensor(out[1], device=DEV)).cpu().numpy())
    h = np.diff(oracle.Oracle(wl.spec).edges())
    d = np.abs(out[0] - out[1]).reshape(wl.n_cells, 40, 3)
    l1 = (h[None, :] * d.sum(axis=2)).sum(axis=1) / m
    assert l1.max() <= {grace.TF32: 1e-4, grace.BF16X3: 2e-6}[form], l1.max()


@pytest.mark.parametrize("pairs", [grace.CTA_PAIRS_ALWAYS, grace.CTA_PAIRS_NEVER], ids=["pairs", "single"])
def test_bounded_wait_timeout_both_launch_forms(pairs):
    spec = W.additive_spec(12, 2, 1e-3, 1e4)
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, grace.BF16X3))
    n = 640
    b = ctx.batch(n)
    g = torch.as_tensor(W.random_coefficients(spec, n, seed=43), device=DEV)
    grace.set_cta_pairs(pairs)
    grace.arm_wait_timeout(2_000_000)
    b.rhs(g, grace.BF16X3)
    assert b.device_error() != 0
    assert b.device_error() == 0
    L = b.rhs(g, grace.BF16X3).cpu().numpy()
    assert b.device_error() == 0
    Lo, S = oracle.Oracle(spec).rhs(g.cpu().numpy())
    assert _scaled(L, Lo, S).max() <= TOL_RHS[grace.BF16X3]




@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_multi_group_pairs_match_oracle_and_single_ctas(form):
    """Uneven batch (groups of one to several cell tiles, odd tile counts): three grouped SSP-RK3
    steps (one multi-group contraction per stage) on CTA pairs against the oracle per cell, and
    against the same steps on single CTAs."""
    specs, group, ic, dt = W.uneven_batch(1200, seed=1109, n_range=(16, 60), orders=(0, 1, 2, 3))
    ctx = grace.Context(specs, 0, precisions=(grace.FP64, form))
    b = ctx.batch(len(group), group)
    b.set_grouped(True)
    off = b.offsets()
    g0 = b.project(W.IC_EXP, ic)
    dtt = torch.as_tensor(dt, device=DEV)
    # trajectory bar: each RHS coefficient is within TOL_RHS of the oracle's scale, and dt is at
    # most half the positivity bound (dt |L| <= g / 2), so one step moves at most TOL_RHS / 2 of the
    # cell's mass away from the oracle; three steps 1.5 TOL_RHS
    n_steps = 3
    out = {}
    for mode in (grace.CTA_PAIRS_MULTI, grace.CTA_PAIRS_NEVER):
        grace.set_cta_pairs(mode)
        g = g0.clone()
        b.step(g, dtt, n_steps, form)
        assert b.device_error() == 0
        out[mode] = g.cpu().numpy()
    gin = g0.cpu().numpy()
    bar = 0.5 * n_steps * TOL_RHS[form]
    for gi, spec in enumerate(specs):
        idx = np.where(group == gi)[0]
        if idx.size == 0:
            continue
        o = oracle.Oracle(spec)
        go, mo, _ = o.step(np.stack([gin[off[c]:off[c + 1]] for c in idx]), dt[idx], n_steps)
        h = np.diff(o.edges())
        for mode, lim in ((grace.CTA_PAIRS_MULTI, bar), (grace.CTA_PAIRS_NEVER, bar)):
            d = np.abs(np.stack([out[mode][off[c]:off[c + 1]] for c in idx]) - go)
            l1 = (h * d.reshape(idx.size, spec.n_bins, -1).sum(axis=2)).sum(axis=1) / np.abs(mo)
            assert l1.max() <= lim, (gi, mode, l1.max())
        d = np.abs(np.stack([out[grace.CTA_PAIRS_MULTI][off[c]:off[c + 1]] - out[grace.CTA_PAIRS_NEVER][off[c]:off[c + 1]]
                             for c in idx]))
        l1 = (h * d.reshape(idx.size, spec.n_bins, -1).sum(axis=2)).sum(axis=1) / np.abs(mo)
        assert l1.max() <= bar / 10, (gi, l1.max())
