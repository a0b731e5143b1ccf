"""The A-in-tensor-memory form of the tensor-core contraction.

grace_set_tc_a_in_tmem(1) keeps the cells' A tile of single-group forward contractions in tensor
memory (tcgen05.cp from a ring slot into TMEM, tcgen05.mma reading A from TMEM, tiles of N <= 192, a
three-deep ring of table copies); 0, the default, keeps A in shared memory.  Both forms are compared with the FP64
oracle at the tolerances of the tensor forms and with each other, over degrees 0..4 (k = 3, 4 with
more than 128 coefficients keep A in shared memory), ragged and single-tile batches, the full
65,536-cell batch sampled and a trajectory; a timed-out launch of the form reports the failure and
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
    "k1_N64": W.additive_spec(64, 1, 1e-4, 1e6),
    "k3": W.GroupSpec(12, 3, 1e-2, 1e4, 0, W.COAG_ADD, (1.0,)),
    "k4_N40": W.GroupSpec(40, 4, 1e-3, 1e6, 0, W.COAG_ADD, (1.0,)),
    "pure_frag": W.pure_fragmentation_spec(10, 2, 1e-6, 1e3),
    "toy_remnant": W.coupled_toy_spec(10, 2, flux_mode=0),
}


@pytest.fixture(autouse=True)
def _restore():
    yield
    grace.set_tc_a_in_tmem(False)


def _scaled(L, Lo, S):
    floor = RANGE_FLOOR * S.max(axis=1, keepdims=True)
    den = np.maximum(np.maximum(np.abs(Lo), S), floor)
    d = np.abs(L - Lo)
    return np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))


def _rhs(b, g, form, at):
    grace.set_tc_a_in_tmem(at)
    L = b.rhs(g, precision=form).cpu().numpy()
    assert b.device_error() == 0
    return L


@pytest.mark.parametrize("form", FORMS, ids=IDS)
@pytest.mark.parametrize("name", sorted(SPECS))
@pytest.mark.parametrize("n", [1, 300, 700])
def test_a_in_tmem_matches_oracle_and_shared_memory_form(name, form, n):
    spec = SPECS[name]
    g_np = W.random_coefficients(spec, n, seed=907 + n)
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(n)
    g = torch.as_tensor(g_np, device=DEV)
    La = _rhs(b, g, form, True)
    Ls = _rhs(b, g, form, False)
    Lo, S = oracle.Oracle(spec).rhs(g_np)
    assert np.isfinite(La).all()
    ea, es = _scaled(La, Lo, S).max(), _scaled(Ls, Lo, S).max()
    assert ea <= TOL_RHS[form], f"A in TMEM {ea:.3e}"
    assert es <= TOL_RHS[form], f"A in shared memory {es:.3e}"
    # different tile shapes (N <= 192 against N <= 256) sum in a different order: the two forms
    # agree within the form's tolerance, far inside it in practice
    assert _scaled(La, Ls, S).max() <= TOL_RHS[form] / 4


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_a_in_tmem_full_size_sampled(form):
    """65,536 cells: 512 cell tiles over every SM, several work items per CTA."""
    wl = W.batched_additive()
    ctx = grace.Context([wl.spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(wl.n_cells)
    g = b.project(wl.ic_kind, wl.ic_params)
    grace.set_tc_a_in_tmem(True)
    L = b.rhs(g, precision=form)
    assert b.device_error() == 0
    sample = np.array([0, 1, 127, 128, 18943, 18944, 40000, 65535])
    Lo, S = oracle.Oracle(wl.spec).rhs(g[sample].cpu().numpy())
    assert _scaled(L[sample].cpu().numpy(), Lo, S).max() <= TOL_RHS[form]


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_a_in_tmem_trajectory_matches_oracle(form):
    """100 SSP-RK3 steps of the batched additive workload at 256 cells (the trajectory bars of the
    tensor forms), mass conserved to round-off."""
    wl = W.batched_additive(n_cells=256)
    ctx = grace.Context([wl.spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(wl.n_cells)
    grace.set_tc_a_in_tmem(True)
    g = b.project(wl.ic_kind, wl.ic_params)
    g0 = g.cpu().numpy()
    m0 = b.mass(g).cpu().numpy()
    mass = torch.zeros(wl.n_cells, dtype=torch.float64, device=DEV)
    b.step(g, torch.as_tensor(wl.dt, device=DEV), wl.n_steps, precision=form, mass=mass)
    assert b.device_error() == 0
    assert np.all(np.abs(mass.cpu().numpy() - m0) <= 1e-13 * np.abs(m0))
    o = oracle.Oracle(wl.spec)
    sample = np.arange(0, 256, 8)
    go, _, _ = o.step(g0[sample], wl.dt[sample], wl.n_steps)
    h = np.diff(o.edges())
    d = np.abs(g.cpu().numpy()[sample] - go).reshape(len(sample), 40, 3)
    l1 = (h[None, :] * d.sum(axis=2)).sum(axis=1) / np.abs(m0[sample])
    assert l1.max() <= {grace.TF32: 1e-3, grace.BF16X3: 2e-5}[form], l1.max()


def test_a_in_tmem_tile_plan_is_narrower():
    """The form's tiles are at most 192 wide; the tile report follows the selected form."""
    spec = SPECS["add_N40_k2"]
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, grace.BF16X3))
    grace.set_tc_a_in_tmem(True)
    ta = ctx.tile_info(0, grace.BF16X3)
    grace.set_tc_a_in_tmem(False)
    ts = ctx.tile_info(0, grace.BF16X3)
    assert ta["max_n"] <= 192 < ts["max_n"] <= 256
    assert ta["nnz_fold"] == ts["nnz_fold"]


def test_a_in_tmem_bounded_wait_timeout():
    spec = W.additive_spec(12, 2, 1e-3, 1e4)
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, grace.BF16X3))
    n = 640
    b = ctx.batch(n)
    g = torch.as_tensor(W.random_coefficients(spec, n, seed=47), device=DEV)
    grace.set_tc_a_in_tmem(True)
    grace.arm_wait_timeout(2_000_000)
    b.rhs(g, grace.BF16X3)
    assert b.device_error() != 0
    assert b.device_error() == 0
    L = b.rhs(g, grace.BF16X3).cpu().numpy()
    assert b.device_error() == 0
    Lo, S = oracle.Oracle(spec).rhs(g.cpu().numpy())
    assert _scaled(L, Lo, S).max() <= TOL_RHS[grace.BF16X3]
