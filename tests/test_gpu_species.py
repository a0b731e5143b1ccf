"""Species of mixed grains (Sec. 5.3): grace_rhs_species / grace_step_species against the oracle's
bilinear species rates L[g_s; g] (the species in the outer-collider slot, the total g in the
partner's) and its species SSP-RK3 steps with the per-species limiter.  FP64 bars: the RHS within
1e-12 of the rounding scale, trajectories within 1e-12 in the mass-weighted L1 norm of the cell."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SPECS = {
    "add": W.additive_spec(10, 2, 1e-3, 1e4),
    "toy": W.coupled_toy_spec(8, 2, flux_mode=0, x_min=1e-3, x_max=1e4),
    "frag": W.pure_fragmentation_spec(8, 1, 1e-3, 1e4, flux_mode=0),
    "k3": W.additive_spec(12, 3, 1e-3, 1e4),
}


def _split(spec, g, S, seed):
    """S partial densities that add up to g: per-bin random shares of every coefficient of the bin,
    the last species taking the remainder."""
    n = g.shape[0]
    w = np.random.default_rng(seed).uniform(0.05, 1.0, (S, n, spec.n_bins, 1))
    w /= w.sum(axis=0, keepdims=True)
    gs = (g.reshape(n, spec.n_bins, -1)[None] * w).reshape(S, n, -1)
    gs[-1] = g - gs[:-1].sum(axis=0)
    return gs


@pytest.mark.parametrize("S", [1, 2, 3, 4])
@pytest.mark.parametrize("name", list(SPECS))
def test_species_rhs_matches_oracle(name, S):
    """300 cells (ten 32-cell warps and a ragged tail)."""
    spec = SPECS[name]
    o = oracle.Oracle(spec)
    g = W.random_coefficients(spec, 300, seed=81)
    gs = _split(spec, g, S, seed=82 + S)
    Lo, So = o.rhs_species(gs)
    b = grace.Context([spec]).batch(300)
    Lg = b.rhs_species(torch.as_tensor(gs, device=DEV)).cpu().numpy()
    err = np.abs(Lg - Lo) / np.maximum(So, 1e-300)
    assert err.max() <= 1e-12, err.max()


def test_species_rates_add_up_to_the_single_species_rhs():
    """Linear in the outer slot: sum_s L_s = L[g] of grace_rhs on the total."""
    spec = SPECS["toy"]
    g = W.random_coefficients(spec, 200, seed=83)
    gs = _split(spec, g, 3, seed=84)
    b = grace.Context([spec]).batch(200)
    Ls = b.rhs_species(torch.as_tensor(gs, device=DEV)).sum(dim=0)
    L = b.rhs(torch.as_tensor(g, device=DEV))
    _, So = oracle.Oracle(spec).rhs(g)
    assert (np.abs((Ls - L).cpu().numpy()) / np.maximum(So, 1e-300)).max() <= 1e-12


def _traj_err(spec, gg, go):
    n = go.shape[-2]
    k1 = spec.order_k + 1
    h = np.diff(oracle.Oracle(spec).edges())
    tot = go.sum(axis=0).reshape(n, spec.n_bins, k1)
    M1 = np.abs((h * tot[:, :, 0]).sum(axis=1))
    d = np.abs(gg - go).reshape(-1, n, spec.n_bins, k1).sum(axis=(0, 3))
    return ((h[None, :] * d).sum(axis=1) / M1).max()


def _species_bound(o, spec, gs):
    """The eq. (dt) bound of every species: min over bins losing mass of g_s,j^0 / |L_s,j^0| (the
    total's bound does not hold for a species whose bin loses mass while the total gains)."""
    L, _ = o.rhs_species(gs)
    S, n = gs.shape[:2]
    g0 = gs.reshape(S, n, spec.n_bins, -1)[..., 0]
    L0 = L.reshape(S, n, spec.n_bins, -1)[..., 0]
    r = np.where(L0 < 0, g0 / np.where(L0 < 0, -L0, 1.0), np.inf)
    return r.min(axis=(0, 2))


@pytest.mark.parametrize("name,limiter,frac", [("add", 1, 0.3), ("add", 0, 0.3), ("toy", 1, 0.05),
                                               ("k3", 1, 0.3)])
def test_species_steps_match_oracle(name, limiter, frac):
    """20 SSP-RK3 steps of 2 species (a tracer holding the two smallest bins, and the rest), 200
    cells, per-cell time steps up to frac of the species' bound; states, per-species M_1 and the
    status bits against the oracle."""
    spec = SPECS[name].replace(limiter=limiter)
    o = oracle.Oracle(spec)
    n = 200
    g = W.random_coefficients(spec, n, seed=86)
    tracer = np.zeros_like(g)
    tracer.reshape(n, spec.n_bins, -1)[:, :2, :] = g.reshape(n, spec.n_bins, -1)[:, :2, :]
    gs = np.stack([tracer, g - tracer])
    dt = np.random.default_rng(85).uniform(frac / 3, frac, n) * _species_bound(o, spec, gs)
    go, mo, fo = o.step_species(gs, dt, 20)
    assert np.all(fo & ~np.uint8(2) == 0)
    b = grace.Context([spec]).batch(n)
    gd = torch.as_tensor(gs, device=DEV)
    mass = torch.zeros((2, n), dtype=torch.float64, device=DEV)
    flags = torch.zeros(n, dtype=torch.uint8, device=DEV)
    b.step_species(gd, torch.as_tensor(dt, device=DEV), 20, mass=mass, flags=flags)
    gg = gd.cpu().numpy()
    assert _traj_err(spec, gg, go) <= 1e-12
    np.testing.assert_allclose(mass.cpu().numpy(), mo, rtol=1e-12, atol=1e-14 * np.abs(mo).max())
    np.testing.assert_array_equal(flags.cpu().numpy(), fo)


def test_species_step_of_one_species_is_grace_step():
    """S = 1 takes the single-distribution path's kernels: equal to grace_step in FP64 to rounding."""
    wl = W.batched_additive(n_cells=300, n_bins=16, order_k=2)
    b = grace.Context([wl.spec]).batch(wl.n_cells)
    g0 = b.project(wl.ic_kind, wl.ic_params)
    dt = torch.as_tensor(wl.dt, device=DEV)
    ref = g0.clone()
    b.step(ref, dt, 5)
    gs = g0.clone()[None].contiguous()
    b.step_species(gs, dt, 5)
    scale = ref.abs().amax(dim=1, keepdim=True)
    assert ((gs[0] - ref).abs() <= 1e-13 * scale).all()


def test_species_rejects_unsupported_batches():
    spec = SPECS["add"]
    b = grace.Context([spec]).batch(8)
    gs = torch.zeros((5, 8, 30), dtype=torch.float64, device=DEV)
    with pytest.raises(grace.GraceError):
        b.rhs_species(gs)
    specs, group, _, _ = W.uneven_batch(64, seed=3, n_range=(8, 10), orders=(1, 2))
    assert len(set(group.tolist())) > 1
    b2 = grace.Context(specs).batch(len(group), group)
    with pytest.raises(grace.GraceError):
        b2.rhs_species(torch.zeros((2, 64, 1), dtype=torch.float64, device=DEV))


TC_FORMS = [grace.TF32, grace.BF16X3]
TC_IDS = ["tf32", "bf16x3"]
TC_TOL = {grace.TF32: 2e-3, grace.BF16X3: 5e-5}
# trajectory bars: the RHS bar accumulated linearly over the 60 stages of 20 steps, each stage
# moving a species by at most 0.3 of its eq. (dt) bound (dt <= 0.3 B): 60 x 0.3 x TOL = 18 TOL
TC_TRAJ = {f: 18 * t for f, t in TC_TOL.items()}


@pytest.mark.parametrize("form", TC_FORMS, ids=TC_IDS)
@pytest.mark.parametrize("S", [1, 2, 4])
@pytest.mark.parametrize("name", ["add", "toy", "k3"])
def test_species_rhs_tensor_forms(name, S, form):
    """One tcgen05 pass over T with the cells' total as the A operand, each species contracting
    the accumulator: within the form's RHS bar of the oracle's species rates (300 cells, three
    128-cell tiles with a ragged tail)."""
    spec = SPECS[name]
    o = oracle.Oracle(spec)
    g = W.random_coefficients(spec, 300, seed=91)
    gs = _split(spec, g, S, seed=92 + S)
    Lo, So = o.rhs_species(gs)
    b = grace.Context([spec], 0, precisions=(grace.FP64, form)).batch(300)
    Lg = b.rhs_species(torch.as_tensor(gs, device=DEV), form).cpu().numpy()
    assert b.device_error() == 0
    err = np.abs(Lg - Lo) / np.maximum(np.maximum(np.abs(Lo), So), 1e-300)
    assert err.max() <= TC_TOL[form], err.max()


@pytest.mark.parametrize("form", TC_FORMS, ids=TC_IDS)
def test_species_steps_tensor_forms(form):
    """20 steps of a tracer and the rest (the additive kernel, limiter on) in a tensor form: the
    trajectory within the form's bar of the oracle, each species' M_1 conserved to round-off, and
    the eq. (dt), negative-mean, non-finite and drift bits equal to the oracle's."""
    spec = SPECS["add"]
    o = oracle.Oracle(spec)
    n = 200
    g = W.random_coefficients(spec, n, seed=86)
    tracer = np.zeros_like(g)
    tracer.reshape(n, spec.n_bins, -1)[:, :2, :] = g.reshape(n, spec.n_bins, -1)[:, :2, :]
    gs = np.stack([tracer, g - tracer])
    dt = np.random.default_rng(85).uniform(0.1, 0.3, n) * _species_bound(o, spec, gs)
    go, mo, fo = o.step_species(gs, dt, 20)
    b = grace.Context([spec], 0, precisions=(grace.FP64, form)).batch(n)
    gd = torch.as_tensor(gs, device=DEV)
    mass = torch.zeros((2, n), dtype=torch.float64, device=DEV)
    flags = torch.zeros(n, dtype=torch.uint8, device=DEV)
    b.step_species(gd, torch.as_tensor(dt, device=DEV), 20, form, mass=mass, flags=flags)
    assert b.device_error() == 0
    err = _traj_err(spec, gd.cpu().numpy(), go)
    assert err <= TC_TRAJ[form], err
    h = np.diff(o.edges())
    m0 = (h[None, None, :] * gs.reshape(2, n, spec.n_bins, -1)[..., 0]).sum(axis=2)
    assert np.all(np.abs(mass.cpu().numpy() - m0) <= 1e-13 * np.abs(m0).sum(axis=0))
    keep = np.uint8(~2 & 0xFF)
    np.testing.assert_array_equal(flags.cpu().numpy() & keep, fo & keep)
