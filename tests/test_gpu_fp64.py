"""Parity of the CUDA FP64 path (through the C ABI) with the FP64 oracle.

RHS-level bar: |L_gpu - L_oracle| <= 1e-12 max(|L_oracle|, S) per coefficient,
S being the oracle's sum of magnitudes of the terms that make up the
coefficient (its rounding scale).  Trajectory bar: 1e-10 relative on the
coefficients of bins holding at least 1e-14 of the cell's mass, and an
L1 difference sum_j h_j sum_i |dg_j^i| <= 1e-12 M_1.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

RHS_SPECS = {
    "const_noncons_k2": W.constant_kernel_spec(12, 2, W.FLUX_NONCONSERVATIVE, 1e-4, 1e6),
    "const_cons_k1": W.constant_kernel_spec(10, 1, W.FLUX_CONSERVATIVE, 1e-4, 1e6),
    "add_cons_k2": W.additive_spec(16, 2, 1e-6, 1e10),
    "mult_k3": W.GroupSpec(9, 3, 1e-2, 1e3, 0, W.COAG_MULT, (0.3,)),
    "k0": W.additive_spec(14, 0, 1e-3, 1e5),
    "two_bins": W.additive_spec(2, 2, 1e-1, 1e1),
    "pure_frag": W.pure_fragmentation_spec(10, 2, 1e-6, 1e3),
    "pure_frag_cons": W.pure_fragmentation_spec(10, 1, 1e-6, 1e3, flux_mode=0),
    "toy_remnant_k2": W.coupled_toy_spec(10, 2, flux_mode=0),
    "toy_remnant_k1_noncons": W.coupled_toy_spec(9, 1, flux_mode=1),
    "toy_k3_cut_larger": W.coupled_toy_spec(7, 3, flux_mode=0).replace(cutoff_mode=1),
    "toy_destructive": W.coupled_toy_spec(8, 2, flux_mode=0).replace(mfrag_mode=1),
    "delta_breakage": W.GroupSpec(8, 2, 1e-3, 1e3, 0, W.COAG_NONE, (), W.FRAG_MULT, (0.5,),
                                  W.BREAK_COAG_DELTA),
    "quad_q6": W.additive_spec(8, 2, 1e-3, 1e4).replace(quad_q=6),
    "const_noncons_k4": W.constant_kernel_spec(12, 4, W.FLUX_NONCONSERVATIVE, 1e-3, 1e15),
    "toy_remnant_k4": W.coupled_toy_spec(8, 4, flux_mode=0),
}


def scaled_err(L, Lo, S):
    """|L - Lo| / max(|Lo|, S), with 0/0 counted as 0 (all-zero bins)."""
    den = np.maximum(np.abs(Lo), S)
    d = np.abs(L - Lo)
    return np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))


def _rhs_err(spec, n_cells, seed):
    g = W.random_coefficients(spec, n_cells, seed=seed)
    ctx = grace.Context([spec])
    b = ctx.batch(n_cells)
    L = b.rhs(torch.as_tensor(g, device=DEV)).cpu().numpy()
    Lo, S = oracle.Oracle(spec).rhs(g)
    return scaled_err(L, Lo, S)


@pytest.mark.parametrize("name", sorted(RHS_SPECS))
def test_rhs_parity_fp64(name):
    err = _rhs_err(RHS_SPECS[name], 37, seed=101)
    assert err.max() <= 1e-12, f"{name}: max scaled error {err.max():.3e}"


def test_rhs_parity_several_tiles_ragged():
    """Batch spanning several 32-cell warps and 128-cell blocks with a ragged tail."""
    err = _rhs_err(W.additive_spec(40, 2), 331, seed=102)
    assert err.max() <= 1e-12


def test_single_cell_batch():
    err = _rhs_err(W.additive_spec(40, 2), 1, seed=103)
    assert err.max() <= 1e-12


def test_projection_and_mass_parity():
    wl = W.batched_additive(n_cells=50)
    ctx = grace.Context([wl.spec])
    b = ctx.batch(wl.n_cells)
    g = b.project(wl.ic_kind, wl.ic_params)
    o = oracle.Oracle(wl.spec)
    go = o.project(wl.ic_kind, wl.ic_params)
    gg = g.cpu().numpy()
    scale = np.abs(go).max(axis=1, keepdims=True)
    assert np.all(np.abs(gg - go) <= 1e-13 * scale)
    m = b.mass(g).cpu().numpy()
    np.testing.assert_allclose(m, o.mass(go), rtol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_limiter_parity(k):
    spec = W.GroupSpec(30, k, 1e-2, 1e2, 0, W.COAG_CONST, (1.0,))
    rng = np.random.default_rng(200 + k)
    g = np.zeros((40, 30, k + 1))
    g[:, :, 0] = rng.uniform(-0.05, 1.0, (40, 30))
    g[:, :, 1:] = np.abs(g[:, :, :1]) * rng.uniform(-1.5, 1.5, (40, 30, k))
    g = g.reshape(40, -1)
    ctx = grace.Context([spec])
    b = ctx.batch(40)
    gt = torch.as_tensor(g, device=DEV)
    fl = torch.zeros(40, dtype=torch.uint8, device=DEV)
    b.limit(gt, fl)
    go, fo = oracle.Oracle(spec).limit(g)
    np.testing.assert_allclose(gt.cpu().numpy(), go, rtol=1e-13, atol=1e-15)
    np.testing.assert_array_equal(fl.cpu().numpy(), fo)


def _trajectory_check(spec, g_gpu, g_orc, edges):
    k = spec.order_k
    h = np.diff(edges)
    n = g_orc.shape[0]
    go = g_orc.reshape(n, spec.n_bins, k + 1)
    gg = g_gpu.reshape(n, spec.n_bins, k + 1)
    M1 = (h * go[:, :, 0]).sum(axis=1)
    diff = np.abs(gg - go)
    significant = np.abs(go[:, :, 0] * h) >= 1e-14 * M1[:, None]
    scale = np.maximum(np.abs(go), np.abs(go[:, :, :1]))
    rel = np.where(significant[:, :, None], diff / np.maximum(scale, 1e-300), 0.0)
    l1 = (h[None, :] * diff.sum(axis=2)).sum(axis=1)
    return rel.max(), (l1 / np.abs(M1)).max()


def test_single_cell_constant_kernel_trajectory():
    """One cell, K = 1, N = 20 on [1e-4, 1e6], k = 2, g0 = x exp(-x), dt = 1e-2 to t = 10."""
    wl = W.single_cell_constant()
    ctx = grace.Context([wl.spec])
    b = ctx.batch(1)
    g = b.project(wl.ic_kind, wl.ic_params)
    g0 = g.cpu().numpy()
    dt = torch.as_tensor(wl.dt, device=DEV)
    mass = torch.zeros(1, dtype=torch.float64, device=DEV)
    flags = torch.zeros(1, dtype=torch.uint8, device=DEV)
    b.step(g, dt, wl.n_steps, mass=mass, flags=flags)
    o = oracle.Oracle(wl.spec)
    go, mo, fo = o.step(g0, wl.dt, wl.n_steps)
    rel, l1 = _trajectory_check(wl.spec, g.cpu().numpy(), go, o.edges())
    assert rel <= 1e-10 and l1 <= 1e-12, (rel, l1)
    np.testing.assert_allclose(mass.cpu().numpy(), mo, rtol=1e-13)
    assert flags.cpu().numpy()[0] == fo[0]


def test_batched_additive_trajectory_conserves_mass():
    """The batched additive-kernel workload (N = 40, k = 2) at 96 cells over its 100 steps."""
    wl = W.batched_additive(n_cells=96)
    ctx = grace.Context([wl.spec])
    b = ctx.batch(wl.n_cells)
    g = b.project(wl.ic_kind, wl.ic_params)
    g0 = g.cpu().numpy()
    m0 = b.mass(g).cpu().numpy()
    dt = torch.as_tensor(wl.dt, device=DEV)
    mass = torch.zeros(wl.n_cells, dtype=torch.float64, device=DEV)
    flags = torch.zeros(wl.n_cells, dtype=torch.uint8, device=DEV)
    b.step(g, dt, wl.n_steps, mass=mass, flags=flags)
    m = mass.cpu().numpy()
    assert np.all(np.abs(m - m0) <= 1e-13 * np.abs(m0))
    o = oracle.Oracle(wl.spec)
    go, mo, fo = o.step(g0, wl.dt, wl.n_steps)
    rel, l1 = _trajectory_check(wl.spec, g.cpu().numpy(), go, o.edges())
    assert rel <= 1e-10 and l1 <= 1e-12, (rel, l1)
    np.testing.assert_array_equal(flags.cpu().numpy(), fo)


def test_full_size_batch_sampled_cells():
    """65,536 cells in the launch configuration of the benchmark; sampled cells against the oracle."""
    wl = W.batched_additive()
    ctx = grace.Context([wl.spec])
    b = ctx.batch(wl.n_cells)
    g = b.project(wl.ic_kind, wl.ic_params)
    sample = np.array([0, 1, 127, 128, 4095, 33333, 65534, 65535])
    g0 = g[sample].cpu().numpy()
    dt = torch.as_tensor(wl.dt, device=DEV)
    b.step(g, dt, 2)
    L = b.rhs(g)
    o = oracle.Oracle(wl.spec)
    go, _, _ = o.step(g0, wl.dt[sample], 2)
    rel, l1 = _trajectory_check(wl.spec, g[sample].cpu().numpy(), go, o.edges())
    assert rel <= 1e-10 and l1 <= 1e-12, (rel, l1)
    Lo, S = o.rhs(g[sample].cpu().numpy())
    err = scaled_err(L[sample].cpu().numpy(), Lo, S)
    assert err.max() <= 1e-12


def test_coupled_toy_trajectory():
    """Coag + power-law/remnant fragmentation (App. B volume term) over 20 steps."""
    spec = W.coupled_toy_spec(10, 2, flux_mode=0)
    ic = np.array([[1.0, 1.0, 0, 0], [0.5, 0.1, 0, 0], [2.0, 3.0, 0, 0]])
    ctx = grace.Context([spec])
    b = ctx.batch(3)
    g = b.project(W.IC_EXP, ic)
    g0 = g.cpu().numpy()
    dt = np.full(3, 0.05)
    b.step(g, torch.as_tensor(dt, device=DEV), 20)
    o = oracle.Oracle(spec)
    go, _, _ = o.step(g0, dt, 20)
    rel, l1 = _trajectory_check(spec, g.cpu().numpy(), go, o.edges())
    assert rel <= 1e-10 and l1 <= 1e-12, (rel, l1)


def test_errors_surface_as_exceptions():
    spec = W.additive_spec(8, 2)
    ctx = grace.Context([spec])
    b = ctx.batch(4)
    g = torch.zeros(4, spec.n_coef, dtype=torch.float64, device=DEV)
    with pytest.raises(grace.GraceError):
        b.rhs(g, precision=grace.TF32)      # tensor-core tiles were not requested
    with pytest.raises(grace.GraceError):
        b.rhs(g.float())                    # wrong dtype


def test_rhs_parity_large_coefficient_count():
    """N = 170 bins of degree 4 (P = 850 coefficients per cell): the FP64 contraction stages 8 cells
    per warp (a 32-cell tile of coefficients would not fit in shared memory) and combines the four
    lanes of a cell with shuffles; same 1e-12 bar against the oracle."""
    spec = W.constant_kernel_spec(170, 4, W.FLUX_NONCONSERVATIVE, 1e-3, 1e15)
    err = _rhs_err(spec, 11, seed=104)
    assert err.max() <= 1e-12, f"max scaled error {err.max():.3e}"


def test_k4_trajectory_with_limiter():
    """Degree 4 over 20 steps with the limiter (bin minimum bracketed between the roots of the
    second derivative on the GPU, by a scan and bisection in the oracle): trajectory bars as above,
    status bits equal."""
    spec = W.constant_kernel_spec(16, 4, W.FLUX_CONSERVATIVE, 1e-3, 1e6)
    n = 24
    rng = np.random.default_rng(105)
    g = np.zeros((n, 16, 5))
    g[:, :, 0] = 10.0 ** rng.uniform(-2, 0, (n, 16))
    g[:, :, 1:] = g[:, :, :1] * rng.uniform(-0.8, 0.8, (n, 16, 4)) / np.arange(1, 5)
    g = g.reshape(n, -1)
    ctx = grace.Context([spec])
    b = ctx.batch(n)
    gt = torch.as_tensor(g, device=DEV)
    dt = torch.full((n,), 2e-2, dtype=torch.float64, device=DEV)
    flags = torch.zeros(n, dtype=torch.uint8, device=DEV)
    b.step(gt, dt, 20, flags=flags)
    o = oracle.Oracle(spec)
    go, _, fo = o.step(g, 2e-2, 20)
    rel, l1 = _trajectory_check(spec, gt.cpu().numpy(), go, o.edges())
    assert rel <= 1e-10 and l1 <= 1e-12, (rel, l1)
    np.testing.assert_array_equal(flags.cpu().numpy(), fo)
    assert (fo & grace.FLAG_LIMITED).any()
