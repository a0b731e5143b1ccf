"""Groups with a per-cell kernel parameter (non-separable kernels): the
ballistic-turbulent coagulation + fragmentation model with alpha_turb per cell.

The CUDA path evaluates the flux functionals from node-space tables and a
per-cell kernel factor; the oracle evaluates the nested quadrature directly,
one cell at a time with that cell's alpha.  Parity bars:
  FP64:    |L_gpu - L_oracle| <= 1e-12 max(|L_oracle|, S)
  TF32 / BF16X3 (fixed pairs on the tensor cores, partial entries in FP32): the
  bars of the separable tensor-core forms, 2e-3 and 5e-5 of max(|L_oracle|, S,
  1e-24 max S), and 1e-3 / 2e-5 of M_1 for trajectories."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _alphas(n, seed):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(1e-4), np.log(1e-2), n))


def _oracle_spec(spec, a):
    p = list(spec.coag_p)
    p[3] = a
    return spec.replace(coag_p=tuple(p), frag_p=tuple(p), cell_alpha=0)


def _coefs(spec, n, seed):
    return W.random_coefficients(spec, n, seed=seed, dynamic_range=6.0) * 1e-12


def _scaled_err(L, Lo, S):
    den = np.maximum(np.abs(Lo), S)
    return np.where(den > 0, np.abs(L - Lo) / np.where(den > 0, den, 1.0), np.abs(L - Lo) > 0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_rhs_matches_oracle_per_cell(k):
    spec = W.disk_spec(n_bins=12, order_k=k)
    n = 24
    alpha = _alphas(n, 300 + k)
    g = _coefs(spec, n, seed=310 + k)
    ctx = grace.Context([spec])
    b = ctx.batch(n)
    b.cell_params(alpha)
    L = b.rhs(torch.as_tensor(g.reshape(-1), device=DEV)).cpu().numpy().reshape(n, -1)
    worst = 0.0
    for c in range(n):
        Lo, S = oracle.Oracle(_oracle_spec(spec, alpha[c])).rhs(g[c:c + 1])
        worst = max(worst, _scaled_err(L[c:c + 1], Lo, S).max())
    assert worst <= 1e-12, worst


def test_pure_coagulation_limit_matches_separable_group():
    # alpha so small that dv < 0.8 v_frag for every pair: the per-cell path must agree
    # with the separable coagulation-only group that uses the precomputed T
    spec = W.disk_spec(n_bins=10, order_k=2)
    a = 1e-12
    sep = _oracle_spec(spec, a).replace(frag_kind=W.FRAG_NONE, frag_p=())
    n = 8
    g = _coefs(spec, n, seed=321)
    ctx = grace.Context([spec, sep])
    b = ctx.batch(n, np.zeros(n, dtype=np.int32))
    b.cell_params(np.full(n, a))
    b2 = ctx.batch(n, np.ones(n, dtype=np.int32))
    gt = torch.as_tensor(g.reshape(-1), device=DEV)
    L1 = b.rhs(gt).cpu().numpy().reshape(n, -1)
    L2 = b2.rhs(gt).cpu().numpy().reshape(n, -1)
    _, S = oracle.Oracle(sep).rhs(g)
    assert _scaled_err(L1, L2, S).max() <= 1e-12


def test_trajectory_matches_oracle_and_conserves_mass():
    spec = W.disk_spec(n_bins=10, order_k=2)
    n = 6
    alpha = _alphas(n, 330)
    g0 = np.abs(_coefs(spec, n, seed=331))
    # time step from the initial RHS: 2 % of the positivity bound min_j g_j^0 / |L_j^0| (larger
    # steps make these random, fragmentation-dominated states blow up in the oracle as well)
    o = [oracle.Oracle(_oracle_spec(spec, alpha[c])) for c in range(n)]
    dt = np.zeros(n)
    for c in range(n):
        L, _ = o[c].rhs(g0[c:c + 1])
        L0 = L.reshape(-1, 3)[:, 0]
        m0 = g0[c].reshape(-1, 3)[:, 0]
        neg = L0 < 0
        dt[c] = 0.02 * np.min(m0[neg] / -L0[neg]) if neg.any() else 1.0
    steps = 4
    ctx = grace.Context([spec])
    b = ctx.batch(n)
    b.cell_params(alpha)
    g = torch.as_tensor(g0.reshape(-1).copy(), device=DEV)
    mass = torch.zeros(n, dtype=torch.float64, device=DEV)
    b.step(g, torch.as_tensor(dt, device=DEV), steps, grace.FP64, mass=mass)
    gg = g.cpu().numpy().reshape(n, -1)
    m0 = b.mass(torch.as_tensor(g0.reshape(-1), device=DEV)).cpu().numpy()
    assert np.all(np.abs(mass.cpu().numpy() - m0) <= 1e-13 * np.abs(m0))
    for c in range(n):
        go, mo, _ = o[c].step(g0[c:c + 1], dt[c], steps)
        h = np.diff(o[c].edges())
        d = np.abs(gg[c] - go[0]).reshape(-1, 3).sum(axis=1)
        assert (h * d).sum() <= 1e-12 * abs(mo[0]), c


def test_mixed_batch_with_separable_group():
    disk = W.disk_spec(n_bins=10, order_k=1)
    add = W.additive_spec(n_bins=8, order_k=1)
    group = np.array([0, 1, 0, 1, 1, 0, 0, 1], dtype=np.int32)
    n = group.size
    alpha = _alphas(n, 340)
    ctx = grace.Context([disk, add])
    b = ctx.batch(n, group)
    b.cell_params(alpha)
    off = b.offsets()
    rng = np.random.default_rng(341)
    parts = []
    for c in range(n):
        spec = disk if group[c] == 0 else add
        gc = W.random_coefficients(spec, 1, seed=int(rng.integers(1 << 30)))[0]
        parts.append(gc * (1e-12 if group[c] == 0 else 1.0))
    g = np.concatenate(parts)
    L = b.rhs(torch.as_tensor(g, device=DEV)).cpu().numpy()
    for c in range(n):
        gc = g[off[c]:off[c + 1]][None]
        spec = _oracle_spec(disk, alpha[c]) if group[c] == 0 else add
        Lo, S = oracle.Oracle(spec).rhs(gc)
        assert _scaled_err(L[off[c]:off[c + 1]][None], Lo, S).max() <= 1e-12, c


def test_errors():
    spec = W.disk_spec(n_bins=8, order_k=1)
    ctx = grace.Context([spec], precisions=(grace.FP64, grace.TF32))
    b = ctx.batch(4)
    g = torch.as_tensor(_coefs(spec, 4, seed=350).reshape(-1), device=DEV)
    with pytest.raises(grace.GraceError, match="cell_params"):
        b.rhs(g)
    with pytest.raises(grace.GraceError, match="cell_params"):
        b.rhs(g, grace.TF32)
    b.cell_params(np.full(4, 1e-3))
    with pytest.raises(grace.GraceError, match="precomputed"):
        b.rhs(g, grace.BF16X3)     # not in the context's precisions
    b.rhs(g)
    b.rhs(g, grace.TF32)


# ------------------------------------------------------------------ tensor-core forms
TOL_RHS = {grace.TF32: 2e-3, grace.BF16X3: 5e-5}
TOL_L1 = {grace.TF32: 1e-3, grace.BF16X3: 2e-5}
RANGE_FLOOR = 1e-24
FORMS = [grace.TF32, grace.BF16X3]
IDS = ["tf32", "bf16x3"]


def _tc_ctx(specs):
    return grace.Context(specs, 0, precisions=(grace.FP64, grace.TF32, grace.BF16X3))


def _tc_scaled(L, Lo, S):
    floor = RANGE_FLOOR * S.max(axis=1, keepdims=True)
    den = np.maximum(np.maximum(np.abs(Lo), S), floor)
    d = np.abs(L - Lo)
    return np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))


def _oracle_rows(spec, alpha, g):
    Lo, S = [], []
    cache = {}
    for c in range(g.shape[0]):
        o = cache.setdefault(alpha[c], oracle.Oracle(_oracle_spec(spec, alpha[c])))
        l, s = o.rhs(g[c:c + 1])
        Lo.append(l[0])
        S.append(s[0])
    return np.array(Lo), np.array(S)


@pytest.mark.parametrize("form", FORMS, ids=IDS)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_rhs_tensor_forms_per_cell(k, form):
    # three 128-cell tiles, the last one ragged; alpha spans the whole ramp
    spec = W.disk_spec(n_bins=12, order_k=k)
    n = 300
    alpha = _alphas(n, 360 + k)
    g = _coefs(spec, n, seed=370 + k)
    ctx = _tc_ctx([spec])
    b = ctx.batch(n)
    b.cell_params(alpha)
    L = b.rhs(torch.as_tensor(g.reshape(-1), device=DEV), form).cpu().numpy().reshape(n, -1)
    assert b.device_error() == 0
    assert np.isfinite(L).all()
    Lo, S = _oracle_rows(spec, alpha, g)
    err = _tc_scaled(L, Lo, S)
    assert err.max() <= TOL_RHS[form], err.max()
    # mass: sum_j h_j L_j^0 telescopes to zero in FP64
    h = np.diff(oracle.Oracle(_oracle_spec(spec, alpha[0])).edges())
    L0 = L.reshape(n, spec.n_bins, k + 1)[:, :, 0]
    assert np.all(np.abs((h * L0).sum(axis=1)) <= 1e-14 * np.abs(h * L0).sum(axis=1))


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_tensor_forms_ramp_limits(form):
    # alpha at both ends of the ramp: no pair fragments (pf = 0 everywhere) / every pair
    # of the larger grains fragments; plus a single-cell batch
    spec = W.disk_spec(n_bins=10, order_k=2)
    alpha = np.array([1e-12, 1e-12, 0.5, 0.5, 1e-3])
    n = alpha.size
    g = _coefs(spec, n, seed=380)
    ctx = _tc_ctx([spec])
    b = ctx.batch(n)
    b.cell_params(alpha)
    L = b.rhs(torch.as_tensor(g.reshape(-1), device=DEV), form).cpu().numpy().reshape(n, -1)
    Lo, S = _oracle_rows(spec, alpha, g)
    assert _tc_scaled(L, Lo, S).max() <= TOL_RHS[form]
    b1 = ctx.batch(1)
    b1.cell_params(alpha[4:])
    L1 = b1.rhs(torch.as_tensor(g[4].copy(), device=DEV), form).cpu().numpy().reshape(1, -1)
    assert _tc_scaled(L1, Lo[4:], S[4:]).max() <= TOL_RHS[form]


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_tensor_forms_disk_workload_sampled(form):
    # the disk workload's sizes (N = 60, k = 2, MRN initial state) at 1,000 cells, sampled
    spec, alpha, ic = W.disk_batch(n_cells=1000, order_k=2)
    ctx = _tc_ctx([spec])
    b = ctx.batch(1000)
    b.cell_params(alpha)
    g = b.project(W.IC_POWERLAW, ic)
    L = b.rhs(g, form).cpu().numpy().reshape(1000, -1)
    # each side projects the initial state itself (Sec. 2.2) from the same parameters
    sample = np.array([0, 1, 127, 128, 500, 999])
    Lo, S = [], []
    for c in sample:
        o = oracle.Oracle(_oracle_spec(spec, alpha[c]))
        l, sc = o.rhs(o.project(W.IC_POWERLAW, ic[c:c + 1]))
        Lo.append(l[0])
        S.append(sc[0])
    assert _tc_scaled(L[sample], np.array(Lo), np.array(S)).max() <= TOL_RHS[form]


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_tensor_forms_trajectory(form):
    spec = W.disk_spec(n_bins=10, order_k=2)
    n = 6
    alpha = _alphas(n, 390)
    g0 = np.abs(_coefs(spec, n, seed=391))
    o = [oracle.Oracle(_oracle_spec(spec, alpha[c])) for c in range(n)]
    dt = np.zeros(n)
    for c in range(n):
        L, _ = o[c].rhs(g0[c:c + 1])
        L0 = L.reshape(-1, 3)[:, 0]
        m0 = g0[c].reshape(-1, 3)[:, 0]
        neg = L0 < 0
        dt[c] = 0.02 * np.min(m0[neg] / -L0[neg]) if neg.any() else 1.0
    steps = 4
    ctx = _tc_ctx([spec])
    b = ctx.batch(n)
    b.cell_params(alpha)
    g = torch.as_tensor(g0.reshape(-1).copy(), device=DEV)
    mass = torch.zeros(n, dtype=torch.float64, device=DEV)
    b.step(g, torch.as_tensor(dt, device=DEV), steps, form, mass=mass)
    gg = g.cpu().numpy().reshape(n, -1)
    m0 = b.mass(torch.as_tensor(g0.reshape(-1), device=DEV)).cpu().numpy()
    assert np.all(np.abs(mass.cpu().numpy() - m0) <= 1e-13 * np.abs(m0))
    for c in range(n):
        go, mo, _ = o[c].step(g0[c:c + 1], dt[c], steps)
        h = np.diff(o[c].edges())
        d = np.abs(gg[c] - go[0]).reshape(-1, 3).sum(axis=1)
        assert (h * d).sum() <= TOL_L1[form] * abs(mo[0]), c


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_tensor_forms_mixed_batch(form):
    disk = W.disk_spec(n_bins=10, order_k=1)
    add = W.additive_spec(n_bins=8, order_k=1)
    rng = np.random.default_rng(400)
    group = rng.integers(0, 2, 260).astype(np.int32)
    n = group.size
    alpha = _alphas(n, 401)
    ctx = _tc_ctx([disk, add])
    b = ctx.batch(n, group)
    b.cell_params(alpha)
    off = b.offsets()
    parts = []
    for c in range(n):
        spec = disk if group[c] == 0 else add
        gc = W.random_coefficients(spec, 1, seed=int(rng.integers(1 << 30)))[0]
        parts.append(gc * (1e-12 if group[c] == 0 else 1.0))
    g = np.concatenate(parts)
    L = b.rhs(torch.as_tensor(g, device=DEV), form).cpu().numpy()
    for c in range(0, n, 13):
        gc = g[off[c]:off[c + 1]][None]
        spec = _oracle_spec(disk, alpha[c]) if group[c] == 0 else add
        Lo, S = oracle.Oracle(spec).rhs(gc)
        assert _tc_scaled(L[off[c]:off[c + 1]][None], Lo, S).max() <= TOL_RHS[form], c
