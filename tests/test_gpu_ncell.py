"""Groups with a per-cell kernel parameter (non-separable kernels): the
ballistic-turbulent coagulation + fragmentation model with alpha_turb per cell.

The CUDA path evaluates the flux functionals from node-space tables and a
per-cell kernel factor; the oracle evaluates the nested quadrature directly,
one cell at a time with that cell's alpha.  Parity bar as for the FP64 form:
|L_gpu - L_oracle| <= 1e-12 max(|L_oracle|, S)."""
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
    b.cell_params(np.full(4, 1e-3))
    with pytest.raises(grace.GraceError):
        b.rhs(g, grace.TF32)
    b.rhs(g)
