"""Caller-supplied bin edges on the GPU: RHS and trajectories on a non-uniform grid against the
oracle on the same grid (FP64 to 1e-12, the tensor forms within their bars), and the explicit log
grid equal to the default bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = {grace.FP64: 1e-12, grace.TF32: 2e-3, grace.BF16X3: 5e-5}


def _random_edges(x_min, x_max, n, seed):
    w = np.random.default_rng(seed).uniform(0.3, 1.8, n)
    t = np.concatenate([[0.0], np.cumsum(w)]) / w.sum()
    e = x_min * (x_max / x_min) ** t
    e[0], e[-1] = x_min, x_max
    return tuple(float(v) for v in e)


SPECS = {
    "add": W.additive_spec(20, 2, 1e-6, 1e10),
    "toy": W.coupled_toy_spec(12, 2, flux_mode=0, x_min=1e-3, x_max=1e4),
}


@pytest.mark.parametrize("form", [grace.FP64, grace.TF32, grace.BF16X3], ids=["fp64", "tf32", "bf16x3"])
@pytest.mark.parametrize("name", sorted(SPECS))
def test_rhs_on_a_nonuniform_grid(name, form):
    base = SPECS[name]
    spec = base.replace(edges=_random_edges(base.x_min, base.x_max, base.n_bins, 111))
    g = W.random_coefficients(spec, 300, seed=112)
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(300)
    L = b.rhs(torch.as_tensor(g, device=DEV), form).cpu().numpy()
    assert b.device_error() == 0
    Lo, S = oracle.Oracle(spec).rhs(g)
    keep = np.abs(g).max(axis=1, keepdims=True) * 1e-24 < np.abs(g) if form != grace.FP64 else np.ones_like(g, bool)
    err = np.abs(L - Lo) / np.maximum(np.maximum(np.abs(Lo), S), 1e-300)
    assert err[keep].max() <= TOL[form], err[keep].max()


def test_trajectory_on_a_nonuniform_grid_and_explicit_log_grid():
    base = SPECS["toy"]
    spec = base.replace(edges=_random_edges(base.x_min, base.x_max, base.n_bins, 113))
    o = oracle.Oracle(spec)
    g0 = W.random_coefficients(spec, 64, seed=114)
    dt = np.full(64, 0.01)
    b = grace.Context([spec]).batch(64)
    g = torch.as_tensor(g0, device=DEV)
    flags = torch.zeros(64, dtype=torch.uint8, device=DEV)
    b.step(g, torch.as_tensor(dt, device=DEV), 10, flags=flags)
    go, _, fo = o.step(g0, dt, 10)
    h = np.diff(o.edges())
    k1 = spec.order_k + 1
    d = (h[None, :] * np.abs(g.cpu().numpy() - go).reshape(64, -1, k1).sum(axis=2)).sum(axis=1)
    M1 = np.abs((h[None, :] * go.reshape(64, -1, k1)[:, :, 0]).sum(axis=1))
    assert (d / M1).max() <= 1e-12
    np.testing.assert_array_equal(flags.cpu().numpy(), fo)
    # the log grid given explicitly is the default grid
    e = tuple(oracle.Oracle(base).edges())
    L1 = grace.Context([base]).batch(64).rhs(torch.as_tensor(g0, device=DEV))
    L2 = grace.Context([base.replace(edges=e)]).batch(64).rhs(torch.as_tensor(g0, device=DEV))
    assert torch.equal(L1, L2)
