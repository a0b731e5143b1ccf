"""Two-dimensional (mass, volume) DG of Sec. 5.3 on the GPU against the oracle.

The CUDA path evaluates the weak form through 1-D factor forms of the separable kernel terms (the
Gauss product rule of each four-dimensional integral factorises exactly), the oracle evaluates the
four-dimensional rules directly: both sum the same nodes, in different orders, so they agree to
rounding.  Bar: |L - L_oracle| <= 1e-11 of the cell's largest |L_oracle| (FP64 sums of a few
thousand terms of mixed signs), the same for steps relative to the cell's largest coefficient.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-11


def _rel(a, b):
    s = np.abs(b).max(axis=1, keepdims=True)
    return (np.abs(a - b) / np.maximum(s, 1e-300)).max()


CASES = {
    "additive_k0": W.mv_additive_spec(4, 4, 0, 6, 0.1, 10.0, 0.1, 10.0),
    "additive_k1": W.mv_additive_spec(4, 4, 1, 6, 0.1, 10.0, 0.1, 10.0),
    "additive_k2": W.mv_additive_spec(3, 3, 2, 6, 0.1, 10.0, 0.1, 10.0),
    "mixed_k3": W.mv_mixed_spec(2, 3, 3, 5, 0.1, 10.0, 0.1, 10.0),
    "mixed_k1_5x3": W.mv_mixed_spec(5, 3, 1, 6, 0.1, 10.0, 0.1, 100.0),
    "mixed_k1_3x5": W.mv_mixed_spec(3, 5, 1, 5, 0.01, 10.0, 0.1, 10.0),
    "product_k1": W.MVSpec(4, 4, 1, 0.1, 10.0, 0.1, 10.0, 6, ((1.0, 1.0, 1.0, 0.0, 0.0),)),
    "additive_k0_5x3": W.mv_additive_spec(5, 3, 0, 6, 0.1, 10.0, 0.1, 10.0),
    "mixed_k2_3x4": W.mv_mixed_spec(3, 4, 2, 5, 0.1, 10.0, 0.1, 10.0),
    "mixed_k4": W.mv_mixed_spec(2, 2, 4, 6, 0.1, 10.0, 0.1, 10.0),
    "mixed_k4_2x4": W.mv_mixed_spec(2, 4, 4, 5, 0.1, 10.0, 0.1, 10.0),
    "cross_k1": W.MVSpec(4, 3, 1, 0.1, 10.0, 0.1, 10.0, 6, ((2.0, 0.5, 0.0, 0.0, 1.0 / 3.0), (2.0, 0.0, 0.5, 1.0 / 3.0, 0.0))),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_matches_oracle(name):
    spec = CASES[name]
    g = W.mv_random_coefficients(spec, 3, seed=71)
    mv = grace.MV(spec)
    L = mv.rhs(torch.as_tensor(g, device=DEV)).cpu().numpy()
    Lo = oracle.MVOracle(spec).rhs(g)
    assert np.isfinite(L).all()
    assert _rel(L, Lo) <= TOL, _rel(L, Lo)


def test_rhs_with_data_in_part_of_the_grid_and_zero_cells():
    spec = CASES["mixed_k1_5x3"]
    g = np.concatenate([W.mv_random_coefficients(spec, 2, seed=73, support=(2, 2)), np.zeros((1, spec.n_coef))])
    mv = grace.MV(spec)
    L = mv.rhs(torch.as_tensor(g, device=DEV)).cpu().numpy()
    assert np.all(L[2] == 0.0)
    Lo = oracle.MVOracle(spec).rhs(g[:2])
    assert _rel(L[:2], Lo) <= TOL
    # an empty batch is a no-op
    mv.rhs(torch.zeros((0, spec.n_coef), dtype=torch.float64, device=DEV))


@pytest.mark.parametrize("name", ["additive_k1", "mixed_k1_5x3"])
def test_steps_match_oracle(name):
    spec = CASES[name]
    g = W.mv_random_coefficients(spec, 2, seed=77)
    # explicit steps well inside stability: dt |L| of about 1 % of the largest coefficient
    rate = np.abs(oracle.MVOracle(spec).rhs(g)).max(axis=1)
    dt = 0.01 * np.abs(g).max(axis=1) / rate * np.array([1.0, 0.5])
    mv = grace.MV(spec)
    gt = torch.as_tensor(g, device=DEV).clone()
    mv.step(gt, torch.as_tensor(dt, device=DEV), 3)
    go = oracle.MVOracle(spec).step(g, dt, 3)
    s = np.abs(go).max(axis=1, keepdims=True)
    assert (np.abs(gt.cpu().numpy() - go) / s).max() <= TOL


def test_workload_grid_sampled_cell():
    """The benchmark's grid shape at a smaller size: 8 x 8 bins over four decades, the mixed kernel,
    data in the lower half (no merger leaves); 512 cells on the GPU, one compared with the oracle."""
    spec, g0, dt = W.mv_batch(n_cells=512, n_x=8, n_v=8, quad_q=4)
    mv = grace.MV(spec)
    g = torch.as_tensor(g0, device=DEV)
    L = mv.rhs(g).cpu().numpy()
    Lo = oracle.MVOracle(spec).rhs(g0[[300]])
    assert _rel(L[[300]], Lo) <= TOL
    # the total mass rate of every cell is small: no merger leaves; the gain and loss rules differ by
    # the quadrature error of Q = 4 nodes on bins of ratio 3.2 only
    o = oracle.MVOracle(spec)
    ex, ev = o.edges()
    Lr = L.reshape(512, spec.n_x, 2, spec.n_v, 2)[:, :, 0, :, 0]
    rate = (np.diff(ex)[None, :, None] * np.diff(ev)[None, None, :] * Lr).sum(axis=(1, 2))
    m = o.mass(g0)
    assert np.all(np.abs(rate) <= 5e-4 * m), (np.abs(rate) / m).max()


def test_full_size_workload_conserves_mass():
    """The benchmark's workload at its full size (16,384 cells of 12 x 12 bins, Q = 8): no merger
    leaves the grid in these steps, and with Q = 8 the gain and loss rules agree to round-off, so
    every cell's mass is kept over three steps (a property that holds at any size)."""
    spec, g0, dt = W.mv_batch()
    mv = grace.MV(spec)
    g = torch.as_tensor(g0, device=DEV)
    mv.step(g, torch.as_tensor(dt, device=DEV), 3)
    K1 = spec.order_k + 1
    o = oracle.MVOracle(spec)
    ex, ev = o.edges()
    w = (np.diff(ex)[:, None] * np.diff(ev)[None, :]).reshape(-1)
    def mass(a):
        return (a.reshape(a.shape[0], spec.n_x, K1, spec.n_v, K1)[:, :, 0, :, 0].reshape(a.shape[0], -1) * w).sum(axis=1)
    m0, m1 = mass(g0), mass(g.cpu().numpy())
    assert np.isfinite(m1).all()
    assert np.abs(m1 - m0).max() <= 1e-12 * np.abs(m0).max()


# FP32 contraction (arithmetic = 1): the factor forms and the cell's coefficients are rounded to FP32
# (unit round-off u = 2^-24 = 6.0e-8) and every sum runs in FP32.  The longest chain of rounded
# operations behind one output, at the sizes here (at most 24 rows and columns per dimension, five
# kernel terms): the two 24-term sums of H and W, 18 lane terms and 5 butterfly levels of <Vg[b], W>,
# 24 row and 5 term accumulations into L and three input roundings, n ~ 200, so
# |dL| <= n u sum|products| ~ 1.2e-5 sum|products|.  With random signed Legendre coefficients the
# products' magnitudes sum to a few times |L| (at most 8x allowed), hence 1e-4 of the cell's largest |L|.
TOL32 = 1e-4


# every degree k = 0 .. 4 with P_v a multiple of 4 (float4 columns: additive_k0, additive_k1,
# mixed_k2_3x4, mixed_k3, mixed_k4_2x4) and not (scalar columns: additive_k0_5x3, mixed_k1_5x3,
# mixed_k1_3x5, cross_k1, additive_k2, mixed_k4)
@pytest.mark.parametrize("name", ["additive_k0", "additive_k0_5x3", "additive_k1", "additive_k2", "mixed_k2_3x4",
                                  "mixed_k3", "mixed_k4", "mixed_k4_2x4", "mixed_k1_5x3", "mixed_k1_3x5", "cross_k1"])
def test_fp32_rhs_matches_oracle(name):
    spec = CASES[name]
    g = W.mv_random_coefficients(spec, 3, seed=79)
    L = grace.MV(spec, fp32=True).rhs(torch.as_tensor(g, device=DEV)).cpu().numpy()
    Lo = oracle.MVOracle(spec).rhs(g)
    assert np.isfinite(L).all()
    err = _rel(L, Lo)
    assert err <= TOL32, err
    # the FP32 contraction does round: it is not the FP64 path
    assert err > 0.0


def test_fp32_steps_match_oracle_and_keep_the_state_fp64():
    spec = CASES["mixed_k1_5x3"]
    g = W.mv_random_coefficients(spec, 2, seed=83)
    rate = np.abs(oracle.MVOracle(spec).rhs(g)).max(axis=1)
    dt = 0.01 * np.abs(g).max(axis=1) / rate
    gt = torch.as_tensor(g, device=DEV).clone()
    grace.MV(spec, fp32=True).step(gt, torch.as_tensor(dt, device=DEV), 3)
    assert gt.dtype == torch.float64
    go = oracle.MVOracle(spec).step(g, dt, 3)
    s = np.abs(go).max(axis=1, keepdims=True)
    # three steps of three stages, each adding dt L with |dt L| ~ 1 % of the largest coefficient
    assert (np.abs(gt.cpu().numpy() - go) / s).max() <= 9 * 0.01 * TOL32


def test_fp32_workload_grid_sampled_cell_and_full_size_mass():
    """The benchmark's grid shape at a smaller size, one sampled cell against the oracle; then the
    full-size workload (16,384 cells of 12 x 12 bins, Q = 8) through three FP32 steps, where mass is
    kept up to the FP32 error of the rates: |dm| <= 9 (dt / 3) sum_bins w |dL| with |dL| bounded by
    TOL32 of the cell's largest |L| (an exact property of the step at any size)."""
    spec, g0, dt = W.mv_batch(n_cells=512, n_x=8, n_v=8, quad_q=4)
    L = grace.MV(spec, fp32=True).rhs(torch.as_tensor(g0, device=DEV)).cpu().numpy()
    assert _rel(L[[300]], oracle.MVOracle(spec).rhs(g0[[300]])) <= TOL32
    spec, g0, dt = W.mv_batch()
    mv = grace.MV(spec, fp32=True)
    g = torch.as_tensor(g0, device=DEV)
    Lmax = np.abs(mv.rhs(g).cpu().numpy()).max(axis=1)
    mv.step(g, torch.as_tensor(dt, device=DEV), 3)
    K1 = spec.order_k + 1
    ex, ev = oracle.MVOracle(spec).edges()
    w = (np.diff(ex)[:, None] * np.diff(ev)[None, :]).reshape(-1)
    def mass(a):
        return (a.reshape(a.shape[0], spec.n_x, K1, spec.n_v, K1)[:, :, 0, :, 0].reshape(a.shape[0], -1) * w).sum(axis=1)
    m0, m1 = mass(g0), mass(g.cpu().numpy())
    assert np.isfinite(m1).all()
    bound = 3 * dt * TOL32 * w.sum() * Lmax * 2  # three steps; 2x for the stages' own rates
    assert np.all(np.abs(m1 - m0) <= bound + 1e-12 * np.abs(m0))
