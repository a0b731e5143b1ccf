"""Adjoint for groups with a per-cell kernel parameter (the ballistic-turbulent model with
alpha_turb per cell; no fixed T): FP64 JVP by polarization with a per-cell power-of-two scale,
VJP through the node-space tables (the fixed pairs' rows and transposed rows, the partial
entries), and the checkpointed trajectory adjoint, against the oracle run one cell at a time
with that cell's alpha (its exact polarization, and its forward-mode derivative build)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SPEC = W.disk_spec(n_bins=10, order_k=2)


def _oracle(a):
    p = list(SPEC.coag_p)
    p[3] = a
    return oracle.Oracle(SPEC.replace(coag_p=tuple(p), frag_p=tuple(p), cell_alpha=0))


def _setup(n, seed):
    rng = np.random.default_rng(seed)
    alpha = np.exp(rng.uniform(np.log(1e-4), np.log(1e-2), n))
    g = W.random_coefficients(SPEC, n, seed=seed + 1, dynamic_range=4.0) * 1e-12
    b = grace.Context([SPEC]).batch(n)
    b.cell_params(alpha)
    return alpha, g, b


def test_jvp_is_the_oracles_polarization():
    n = 6
    alpha, g, b = _setup(n, 701)
    v = W.random_coefficients(SPEC, n, seed=703, dynamic_range=4.0) * 1e-13
    Jv = b.jvp(torch.as_tensor(g, device=DEV), torch.as_tensor(v, device=DEV)).cpu().numpy()
    for c in range(n):
        o = _oracle(alpha[c])
        Lp, Sp = o.rhs(g[c:c + 1] + v[c:c + 1])
        Lm, Sm = o.rhs(g[c:c + 1] - v[c:c + 1])
        ref = 0.5 * (Lp - Lm)[0]
        assert np.all(np.abs(Jv[c] - ref) <= 1e-11 * np.maximum(Sp, Sm)[0]), c


def test_vjp_matches_the_oracles_exact_transpose():
    """Component p of J^T lambda against lambda . J e_p, J e_p from the oracle's polarization."""
    n = 3
    alpha, g, b = _setup(n, 711)
    lam = np.random.default_rng(712).normal(size=g.shape)
    w = b.vjp(torch.as_tensor(g, device=DEV), torch.as_tensor(lam, device=DEV)).cpu().numpy()
    P = SPEC.n_coef
    for c in range(n):
        o = _oracle(alpha[c])
        scale = np.abs(g[c]).max()
        E = np.eye(P) * scale
        Lp, Sp = o.rhs(g[c][None] + E)
        Lm, Sm = o.rhs(g[c][None] - E)
        ref = (0.5 * (Lp - Lm) / scale) @ lam[c]
        bound = (np.abs(lam[c])[None, :] * (Sp + Sm) / (2 * scale)).sum(axis=1)
        assert np.all(np.abs(w[c] - ref) <= 1e-11 * bound), (c, np.max(np.abs(w[c] - ref) / bound))


def test_vjp_dot_product_identity():
    n = 40
    alpha, g, b = _setup(n, 721)
    rng = np.random.default_rng(722)
    v = torch.as_tensor(rng.normal(size=g.shape) * 1e-12, device=DEV)
    lam = torch.as_tensor(rng.normal(size=g.shape), device=DEV)
    gd = torch.as_tensor(g, device=DEV)
    lhs = (b.vjp(gd, lam) * v).sum(dim=1)
    rhs = (b.jvp(gd, v) * lam).sum(dim=1)
    assert ((lhs - rhs).abs() / (lhs.abs() + rhs.abs())).max().item() < 1e-11


@pytest.mark.parametrize("ckpt", [1, 3])
def test_trajectory_adjoint_vs_oracle_tangent(ckpt):
    """8 limited SSP-RK3 steps at a fifth of each cell's eq. (dt) bound: <lambda_0, v> against
    <lambda_T, dg_T> with dg_T the oracle's forward-mode derivative of that cell's trajectory."""
    n = 4
    alpha, g, b = _setup(n, 731)
    steps = 8
    dt = np.array([0.2 / _oracle(alpha[c]).substep_counts(g[c:c + 1], 1.0, 1.0)[0] for c in range(n)])
    rng = np.random.default_rng(732)
    lamT = rng.normal(size=g.shape)
    v = rng.uniform(-0.1, 0.1, size=g.shape) * g
    lam0, _ = b.adjoint(torch.as_tensor(g, device=DEV), torch.as_tensor(dt, device=DEV), steps,
                        torch.as_tensor(lamT, device=DEV), ckpt)
    lam0 = lam0.cpu().numpy()
    for c in range(n):
        _, dg = _oracle(alpha[c]).tangent_step(g[c:c + 1], dt[c], steps, gdot=v[c:c + 1])
        ref = (dg[0] * lamT[c]).sum()
        ad = (lam0[c] * v[c]).sum()
        assert abs(ad - ref) <= 1e-10 * abs(ref) + 1e-12 * np.abs(dg[0] * lamT[c]).sum(), (c, ad, ref)


def test_tensor_forms_and_parameter_gradients_are_refused():
    alpha, g, b = _setup(2, 741)
    with pytest.raises(grace.GraceError):
        b.jvp(torch.as_tensor(g, device=DEV), torch.as_tensor(g, device=DEV), grace.BF16X3)
    ctx = grace.Context([SPEC])
    with pytest.raises(grace.GraceError):
        ctx.param_grad_setup([11])
