"""grace_rosenbrock_step: the linearly implicit Euler step (I - dt J) k = dt L[g], g += k, solved per
cell by restarted GMRES on the library's JVPs, against the dense solve with the oracle's exact
Jacobian (columns by polarization of the quadratic L)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _system(o, g, dt):
    """(A, b) of the step: A = I - dt J with the oracle's J (J e_q = (L(g + e_q) - L(g - e_q)) / 2,
    exact for the quadratic L), b = dt L[g]."""
    P = g.shape[0]
    L0, _ = o.rhs(g[None])
    E = np.eye(P)
    Lp, _ = o.rhs(g[None] + E)
    Lm, _ = o.rhs(g[None] - E)
    J = 0.5 * (Lp - Lm).T
    return np.eye(P) - dt * J, dt * L0[0]


def _bound(o, spec, g):
    L, _ = o.rhs(g[None])
    m, Lm = g.reshape(spec.n_bins, -1)[:, 0], L[0].reshape(spec.n_bins, -1)[:, 0]
    return (m[Lm < 0] / -Lm[Lm < 0]).min()


@pytest.mark.parametrize("name", ["add", "toy"])
def test_rosenbrock_step_matches_the_dense_solve(name):
    """Four cells, dt from 2x to 50x the explicit positivity bound; FP64 JVPs, rtol 1e-13."""
    spec = {"add": W.additive_spec(12, 2, 1e-3, 1e4), "toy": W.coupled_toy_spec(10, 2, flux_mode=0)}[name]
    o = oracle.Oracle(spec)
    g = o.project(W.IC_EXP, [[1.0, 0.5, 0, 0], [2.0, 1.0, 0, 0], [0.7, 2.0, 0, 0], [1.5, 0.2, 0, 0]])
    dt = np.array([2.0, 10.0, 20.0, 50.0]) * np.array([_bound(o, spec, gc) for gc in g])
    systems = [_system(o, g[c], dt[c]) for c in range(4)]
    ref = np.stack([g[c] + np.linalg.solve(A, rhs) for c, (A, rhs) in enumerate(systems)])
    b = grace.Context([spec]).batch(4)
    gd = torch.as_tensor(g, device=DEV)
    it = b.rosenbrock_step(gd, torch.as_tensor(dt, device=DEV), grace.FP64, krylov_dim=spec.n_coef,
                           max_restarts=3, rtol=1e-13)
    assert 0 < it <= 4 * spec.n_coef
    got = gd.cpu().numpy()
    for c, (A, rhs) in enumerate(systems):
        k = got[c] - g[c]
        # what GMRES guarantees: a small residual of the system it solves; the GPU's JVP tables agree
        # with the oracle's J to 1e-12 of the flux terms' magnitude, which here exceeds |L| by up to
        # ~100x, so the exact system's residual is held to 1e-9 of ||dt L||
        assert np.linalg.norm(A @ k - rhs) <= 1e-9 * np.linalg.norm(rhs), c
        # and the increment within the system's condition number of the dense solve
        kref = ref[c] - g[c]
        kappa = np.linalg.cond(A)
        assert np.abs(k - kref).max() <= max(1e-9, 1e-13 * kappa) * np.abs(kref).max(), (c, kappa)
    # conservative fluxes: the implicit step keeps M_1 (sum_j h_j (J v)_j^0 = 0 for every v)
    h = np.diff(o.edges())
    m0 = (h * g.reshape(4, spec.n_bins, -1)[:, :, 0]).sum(axis=1)
    m1 = (h * got.reshape(4, spec.n_bins, -1)[:, :, 0]).sum(axis=1)
    assert np.all(np.abs(m1 - m0) <= 1e-11 * m0)


@pytest.mark.parametrize("form", [grace.TF32, grace.BF16X3], ids=["tf32", "bf16x3"])
def test_rosenbrock_step_tensor_form_jvps(form):
    """200 cells (two tiles, ragged tail) at 10x the explicit bound with the tensor forms' JVPs.  The
    JVP and L[g] of the form carry a relative error of at most its RHS bar TOL, so the increment
    solves a system perturbed by O(TOL) and moves from the FP64-JVP increment by at most about
    kappa(I - dt J) TOL: each cell's deviation is held to 10 kappa TOL (kappa from the oracle's J)."""
    spec = W.additive_spec(16, 2, 1e-3, 1e4)
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(631)
    n = 200
    g = o.project(W.IC_EXP, np.stack([rng.uniform(0.5, 2.0, n), rng.uniform(0.2, 2.0, n), np.zeros(n),
                                      np.zeros(n)], axis=1))
    dt = 10.0 * np.array([_bound(o, spec, gc) for gc in g])
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(n)
    dtt = torch.as_tensor(dt, device=DEV)
    g64 = torch.as_tensor(g, device=DEV)
    b.rosenbrock_step(g64, dtt, grace.FP64, krylov_dim=48, max_restarts=4, rtol=1e-12)
    gt = torch.as_tensor(g, device=DEV)
    b.rosenbrock_step(gt, dtt, form, krylov_dim=48, max_restarts=4, rtol=1e-12)
    assert b.device_error() == 0
    k64, kt = (g64.cpu().numpy() - g), (gt.cpu().numpy() - g)
    assert np.isfinite(kt).all()
    tol = {grace.TF32: 2e-3, grace.BF16X3: 5e-5}[form]
    kappa = np.array([np.linalg.cond(_system(o, g[c], dt[c])[0]) for c in range(n)])
    err = np.abs(kt - k64).max(axis=1) / np.abs(k64).max(axis=1)
    assert np.all(err <= 10 * kappa * tol), (err / (kappa * tol)).max()
    assert np.median(err) <= 100 * tol      # and typically close to the form's bar


def test_rosenbrock_step_rejects_bad_arguments():
    spec = W.additive_spec(8, 1, 1e-3, 1e4)
    b = grace.Context([spec]).batch(2)
    g = b.project(W.IC_EXP, [[1.0, 1.0, 0, 0]] * 2)
    dt = torch.ones(2, dtype=torch.float64, device=DEV)
    with pytest.raises(grace.GraceError):
        b.rosenbrock_step(g, dt, krylov_dim=65)
    with pytest.raises(grace.GraceError):
        b.rosenbrock_step(g, dt, rtol=0.0)
