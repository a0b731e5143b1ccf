"""Tangent-linear and adjoint of the RHS and of the SSP-RK3 trajectory (FP64 and tensor forms).

Pins: L is a quadratic form, so (L(g+v) - L(g-v))/2 = J(g) v exactly; the
oracle supplies that exact directional derivative.  The VJP is checked by the
dot-product identity against the JVP; the trajectory adjoint and the parameter
gradients against the oracle's forward-mode derivative build (the oracle on dual
numbers: the exact derivative of its FP64 trajectory, limiter included), to 1e-10;
and against torch.autograd.gradcheck.

Tensor forms (TF32, BF16x3), with the forward bars of R15 (TOL = 2e-3 / 5e-5 of the
oracle's term-magnitude scale S):
  JVP   = [L(g + eps v) - L(g - eps v)] / (2 eps), eps a power of two per cell: each forward
          is within TOL S of the oracle, so the JVP is within TOL (S+ + S-) / (2 eps).
  VJP   component p against the oracle's lambda . J (s e_p) / s (exact by polarization), within
          TOL sum_j |lambda_j| (S+ + S-)_j / (2 s), an upper bound of the rounding of
          sum_r |mu_r| sum_q |(T_r + T_r^T)[p, q] g_q|.
  trajectory adjoint: within 36 TOL of max |directional derivative| (12 steps x 3 stages of
          per-RHS error, accumulated linearly).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SPECS = {
    "add_k2": W.additive_spec(16, 2, 1e-4, 1e6),
    "toy_remnant_k2": W.coupled_toy_spec(10, 2, flux_mode=0),
    "pure_frag_k1": W.pure_fragmentation_spec(10, 1, 1e-6, 1e3, flux_mode=0),
    "const_k3": W.GroupSpec(8, 3, 1e-2, 1e3, 0, W.COAG_CONST, (1.0,)),
}


@pytest.mark.parametrize("name", sorted(SPECS))
def test_jvp_equals_exact_central_difference_of_oracle(name):
    spec = SPECS[name]
    g = W.random_coefficients(spec, 9, seed=601)
    v = W.random_coefficients(spec, 9, seed=602) * 0.3
    ctx = grace.Context([spec])
    b = ctx.batch(9)
    Jv = b.jvp(torch.as_tensor(g, device=DEV), torch.as_tensor(v, device=DEV)).cpu().numpy()
    o = oracle.Oracle(spec)
    Lp, Sp = o.rhs(g + v)
    Lm, Sm = o.rhs(g - v)
    ref = 0.5 * (Lp - Lm)
    scale = np.maximum(Sp, Sm)
    assert np.all(np.abs(Jv - ref) <= 1e-12 * np.maximum(scale, 1e-300)), name


@pytest.mark.parametrize("name", sorted(SPECS))
def test_vjp_dot_product_identity(name):
    spec = SPECS[name]
    n = 40
    g = torch.as_tensor(W.random_coefficients(spec, n, seed=603), device=DEV)
    w = torch.as_tensor(np.random.default_rng(604).normal(size=(n, spec.n_coef)), device=DEV)
    lam = torch.as_tensor(np.random.default_rng(605).normal(size=(n, spec.n_coef)), device=DEV)
    ctx = grace.Context([spec])
    b = ctx.batch(n)
    lhs = (w * b.vjp(g, lam)).sum(dim=1)
    rhs = (b.jvp(g, w) * lam).sum(dim=1)
    rel = ((lhs - rhs).abs() / (lhs.abs() + rhs.abs())).max().item()
    assert rel < 1e-12, rel


def _traj_setup(spec, n, seed):
    o = oracle.Oracle(spec)
    g0 = o.project(W.IC_EXP, np.column_stack([np.full(n, 1.0), np.linspace(0.5, 2.0, n), np.zeros(n), np.zeros(n)]))
    rng = np.random.default_rng(seed)
    return o, g0, rng


@pytest.mark.parametrize("ckpt", [1, 4, 20])
def test_trajectory_adjoint_vs_oracle_tangent(ckpt):
    """<lambda_0, v> of the adjoint equals <lambda_T, dg_T> with dg_T the oracle's exact derivative
    of its trajectory along v (forward mode): two exact FP64 derivatives, equal to rounding."""
    spec = W.additive_spec(12, 2, 1e-3, 1e4).replace(limiter=0)
    n, steps, dt = 4, 12, 0.05
    o, g0, rng = _traj_setup(spec, n, 606)
    lamT = rng.normal(size=g0.shape)
    v = rng.uniform(-0.1, 0.1, size=g0.shape) * g0
    ctx = grace.Context([spec])
    b = ctx.batch(n)
    dtt = torch.full((n,), dt, dtype=torch.float64, device=DEV)
    lam0, _ = b.adjoint(torch.as_tensor(g0, device=DEV), dtt, steps, torch.as_tensor(lamT, device=DEV), ckpt)
    _, dg = o.tangent_step(g0, dt, steps, gdot=v)
    ref = (dg * lamT).sum(axis=1)
    ad = (lam0.cpu().numpy() * v).sum(axis=1)
    assert np.allclose(ad, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max()), (ad, ref)


def test_trajectory_adjoint_with_active_limiter():
    """Limiter on (it rescales bins in every step): the adjoint's limiter term (envelope theorem at
    the bin minimum) against the oracle's forward-mode derivative of the same trajectory."""
    spec = W.coupled_toy_spec(10, 2, flux_mode=0)
    n, steps, dt = 3, 10, 0.05
    o, g0, rng = _traj_setup(spec, n, 607)
    g0 = o.project(W.IC_EXP, [[1.0, 0.3, 0, 0], [2.0, 1.0, 0, 0], [0.5, 3.0, 0, 0]])
    assert np.all(o.step(g0, dt, steps)[2] & 2)      # the limiter acted in every cell
    lamT = rng.normal(size=g0.shape)
    v = rng.uniform(-0.1, 0.1, size=g0.shape) * g0
    ctx = grace.Context([spec])
    b = ctx.batch(n)
    dtt = torch.full((n,), dt, dtype=torch.float64, device=DEV)
    lam0, _ = b.adjoint(torch.as_tensor(g0, device=DEV), dtt, steps, torch.as_tensor(lamT, device=DEV), 5)
    _, dg = o.tangent_step(g0, dt, steps, gdot=v)
    ref = (dg * lamT).sum(axis=1)
    ad = (lam0.cpu().numpy() * v).sum(axis=1)
    assert np.allclose(ad, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max()), (ad, ref)


PARAM_CASES = {
    # Sec. 4.5 physics: dv_rms and v_bounce of the coagulation probability, dv_rms and v_frag of the
    # fragmentation probability, the fragment index alpha (eqs. break, inte1, inte2, App. B)
    "toy": (W.coupled_toy_spec(10, 2, flux_mode=0), [0, 1, 8, 9, 16], 0.05),
    # the disk physics with one alpha_turb (ramp inside the grid): rho_s, alpha_turb, v_frag, alpha
    "ballistic": (W.disk_spec(n_bins=10, order_k=2, cell_alpha=0, alpha=5e-6), [0, 11, 12, 16], None),
}


@pytest.mark.parametrize("name", sorted(PARAM_CASES))
def test_parameter_gradients_vs_oracle_tangent(name):
    """dJ/dtheta, J = <lambda_T, g_T>, from the exact dT/dtheta (forward mode through the FP64
    precompute) against <lambda_T, dg_T/dtheta> of the oracle's forward-mode trajectory."""
    spec, ids, dt = PARAM_CASES[name]
    n, steps = 3, 8
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(608)
    g0 = W.random_coefficients(spec, n, seed=609)
    if dt is None:
        # a quarter of the eq. (dt) bound of the initial state
        dt = 0.25 / o.substep_counts(g0, 1.0, 1.0).max()
    lamT = rng.normal(size=g0.shape)
    ctx = grace.Context([spec])
    ctx.param_grad_setup(ids)
    b = ctx.batch(n)
    dtt = torch.full((n,), dt, dtype=torch.float64, device=DEV)
    _, dth = b.adjoint(torch.as_tensor(g0, device=DEV), dtt, steps, torch.as_tensor(lamT, device=DEV), 4,
                       param_grads=True)
    dth = dth.cpu().numpy()
    for col, pid in enumerate(ids):
        _, dg = o.tangent_step(g0, dt, steps, param_id=pid)
        ref = (dg * lamT).sum(axis=1)
        assert np.abs(ref).max() > 0.0, pid
        assert np.allclose(dth[:, col], ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max()), (pid, dth[:, col], ref)


def test_finite_difference_tables_agree_with_the_exact_ones():
    """The central-difference dT/dtheta (rel_step > 0, kept for cross-checks) gives the same
    gradients as the exact tables to its truncation error."""
    spec, ids, dt = PARAM_CASES["toy"]
    n, steps = 3, 6
    g0 = W.random_coefficients(spec, n, seed=610)
    lamT = torch.as_tensor(np.random.default_rng(611).normal(size=g0.shape), device=DEV)
    out = []
    for rel in (0.0, 1e-6):
        ctx = grace.Context([spec])
        ctx.param_grad_setup(ids, rel_step=rel)
        b = ctx.batch(n)
        dtt = torch.full((n,), dt, dtype=torch.float64, device=DEV)
        _, dth = b.adjoint(torch.as_tensor(g0, device=DEV), dtt, steps, lamT, 3, param_grads=True)
        out.append(dth.cpu().numpy())
    assert np.allclose(out[1], out[0], rtol=1e-6, atol=1e-8 * np.abs(out[0]).max())


def test_autograd_function_gradcheck():
    spec = W.additive_spec(4, 1, 1e-2, 1e2).replace(limiter=0)
    ctx = grace.Context([spec])
    b = ctx.batch(1)
    g0 = b.project(W.IC_EXP, [[1.0, 1.0, 0.0, 0.0]]).requires_grad_(True)
    dt = torch.full((1,), 0.05, dtype=torch.float64, device=DEV)
    f = lambda g: grace.step_autograd(g, b, dt, 3, 2)
    assert torch.autograd.gradcheck(f, (g0,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_autograd_parameter_gradients_in_every_form():
    """step_autograd with theta: the gradient reaching theta is grace_adjoint's dJ/dtheta summed over
    the cells (FP64), and the BF16x3 form's gradients (g0 and theta) stay within the trajectory
    bar of the FP64 ones; J = <lambda_T, g_T> through torch.autograd."""
    spec = W.coupled_toy_spec(10, 2, flux_mode=0)
    n, steps, dt = 3, 8, 0.05
    o, g0, rng = _traj_setup(spec, n, 611)
    lamT = torch.as_tensor(rng.normal(size=g0.shape), device=DEV)
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, grace.BF16X3))
    ctx.param_grad_setup([9, 16])                 # frag_p[1] = v_f, break_p[0] = alpha
    b = ctx.batch(n)
    dtt = torch.full((n,), dt, dtype=torch.float64, device=DEV)
    grads = {}
    for form in (grace.FP64, grace.BF16X3):
        gin = torch.as_tensor(g0, device=DEV).clone().requires_grad_(True)
        theta = torch.zeros(2, dtype=torch.float64, device=DEV, requires_grad=True)
        gT = grace.step_autograd(gin, b, dtt, steps, 4, precision=form, theta=theta)
        (gT * lamT).sum().backward()
        grads[form] = (gin.grad.cpu().numpy(), theta.grad.cpu().numpy())
    _, dth = b.adjoint(torch.as_tensor(g0, device=DEV), dtt, steps, lamT, 4, param_grads=True)
    np.testing.assert_allclose(grads[grace.FP64][1], dth.sum(dim=0).cpu().numpy(), rtol=1e-12)
    for a, r in zip(grads[grace.BF16X3], grads[grace.FP64]):
        assert np.abs(a - r).max() <= 36 * 5e-5 * np.abs(r).max(), (np.abs(a - r).max(), np.abs(r).max())


def test_rosenbrock_step_with_gpu_jvps():
    """A linearly implicit (Rosenbrock-Euler) step (I - dt J) k = dt L(g), g+ = g + k, solved by GMRES
    whose matrix-vector products are the GPU's FP64 JVPs, against the dense solve with the oracle's
    exact Jacobian (polarization of the quadratic L, column by column); dt 20x the explicit
    positivity bound (a stiff step for the explicit scheme)."""
    from scipy.sparse.linalg import LinearOperator, gmres
    spec = W.additive_spec(12, 2, 1e-3, 1e4)
    o = oracle.Oracle(spec)
    g = o.project(W.IC_EXP, [[1.0, 0.5, 0, 0]])[0]
    P = spec.n_coef
    L0, _ = o.rhs(g[None])
    L0 = L0[0]
    means, Lm = g.reshape(-1, 3)[:, 0], L0.reshape(-1, 3)[:, 0]
    dt = 20.0 * (means[Lm < 0] / -Lm[Lm < 0]).min()
    J = np.zeros((P, P))
    for q in range(P):
        e = np.zeros(P)
        e[q] = 1.0
        Lp, _ = o.rhs((g + e)[None])
        Lm_, _ = o.rhs((g - e)[None])
        J[:, q] = 0.5 * (Lp[0] - Lm_[0])
    k_ref = np.linalg.solve(np.eye(P) - dt * J, dt * L0)
    ctx = grace.Context([spec])
    b = ctx.batch(1)
    gd = torch.as_tensor(g[None], device=DEV)

    def matvec(v):
        Jv = b.jvp(gd, torch.as_tensor(np.asarray(v, dtype=np.float64).reshape(1, P), device=DEV))
        return np.asarray(v).reshape(P) - dt * Jv.cpu().numpy().reshape(P)

    rhs = dt * b.rhs(gd).cpu().numpy().reshape(P)
    k_gpu, info = gmres(LinearOperator((P, P), matvec=matvec, dtype=np.float64), rhs, rtol=1e-14, atol=0.0,
                        restart=P, maxiter=10 * P)
    assert info == 0
    assert np.abs(k_gpu - k_ref).max() <= 1e-9 * np.abs(k_ref).max()


# ------------------------------------------------------------------ tensor forms
TOL_RHS = {grace.TF32: 2e-3, grace.BF16X3: 5e-5}
RANGE_FLOOR = 1e-24
FORMS = [grace.TF32, grace.BF16X3]
IDS = ["tf32", "bf16x3"]


def _tc_ctx(spec):
    return grace.Context([spec], 0, precisions=(grace.FP64, grace.TF32, grace.BF16X3))


def _pow2(x):
    """2^e with e the binary exponent of x (x = f 2^e, f in [0.5, 1)), per row."""
    return np.ldexp(1.0, np.frexp(x)[1])


@pytest.mark.parametrize("form", FORMS, ids=IDS)
@pytest.mark.parametrize("name", sorted(SPECS))
def test_jvp_tensor_forms_vs_oracle(name, form):
    spec = SPECS[name]
    n = 130                                   # two 128-cell tiles, the second ragged
    g = W.random_coefficients(spec, n, seed=611)
    v = W.random_coefficients(spec, n, seed=612) * 0.3
    ctx = _tc_ctx(spec)
    b = ctx.batch(n)
    Jv = b.jvp(torch.as_tensor(g, device=DEV), torch.as_tensor(v, device=DEV), form).cpu().numpy()
    assert np.isfinite(Jv).all()
    eps = (_pow2(np.abs(g).max(axis=1)) / _pow2(np.abs(v).max(axis=1)))[:, None]
    o = oracle.Oracle(spec)
    Lp, Sp = o.rhs(g + eps * v)
    Lm, Sm = o.rhs(g - eps * v)
    ref = (Lp - Lm) / (2 * eps)
    fl_p = RANGE_FLOOR * Sp.max(axis=1, keepdims=True)
    fl_m = RANGE_FLOOR * Sm.max(axis=1, keepdims=True)
    bound = TOL_RHS[form] * (np.maximum(Sp, fl_p) + np.maximum(Sm, fl_m)) / (2 * eps)
    worst = (np.abs(Jv - ref) / bound).max()
    assert worst <= 1.0, (name, worst)


@pytest.mark.parametrize("form", FORMS, ids=IDS)
@pytest.mark.parametrize("name", sorted(SPECS))
def test_vjp_tensor_forms_vs_oracle_directions(name, form):
    spec = SPECS[name]
    n, P = 3, spec.n_coef
    g = W.random_coefficients(spec, n, seed=613)
    lam = np.random.default_rng(614).normal(size=(n, P))
    ctx = _tc_ctx(spec)
    b = ctx.batch(n)
    w = b.vjp(torch.as_tensor(g, device=DEV), torch.as_tensor(lam, device=DEV), form).cpu().numpy()
    assert np.isfinite(w).all()
    o = oracle.Oracle(spec)
    for c in range(n):
        s = _pow2(np.abs(g[c]).max())
        X = g[c][None, :] + s * np.eye(P)
        Y = g[c][None, :] - s * np.eye(P)
        Lp, Sp = o.rhs(X)
        Lm, Sm = o.rhs(Y)
        ref = ((Lp - Lm) / (2 * s)) @ lam[c]
        bound = TOL_RHS[form] * ((Sp + Sm) / (2 * s)) @ np.abs(lam[c])
        worst = (np.abs(w[c] - ref) / bound).max()
        assert worst <= 1.0, (name, c, worst)


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_trajectory_adjoint_tensor_forms_vs_oracle(form):
    spec = W.additive_spec(12, 2, 1e-3, 1e4).replace(limiter=0)
    n, steps, dt = 4, 12, 0.05
    o, g0, rng = _traj_setup(spec, n, 615)
    lamT = rng.normal(size=g0.shape)
    v = rng.uniform(-0.1, 0.1, size=g0.shape) * g0
    ctx = _tc_ctx(spec)
    b = ctx.batch(n)
    dtt = torch.full((n,), dt, dtype=torch.float64, device=DEV)
    lam0, _ = b.adjoint(torch.as_tensor(g0, device=DEV), dtt, steps, torch.as_tensor(lamT, device=DEV), 4,
                        precision=form)
    lam0 = lam0.cpu().numpy()
    assert np.isfinite(lam0).all()
    eps = 1e-4
    gp, _, _ = o.step(g0 + eps * v, dt, steps)
    gm, _, _ = o.step(g0 - eps * v, dt, steps)
    fd = ((gp - gm) / (2 * eps) * lamT).sum(axis=1)
    ad = (lam0 * v).sum(axis=1)
    err = np.abs(ad - fd).max() / np.abs(fd).max()
    assert err <= 36 * TOL_RHS[form], (form, err, ad, fd)


def test_tensor_form_adjoint_errors():
    spec = SPECS["add_k2"]
    ctx = grace.Context([spec])                 # FP64 only: no tensor tiles
    b = ctx.batch(4)
    g = torch.as_tensor(W.random_coefficients(spec, 4, seed=616), device=DEV)
    with pytest.raises(grace.GraceError, match="precomputed"):
        b.vjp(g, g, grace.TF32)
    with pytest.raises(grace.GraceError, match="precomputed"):
        b.jvp(g, g, grace.BF16X3)


def test_jvp_vjp_adjoint_use_the_batch_group():
    """A context with two groups and a batch whose cells all belong to the second: the JVP, the
    VJP (dot-product identity) and the trajectory adjoint use that group's tables (oracle of that
    group's physics)."""
    spec0 = W.additive_spec(10, 2, 1e-3, 1e4)
    spec1 = W.coupled_toy_spec(10, 2, flux_mode=0)
    n = 5
    ctx = grace.Context([spec0, spec1])
    b = ctx.batch(n, np.ones(n, dtype=np.int32))
    o = oracle.Oracle(spec1)
    g = W.random_coefficients(spec1, n, seed=621)
    v = W.random_coefficients(spec1, n, seed=622) * 0.3
    Jv = b.jvp(torch.as_tensor(g, device=DEV), torch.as_tensor(v, device=DEV)).cpu().numpy()
    Lp, Sp = o.rhs(g + v)
    Lm, Sm = o.rhs(g - v)
    assert np.all(np.abs(Jv - 0.5 * (Lp - Lm)) <= 1e-12 * np.maximum(Sp, Sm))
    lam = np.random.default_rng(623).normal(size=g.shape)
    w = b.vjp(torch.as_tensor(g, device=DEV), torch.as_tensor(lam, device=DEV)).cpu().numpy()
    lhs, rhs = (w * v).sum(axis=1), (Jv * lam).sum(axis=1)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * (np.abs(lhs) + np.abs(rhs)))
    dt, steps = 0.02, 5
    lamT = np.random.default_rng(624).normal(size=g.shape)
    lam0, _ = b.adjoint(torch.as_tensor(g, device=DEV), torch.full((n,), dt, dtype=torch.float64, device=DEV), steps,
                        torch.as_tensor(lamT, device=DEV), 2)
    _, dg = o.tangent_step(g, dt, steps, gdot=v)
    ref = (dg * lamT).sum(axis=1)
    ad = (lam0.cpu().numpy() * v).sum(axis=1)
    assert np.allclose(ad, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
