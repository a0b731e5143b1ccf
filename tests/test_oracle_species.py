"""Pins for the oracle's species of mixed grains (Sec. 5.3, reading R24): each species' partial mass
density g_s takes the outer-collider slot of every flux integral, the total g = sum_s g_s the
partner's, so the species' rates are bilinear forms L[g_s; g] sharing the tables of L[g]."""
import numpy as np
import pytest
from numpy.polynomial import Polynomial as Poly

import oracle
from paper_2607_13740_b300 import workloads as W


def _project_poly(o, coeffs):
    g = np.zeros(o.P)
    for p, c in enumerate(coeffs):
        g += o.project(W.IC_POWERLAW, [c, float(p), 0.0, 1e300])[0]
    return g


def test_uv_kernel_species_flux_is_exact():
    """K = uv with polynomial g_s and g: the species' interface flux
    F_s(x) = int_{x_min}^x u g_s(u) [G(v_max(u)) - G(x - u + x_min)] du (G' = g) is integrated exactly by
    the Q = k+1 rule; the species' mean-row rate in bin j is (F_s(x_{j-1/2}) - F_s(x_{j+1/2})) / h_j."""
    spec = W.GroupSpec(5, 3, 1e-1, 1e2, 0, W.COAG_MULT, (1.0,))
    o = oracle.Oracle(spec)
    cs, cg = [0.4, 0.3, 0.2], [0.5, 0.8, 0.4]
    gs, g = _project_poly(o, cs), _project_poly(o, cg)
    e = o.edges()
    Gp = Poly(cg).integ()
    u = Poly([0.0, 1.0])

    def F(x):
        lo = Poly([x + spec.x_min, -1.0])
        hi = Poly([spec.x_max + spec.x_min, -1.0])
        outer = (u * Poly(cs) * (Gp(hi) - Gp(lo))).integ()
        return outer(x) - outer(spec.x_min)

    Fe = np.array([0.0] + [F(x) for x in e[1:-1]] + [0.0])
    L, _ = o.rhs_species(np.stack([gs[None], (g - gs)[None]]))
    L0 = L[0, 0].reshape(spec.n_bins, -1)[:, 0]
    ref = (Fe[:-1] - Fe[1:]) / np.diff(e)
    np.testing.assert_allclose(L0, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("spec", [
    W.additive_spec(10, 2, 1e-3, 1e4),
    W.coupled_toy_spec(8, 2, flux_mode=0, x_min=1e-3, x_max=1e4),
    W.pure_fragmentation_spec(8, 1, 1e-3, 1e4, flux_mode=0),
], ids=["add", "toy", "frag"])
def test_species_partition_rates(spec):
    """Linear in the outer slot: the species' rates add up to L[g] (sum_s g_s = g); a species holding a
    fixed fraction f of every bin gets f L[g]; each species' mass is conserved with conservative
    fluxes (its mean-row rates telescope); one species is the single-species RHS."""
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(71)
    g = W.random_coefficients(spec, 4, seed=72)
    w = rng.uniform(0.0, 1.0, (3, 4, spec.n_bins, 1))
    w /= w.sum(axis=0, keepdims=True)
    gs = (g.reshape(4, spec.n_bins, -1)[None] * w).reshape(3, 4, -1)
    gs[2] = g - gs[0] - gs[1]
    L, Sc = o.rhs_species(gs)
    Lt, St = o.rhs(g)
    assert np.all(np.abs(L.sum(axis=0) - Lt) <= 1e-13 * np.maximum(St, Sc.sum(axis=0)))
    f = 0.3
    Lf, _ = o.rhs_species(np.stack([f * g, (1 - f) * g]))
    assert np.all(np.abs(Lf[0] - f * Lt) <= 1e-13 * St)
    h = np.diff(o.edges())
    for s in range(3):
        ms = (h[None, :] * L[s].reshape(4, spec.n_bins, -1)[:, :, 0]).sum(axis=1)
        sc = (h[None, :] * Sc[s].reshape(4, spec.n_bins, -1)[:, :, 0]).sum(axis=1)
        assert np.all(np.abs(ms) <= 1e-14 * sc)
    L1, _ = o.rhs_species(g[None])
    np.testing.assert_array_equal(L1[0], Lt)


def test_species_steps_add_up_and_tracer_moves_up():
    """SSP-RK3 on the species: without the limiter the species' states add up to the single-species
    trajectory of the total (to rounding), each species' mass is conserved, and a species that starts
    in the smallest grains only ever leaves them by coagulation (its bin-0 mass falls)."""
    spec = W.additive_spec(10, 2, 1e-3, 1e4).replace(limiter=0)
    o = oracle.Oracle(spec)
    g = o.project(W.IC_EXP, [[1.0, 1.0, 0, 0], [2.0, 0.3, 0, 0]])
    tracer = np.zeros_like(g)
    tracer.reshape(2, spec.n_bins, -1)[:, 0, :] = g.reshape(2, spec.n_bins, -1)[:, 0, :]
    gs = np.stack([tracer, g - tracer])
    gT, mT, fT = o.step_species(gs, 0.02, 30)
    gref, mref, _ = o.step(g, 0.02, 30)
    scale = np.abs(gref).max(axis=1, keepdims=True)
    assert np.all(np.abs(gT.sum(axis=0) - gref) <= 1e-12 * scale)
    h = np.diff(o.edges())
    m0 = (h * gs.reshape(2, 2, spec.n_bins, -1)[:, :, :, 0]).sum(axis=2)
    np.testing.assert_allclose(mT, m0, rtol=1e-12)
    b0 = gT[0].reshape(2, spec.n_bins, -1)[:, 0, 0]
    assert np.all(b0 < tracer.reshape(2, spec.n_bins, -1)[:, 0, 0])
    assert np.all(fT & 16 == 0)
