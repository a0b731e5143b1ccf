"""Pins for caller-supplied bin edges (the grid of Sec. 3.1 generalised to any increasing edges):
the explicit log grid reproduces the default bit for bit; on a random non-uniform grid the K = uv
flux of a polynomial distribution is integrated exactly by the Q = k+1 rule and the mean-row rates
are the exact flux differences over the bin widths; conservative fluxes conserve M_1; invalid
grids are rejected."""
import numpy as np
import pytest
from numpy.polynomial import Polynomial as Poly

import oracle
from paper_2607_13740_b300 import workloads as W


def _random_edges(x_min, x_max, n, seed):
    """n bins whose log-widths vary by a factor of up to ~6."""
    w = np.random.default_rng(seed).uniform(0.3, 1.8, n)
    t = np.concatenate([[0.0], np.cumsum(w)]) / w.sum()
    e = x_min * (x_max / x_min) ** t
    e[0], e[-1] = x_min, x_max
    return tuple(float(v) for v in e)


def test_explicit_log_grid_equals_the_default():
    spec = W.coupled_toy_spec(8, 2, flux_mode=0, x_min=1e-3, x_max=1e4)
    o = oracle.Oracle(spec)
    e = o.edges()
    o2 = oracle.Oracle(spec.replace(edges=tuple(e)))
    g = W.random_coefficients(spec, 4, seed=101)
    np.testing.assert_array_equal(o2.rhs(g)[0], o.rhs(g)[0])
    np.testing.assert_array_equal(o2.step(g, 0.01, 3)[0], o.step(g, 0.01, 3)[0])


def _project_poly(o, coeffs):
    g = np.zeros(o.P)
    for p, c in enumerate(coeffs):
        g += o.project(W.IC_POWERLAW, [c, float(p), 0.0, 1e300])[0]
    return g


@pytest.mark.parametrize("seed", [102, 103])
def test_uv_flux_is_exact_on_a_nonuniform_grid(seed):
    """K = uv, g a quadratic on every bin (k = 2, the projection is exact): the interface flux
    F(x) = int_{x_min}^x u g(u) [G(v_max(u)) - G(x - u + x_min)] du (G' = g) is a polynomial the
    Q = 3 rule integrates exactly, and L_j^0 = (F(x_{j-1/2}) - F(x_{j+1/2})) / h_j."""
    spec = W.GroupSpec(7, 2, 1e-1, 1e2, 0, W.COAG_MULT, (1.0,))
    spec = spec.replace(edges=_random_edges(spec.x_min, spec.x_max, spec.n_bins, seed))
    o = oracle.Oracle(spec)
    np.testing.assert_array_equal(o.edges(), np.array(spec.edges))
    cg = [0.5, 0.8, 0.4]
    g = _project_poly(o, cg)
    e = o.edges()
    Gp = Poly(cg).integ()
    u = Poly([0.0, 1.0])

    def F(x):
        lo = Poly([x + spec.x_min, -1.0])
        hi = Poly([spec.x_max + spec.x_min, -1.0])
        outer = (u * Poly(cg) * (Gp(hi) - Gp(lo))).integ()
        return outer(x) - outer(spec.x_min)

    Fe = np.array([0.0] + [F(x) for x in e[1:-1]] + [0.0])
    L, _ = o.rhs(g[None])
    ref = (Fe[:-1] - Fe[1:]) / np.diff(e)
    np.testing.assert_allclose(L[0].reshape(spec.n_bins, -1)[:, 0], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_mass_is_conserved_on_a_nonuniform_grid():
    spec = W.coupled_toy_spec(9, 2, flux_mode=0, x_min=1e-3, x_max=1e4)
    spec = spec.replace(edges=_random_edges(spec.x_min, spec.x_max, spec.n_bins, 104))
    o = oracle.Oracle(spec)
    g = W.random_coefficients(spec, 5, seed=105)
    L, S = o.rhs(g)
    h = np.diff(o.edges())
    dm = (h[None, :] * L.reshape(5, spec.n_bins, -1)[:, :, 0]).sum(axis=1)
    sc = (h[None, :] * S.reshape(5, spec.n_bins, -1)[:, :, 0]).sum(axis=1)
    assert np.all(np.abs(dm) <= 1e-14 * sc)


@pytest.mark.parametrize("bad", ["decreasing", "ends"])
def test_invalid_grids_are_rejected(bad):
    spec = W.additive_spec(6, 1, 1e-2, 1e2)
    e = list(_random_edges(spec.x_min, spec.x_max, spec.n_bins, 106))
    if bad == "decreasing":
        e[2], e[3] = e[3], e[2]
    else:
        e[-1] = 2e2
    with pytest.raises(RuntimeError):
        oracle.Oracle(spec.replace(edges=tuple(e))).rhs(W.random_coefficients(spec, 1))
