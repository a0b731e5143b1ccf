"""Pins for the oracle's grid, basis, quadrature, projection and physics helpers.

Each check compares the oracle with something other than itself: closed forms
printed in the paper or in textbooks, numpy/scipy library routines, or exact
integrals.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npl
from scipy import integrate

import oracle
from paper_2607_13740_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_gauss_closed_forms():
    """eq. (quad): textbook nodes and weights for Q <= 4 (golden fixture)."""
    rows = _golden("gauss_closed_forms.txt")
    for Q in (1, 2, 3, 4):
        ref = np.array([[float(r[1]), float(r[2])] for r in rows if int(r[0]) == Q])
        s, w = oracle.gauss(Q)
        np.testing.assert_allclose(s, ref[:, 0], rtol=0, atol=2e-16)
        np.testing.assert_allclose(w, ref[:, 1], rtol=2e-15, atol=0)


@pytest.mark.parametrize("Q", list(range(1, 33)))
def test_gauss_matches_library_and_is_exact(Q):
    s, w = oracle.gauss(Q)
    sl, wl = npl.leggauss(Q)
    np.testing.assert_allclose(s, sl, rtol=0, atol=4e-15)
    np.testing.assert_allclose(w, wl, rtol=1e-14 if Q <= 8 else 1e-12, atol=0)
    assert abs(w.sum() - 2.0) < 1e-14
    # exact for polynomials of degree <= 2Q - 1
    for p in range(0, 2 * Q):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * s ** p) - exact) < 1e-13


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 6])
def test_legendre_matches_library(k):
    """eq. (2.4) values and derivatives against numpy's Legendre series."""
    for xi in np.linspace(-1, 1, 11):
        P, dP = oracle.legendre(k, xi)
        for i in range(k + 1):
            c = np.zeros(i + 1)
            c[i] = 1.0
            assert abs(P[i] - npl.legval(xi, c)) < 1e-14
            assert abs(dP[i] - npl.legval(xi, npl.legder(c))) < 1e-12


def test_orthogonality_mass_matrix():
    """eq. (2.5): int phi_i phi_m = delta_im * 2/(2i+1)."""
    s, w = npl.leggauss(20)
    k = 6
    Ps = np.array([oracle.legendre(k, x)[0] for x in s])
    M = (Ps * w[:, None]).T @ Ps
    np.testing.assert_allclose(M, np.diag(2.0 / (2 * np.arange(k + 1) + 1)), atol=1e-14)


def test_log_grid_edges():
    spec = W.additive_spec(40, 2)
    e = oracle.Oracle(spec).edges()
    assert e[0] == spec.x_min and e[-1] == spec.x_max
    r = e[1:] / e[:-1]
    np.testing.assert_allclose(r, (spec.x_max / spec.x_min) ** (1 / 40), rtol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_projection_reproduces_polynomials(k):
    """eq. (init) reproduces g0 = x (k >= 1) and g0 = x^2 (k >= 2) exactly:
    x = x_c + (h/2) xi and x^2 = x_c^2 + h^2/12 + x_c h xi + (h^2/6) P_2(xi)."""
    spec = W.GroupSpec(6, k, 1e-2, 1e2)
    o = oracle.Oracle(spec)
    e = o.edges()
    xc, h = 0.5 * (e[1:] + e[:-1]), np.diff(e)
    g = o.project(W.IC_POWERLAW, [2.0, 1.0, 0.0, 1e9])[0].reshape(6, k + 1)
    np.testing.assert_allclose(g[:, 0], 2 * xc, rtol=1e-13)
    np.testing.assert_allclose(g[:, 1], 2 * h / 2, rtol=1e-13)
    if k >= 2:
        np.testing.assert_allclose(g[:, 2:], 0.0, atol=1e-13 * np.max(np.abs(g)))
        g2 = o.project(W.IC_POWERLAW, [1.0, 2.0, 0.0, 1e9])[0].reshape(6, k + 1)
        np.testing.assert_allclose(g2[:, 0], xc ** 2 + h ** 2 / 12, rtol=1e-13)
        np.testing.assert_allclose(g2[:, 1], xc * h, rtol=1e-13)
        np.testing.assert_allclose(g2[:, 2], h ** 2 / 6, rtol=1e-12)


def test_mfrag_knots_golden():
    """eq. (mfrag) values at the branch knots (golden fixture) and continuity."""
    for r in _golden("mfrag_knots.txt"):
        q, val = float(r[0]), float(r[1])
        assert abs(oracle.mfrag_ratio(q) - val) <= 2e-16 * max(1.0, val) + 1e-17
    for q in (10.0, 12.0, 15.0, 50.0):
        lo, hi = oracle.mfrag_ratio(q * (1 - 1e-12)), oracle.mfrag_ratio(q * (1 + 1e-12))
        assert abs(lo - hi) < 1e-9


def test_maxwellian_probabilities_vs_quadrature():
    """beta_coag, beta_frag of Sec. 4.5 against scipy quadrature of f_v."""
    dv, vb, vf = 0.5, 0.1, 1.0
    fv = lambda v: 4 * math.pi * v * v * (3 / (2 * math.pi * dv * dv)) ** 1.5 * math.exp(-3 * v * v / (2 * dv * dv))
    bc = integrate.quad(fv, 0, vb, epsabs=1e-15, epsrel=1e-13)[0]
    bf = integrate.quad(fv, vf, np.inf, epsabs=1e-15, epsrel=1e-13)[0]
    spec = W.coupled_toy_spec()
    o = oracle.Oracle(spec)
    u = np.array([1e-3, 0.7, 5.0])
    v = np.array([2e-2, 0.7, 1e-5])
    kc, kf = o.kernels(u, v)
    sigma = np.pi * (np.cbrt(u) + np.cbrt(v)) ** 2
    np.testing.assert_allclose(kc / (sigma * dv), bc, rtol=1e-12)
    np.testing.assert_allclose(kf / (sigma * dv), bf, rtol=1e-12)


def _powerlaw_spec(cutoff_mode=0, mfrag_mode=0):
    return W.coupled_toy_spec().replace(cutoff_mode=cutoff_mode, mfrag_mode=mfrag_mode)


@pytest.mark.parametrize("cutoff_mode", [0, 1])
def test_product_mass_split(cutoff_mode):
    """eqs. (inte1)+(inte2): mass above x plus mass in [x_min, x] equals u + v
    (local mass conservation of eq. break) whenever the remnant lies in the
    domain; brute-force check of the power-law part by quadrature of w b(w)."""
    spec = _powerlaw_spec(cutoff_mode)
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(3)
    u = 10 ** rng.uniform(-5, 2, 400)
    v = 10 ** rng.uniform(-5, 2, 400)
    x = 10 ** rng.uniform(-6, 3, 400)
    a, b = o.mass_split(x, u, v)
    q = np.maximum(u, v) / np.minimum(u, v)
    mfrag = (u + v) * np.array([oracle.mfrag_ratio(t) for t in q])
    mleft = u + v - mfrag
    ok = (mleft >= spec.x_min) | (mleft <= 1e-300)
    np.testing.assert_allclose((a + b)[ok], (u + v)[ok], rtol=1e-12)
    assert np.all(a >= 0) and np.all(b >= 0)
    # independent power-law mass above x for a few destructive collisions (m_left = 0)
    alpha, xmin = spec.break_p[0], spec.x_min
    for i in np.where(q < 5)[0][:20]:
        mcut = (u[i] + v[i]) if cutoff_mode == 0 else max(u[i], v[i])
        if x[i] >= mcut:
            assert a[i] == 0.0
            continue
        A = (2 + alpha) * mfrag[i] / (mcut ** (2 + alpha) - xmin ** (2 + alpha))
        ref = integrate.quad(lambda w: w * A * w ** alpha, x[i], mcut, epsrel=1e-12)[0]
        assert abs(a[i] - ref) <= 1e-9 * mfrag[i]


def test_uniform_binary_mass_split():
    """Sec. 4.4 uniform binary breakage: above + below = u + v - x_min^2/u - x_min^2/v."""
    spec = W.pure_fragmentation_spec()
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(4)
    u = 10 ** rng.uniform(-5, 2, 200)
    v = 10 ** rng.uniform(-5, 2, 200)
    x = 10 ** rng.uniform(-6, 3, 200)
    a, b = o.mass_split(x, u, v)
    xm = spec.x_min
    np.testing.assert_allclose(a + b, u + v - xm * xm / u - xm * xm / v, rtol=1e-12)
