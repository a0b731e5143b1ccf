"""Pins for the oracle's flux evaluation (Sec. 3.3, App. B) against exact
polynomial integrals, brute-force adaptive quadrature and identities."""
import warnings

import numpy as np
import pytest
from numpy.polynomial import Polynomial as Poly
from numpy.polynomial import legendre as npl
from scipy import integrate

import oracle
from paper_2607_13740_b300 import workloads as W
from analytic import dg_eval


def _project_poly(o, coeffs):
    """Coefficients of the global polynomial sum_p c_p x^p (projection is exact for p <= k)."""
    g = np.zeros(o.P)
    for p, c in enumerate(coeffs):
        g += o.project(W.IC_POWERLAW, [c, float(p), 0.0, 1e300])[0]
    return g


def _exact_uv_flux(spec, coeffs, x):
    """F(x) of eq. (Fcoagtrun) for K = uv and a global polynomial g, integrated exactly:
    F = int_{x_min}^x u g(u) [G(v_max(u)) - G(x - u + x_min)] du with G' = g."""
    g = Poly(coeffs)
    G = g.integ()
    u = Poly([0.0, 1.0])
    lo = Poly([x + spec.x_min, -1.0])
    hi = Poly([spec.x_max + spec.x_min, -1.0]) if spec.flux_mode == 0 else Poly([spec.x_max])
    outer = (u * g * (G(hi) - G(lo))).integ()
    return outer(x) - outer(spec.x_min)


@pytest.mark.parametrize("k,coeffs", [(2, [0.7, 1.3]), (3, [0.5, 0.8, 0.4])])
@pytest.mark.parametrize("mode", [0, 1])
def test_uv_kernel_flux_is_exact(k, coeffs, mode):
    """With K = uv the integrand u g(u) g(v) is a polynomial of degree <= 2Q - 1 in each
    variable when g is a global polynomial of degree <= k - 1, so the nested Q = k+1 rule
    (partial bins A, B and, inside a bin, the partial outer piece) is exact."""
    spec = W.GroupSpec(5, k, 1e-1, 1e2, mode, W.COAG_MULT, (1.0,))
    o = oracle.Oracle(spec)
    e = o.edges()
    g = _project_poly(o, coeffs)
    xs = np.concatenate([e[1:-1], [0.37, 2.2, 45.0, 99.0]])
    F, _ = o.flux_point(g, xs, 1)
    ex = np.array([_exact_uv_flux(spec, coeffs, x) for x in xs])
    np.testing.assert_allclose(F, ex, rtol=1e-13)
    # the same exactness through the fragmentation path with b = delta(w - u - v)
    fspec = spec.replace(coag_kind=W.COAG_NONE, coag_p=(), frag_kind=W.FRAG_MULT, frag_p=(1.0,),
                         break_kind=W.BREAK_COAG_DELTA)
    Ff, _ = oracle.Oracle(fspec).flux_point(g, xs, 2)
    np.testing.assert_allclose(Ff, ex, rtol=1e-13)


def _brute_coag(spec, coef, x, kern):
    e = oracle.Oracle(spec).edges()
    xmin, xmax, k = spec.x_min, spec.x_max, spec.order_k
    g = lambda y: dg_eval(coef, e, k, np.array([y]))[0]

    def inner(u):
        lo = x - u + xmin
        hi = xmax - u + xmin if spec.flux_mode == 0 else xmax
        if hi <= lo:
            return 0.0
        pts = [p for p in e if lo < p < hi]
        return integrate.quad(lambda v: kern(u, v) * g(v) / v, lo, hi, points=pts or None,
                              limit=200, epsabs=0, epsrel=1e-12)[0]

    # the inner lower limit crosses a bin edge at u = x + x_min - edge (a kink in u)
    pts = [p for p in e if xmin < p < x] + [x + xmin - p for p in e if xmin < x + xmin - p < x]
    if spec.flux_mode == 0:
        pts += [xmax + xmin - p for p in e if xmin < xmax + xmin - p < x]
    return integrate.quad(lambda u: g(u) * inner(u), xmin, x, points=sorted(set(pts)) or None,
                          limit=400, epsabs=0, epsrel=1e-11)[0]


def test_additive_flux_converges_to_adaptive_quadrature():
    """eq. (Fcoagtrun) with K = x + y: the nested Gauss rule converges to an
    adaptive double integral (breakpoints at edges and kinks) as Q grows."""
    spec = W.GroupSpec(4, 1, 1e-2, 1e2, 0, W.COAG_ADD, (1.0,))
    coef = W.random_coefficients(spec, 1, seed=5, dynamic_range=1.0)[0]
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        for x in (0.3, 7.0):
            ex = _brute_coag(spec, coef, x, lambda u, v: u + v)
            err = []
            for Q in (2, 24):
                F, _ = oracle.Oracle(spec.replace(quad_q=Q)).flux_point(coef, [x], 1)
                err.append(abs(F[0] - ex) / abs(ex))
            assert err[0] < 5e-2
            assert err[1] < 5e-5 and err[1] < err[0] / 100


def test_pure_fragmentation_flux_converges_to_adaptive_quadrature():
    """eq. (Ffragtrun) with K_frag = xy and uniform binary breakage: positive
    minus negative flux against a brute-force nested quadrature."""
    spec = W.pure_fragmentation_spec(4, 1, 1e-2, 1e2)
    o = oracle.Oracle(spec)
    e = o.edges()
    xmin, xmax, k = spec.x_min, spec.x_max, spec.order_k
    coef = W.random_coefficients(spec, 1, seed=6, dynamic_range=1.0)[0]
    g = lambda y: dg_eval(coef, e, k, np.array([y]))[0]
    x = 0.3

    def above(u, v):  # Sec. 4.4: (y^2 - x^2)/y for each fragmenting particle y > x
        return ((u * u - x * x) / u if u > x else 0.0) + ((v * v - x * x) / v if v > x else 0.0)

    def below(u, v):
        return (min(x, u) ** 2 - xmin ** 2) / u + (min(x, v) ** 2 - xmin ** 2) / v

    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        vmax = lambda u: xmax if spec.flux_mode else xmax - u + xmin
        pos = integrate.quad(lambda u: g(u) * integrate.quad(
            lambda v: u * v * g(v) * above(u, v) / (v * (u + v)), x - u + xmin, vmax(u),
            points=[p for p in list(e) + [x] if x - u + xmin < p < vmax(u)] or None, limit=300,
            epsrel=1e-10)[0], xmin, x,
            points=sorted(set([p for p in e if xmin < p < x] + [x + xmin - p for p in e if xmin < x + xmin - p < x])) or None,
            limit=300, epsrel=1e-9)[0]
        neg = integrate.quad(lambda u: g(u) * integrate.quad(
            lambda v: u * v * g(v) * below(u, v) / (v * (u + v)), xmin, vmax(u),
            points=[p for p in list(e) + [x] if xmin < p < vmax(u)] or None, limit=300, epsrel=1e-10)[0],
            x, xmax, points=[p for p in e if x < p < xmax] or None, limit=300, epsrel=1e-9)[0]
    ex = pos - neg
    err = []
    for Q in (2, 24):
        F, _ = oracle.Oracle(spec.replace(quad_q=Q)).flux_point(coef, [x], 2)
        err.append(abs(F[0] - ex) / abs(ex))
    assert err[0] < 5e-2
    assert err[1] < 1e-3 and err[1] < err[0] / 20


@pytest.mark.parametrize("spec", [
    W.additive_spec(6, 2, 1e-2, 1e3),
    W.pure_fragmentation_spec(6, 2, 1e-2, 1e3, flux_mode=0),
    W.coupled_toy_spec(6, 2, flux_mode=0, x_min=1e-2, x_max=1e3),
], ids=["coag", "frag", "toy"])
def test_boundary_fluxes_vanish(spec):
    """Sec. 3.3: F(x_min) = 0 in both modes; F(x_max) = 0 for the conservative fluxes.
    With Delta x = 0 the flux through x_max is non-zero when coagulation is present
    (pure uniform binary breakage never makes products heavier than a collider)."""
    o = oracle.Oracle(spec)
    g = W.random_coefficients(spec, 1, seed=9)[0]
    F, Fa = o.flux_point(g, [spec.x_min, spec.x_max], 3)
    assert F[0] == 0.0 and F[1] == 0.0
    Fi, _ = o.flux_point(g, [np.sqrt(spec.x_min * spec.x_max)], 3)
    assert Fi[0] != 0.0
    ospec = spec.replace(flux_mode=1)
    F2, _ = oracle.Oracle(ospec).flux_point(g, [spec.x_min, spec.x_max], 3)
    assert F2[0] == 0.0
    assert (F2[1] != 0.0) == (spec.coag_kind != W.COAG_NONE)


def test_delta_breakage_equals_coagulation_rhs():
    """eq. (Ffrag) with b = delta(w - (u + v)) is the coagulation flux (end of Sec. 2.2);
    the whole L[g] through the fragmentation path equals the coagulation one."""
    cspec = W.GroupSpec(8, 2, 1e-3, 1e3, 0, W.COAG_MULT, (0.5,))
    fspec = cspec.replace(coag_kind=W.COAG_NONE, coag_p=(), frag_kind=W.FRAG_MULT, frag_p=(0.5,),
                          break_kind=W.BREAK_COAG_DELTA)
    g = W.random_coefficients(cspec, 3, seed=11)
    Lc, Sc = oracle.Oracle(cspec).rhs(g)
    Lf, _ = oracle.Oracle(fspec).rhs(g)
    assert np.all(np.abs(Lc - Lf) <= 1e-14 * Sc)


@pytest.mark.parametrize("spec0", [
    W.coupled_toy_spec(3, 2, flux_mode=0, x_min=1e-2, x_max=1e2),
    W.coupled_toy_spec(3, 2, flux_mode=0, x_min=1e-2, x_max=1e2).replace(cutoff_mode=1),
    W.disk_spec(n_bins=3, order_k=2, a_min=1e-4, a_max=1e-1, cell_alpha=0, alpha=3e-3),
], ids=["toy_cut_mfrag", "toy_cut_larger", "disk_physics"])
def test_appB_volume_term_converges_to_pointwise_flux_integral(spec0):
    """App. B reordering: sum over (u, v) of the five sub-interval integrals equals
    int_{I_j} F_frag(x) d_x phi_i dx computed from the pointwise flux; both converge
    to the same value as the Gauss order grows (R7, R8).  Cases: the paper's cutoff
    m_cut = m_frag, the cutoff at the larger collider mass, and the disk workload's physics
    (ballistic-turbulent kernels with the fragmentation ramp, one alpha)."""
    coef = W.random_coefficients(spec0, 1, seed=8, dynamic_range=1.0)[0]
    s8, w8 = npl.leggauss(8)
    diffs = {}
    for Q in (3, 24):
        o = oracle.Oracle(spec0.replace(quad_q=Q))
        e = o.edges()
        for j in range(3):
            V, Va = o.vol_frag(coef, j)
            h = e[j + 1] - e[j]
            acc = np.zeros(3)
            for p in range(64):
                a, b = e[j] + h * p / 64, e[j] + h * (p + 1) / 64
                xs = 0.5 * (a + b) + 0.5 * (b - a) * s8
                F, _ = o.flux_point(coef, xs, 2)
                xi = 2 * (xs - 0.5 * (e[j] + e[j + 1])) / h
                for i in (1, 2):
                    c = np.zeros(i + 1)
                    c[i] = 1
                    acc[i] += np.sum(0.5 * (b - a) * w8 * F * (2 / h) * npl.legval(xi, npl.legder(c)))
            diffs[(Q, j)] = np.max(np.abs(V[1:] - acc[1:]) / Va[1:])
            assert V[0] == 0.0
    for j in range(3):
        assert diffs[(24, j)] < 5e-3
        assert diffs[(24, j)] < diffs[(3, j)] / 5


def test_ballistic_turbulent_fluxes_converge_to_adaptive_quadrature():
    """The ballistic-turbulent model of the disk workload (per-cell alpha, fragmentation ramp,
    power-law fragments with a remnant): the oracle's nested Q-point rule for the coagulation
    flux (eq. Fcoagtrun) and for the fragmentation flux (eq. Ffragtrun, positive minus negative
    part) converges to adaptive double integrals of the same integrands, evaluated with the
    oracle's own kernel and product-mass functions, breakpoints at the bin edges, the end-bin
    kinks and the masses where the ramp starts and saturates.  This pins the quadrature with this
    kernel; the kernel itself is a library model (not in the paper)."""
    spec = W.disk_spec(n_bins=4, order_k=1, a_min=1e-4, a_max=1e-1, cell_alpha=0, alpha=1e-3)
    o = oracle.Oracle(spec)
    e = o.edges()
    xmin, xmax, k = spec.x_min, spec.x_max, spec.order_k
    coef = W.random_coefficients(spec, 1, seed=7, dynamic_range=1.0)[0]
    g = lambda y: dg_eval(coef, e, k, np.array([y]))[0]
    m = np.geomspace(xmin, xmax, 4000)
    kc, kf = o.kernels(m, np.full_like(m, xmin))
    tot = kc + kf
    pf = np.where(tot > 0, kf / np.where(tot > 0, tot, 1.0), 0.0)
    kinks = [float(np.sqrt(m[i] * m[i + 1])) for i in range(len(m) - 1)
             if (pf[i] == 0) != (pf[i + 1] == 0) or (pf[i] == 1) != (pf[i + 1] == 1)]
    assert len(kinks) >= 2                      # the ramp lies inside the grid
    x = float(np.sqrt(e[1] * e[2]))
    Kc = lambda u, v: o.kernels([u], [v])[0][0]
    Kf = lambda u, v: o.kernels([u], [v])[1][0]
    above = lambda u, v: o.mass_split([x], [u], [v])[0][0]
    below = lambda u, v: o.mass_split([x], [u], [v])[1][0]
    vmax = lambda u: xmax - u + xmin

    def pts(lo, hi, extra=()):
        p = sorted(set(q for q in list(e) + kinks + list(extra) if lo < q < hi))
        return p or None

    def nested(f, ulo, uhi, vlo, vhi, upts, vextra):
        inner = lambda u: integrate.quad(lambda v: f(u, v), vlo(u), vhi(u), points=pts(vlo(u), vhi(u), vextra(u)),
                                         limit=100, epsrel=1e-8)[0]
        return integrate.quad(lambda u: g(u) * inner(u), ulo, uhi, points=pts(ulo, uhi, upts), limit=100,
                              epsrel=1e-7)[0]

    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        lo = lambda u: x - u + xmin
        ukinks = [x + xmin - q for q in list(e) + kinks] + kinks
        coag = nested(lambda u, v: Kc(u, v) * g(v) / v, xmin, x, lo, vmax, ukinks, lambda u: [u])
        pos = nested(lambda u, v: Kf(u, v) * g(v) * above(u, v) / (v * (u + v)), xmin, x, lo, vmax, ukinks,
                     lambda u: [u, x])
        neg = nested(lambda u, v: Kf(u, v) * g(v) * below(u, v) / (v * (u + v)), x, xmax, lambda u: xmin, vmax,
                     kinks, lambda u: [u, x])
    frag = pos - neg
    assert coag != 0.0 and frag != 0.0
    ec, ef = [], []
    for Q in (2, 32):
        oq = oracle.Oracle(spec.replace(quad_q=Q))
        ec.append(abs(oq.flux_point(coef, [x], 1)[0][0] - coag) / abs(coag))
        ef.append(abs(oq.flux_point(coef, [x], 2)[0][0] - frag) / abs(frag))
    assert ec[1] < 1e-2 and ec[1] < ec[0] / 50, ec
    assert ef[1] < 1e-3 and ef[1] < ef[0] / 100, ef


def _split_by_definition(x, u, v, xmin, cutoff_mode, alpha):
    """Products of one fragmenting collision from the breakage distribution of eq. (break):
    m_frag = (u + v) mfrag_ratio(max/min) (eq. mfrag, pinned by its knots) spread as a power
    law n(w) ~ w^alpha over [x_min, m_cut], plus a remnant of mass m_left = u + v - m_frag at
    w = m_left.  The power law's mass above / below x is integrated numerically from w n(w);
    m_cut <= x_min puts the fragment mass at x_min (R10); a remnant below x_min is outside the
    domain (R10).  Returns (above, below) as in eqs. (inte1), (inte2)."""
    big, small = max(u, v), min(u, v)
    mfrag = (u + v) * oracle.mfrag_ratio(big / small)
    mleft = max(u + v - mfrag, 0.0)
    mcut = big if cutoff_mode == 1 else mfrag
    if mcut > xmin:
        dens = lambda w: w ** (1.0 + alpha)
        tot = integrate.quad(dens, xmin, mcut, epsabs=0, epsrel=1e-13, limit=200)[0]
        lo = min(max(x, xmin), mcut)
        below = mfrag * integrate.quad(dens, xmin, lo, epsabs=0, epsrel=1e-13, limit=200)[0] / tot
        above = mfrag - below
    else:
        below, above = (mfrag, 0.0) if x > xmin else (0.0, mfrag)
    if mleft > x:
        above += mleft
    elif xmin <= mleft:
        below += mleft
    return above, below


# (u, v) pairs relative to x_min = 1e-2 on a 3-bin grid up to 1e2: equal and very unequal
# masses, the eq. (mfrag) branches, small colliders whose fragment mass falls below x_min (R10:
# v < x_min / 0.9 with u / v > 50) and remnants inside and outside the domain
_PAIRS = [(0.05, 0.04), (0.3, 0.02), (3.0, 0.011), (40.0, 0.0105), (7.0, 0.6), (0.5, 0.45),
          (20.0, 0.9), (60.0, 30.0), (2.0, 0.15), (0.012, 0.011), (90.0, 0.0102)]


@pytest.mark.parametrize("cutoff_mode", [0, 1])
def test_powerlaw_mass_split_matches_the_breakage_distribution(cutoff_mode):
    """eqs. (inte1), (inte2): the oracle's mass of products above and below x for power-law
    fragments plus a remnant equals the numerical w-integral of the breakage distribution, for
    both cutoffs (m_frag, and the larger collider mass) and the R10 cases."""
    spec = W.coupled_toy_spec(3, 2, flux_mode=0, x_min=1e-2, x_max=1e2).replace(cutoff_mode=cutoff_mode)
    o = oracle.Oracle(spec)
    alpha = spec.break_p[0]
    xs = [1e-2, 1.05e-2, 0.013, 0.04, 0.3, 2.0, 35.0, 95.0]
    r10 = 0
    for u, v in _PAIRS:
        for x in xs:
            a, b = o.mass_split([x], [u], [v])
            ea, eb = _split_by_definition(x, u, v, spec.x_min, cutoff_mode, alpha)
            assert abs(a[0] - ea) <= 1e-11 * (u + v) and abs(b[0] - eb) <= 1e-11 * (u + v), (u, v, x)
        r10 += (u + v) * oracle.mfrag_ratio(max(u, v) / min(u, v)) <= spec.x_min
    assert r10 >= 3        # the R10 branch is exercised


def _pair_flux_integral(o, spec, j, u, v):
    """int_{I_j} f_uv(x) d_x phi_i dx by adaptive quadrature of the pointwise pair flux of
    eq. (Ffragtrun): the products above x while u < x <= u + v - x_min (positive part, the v range
    starting at x - u + x_min), minus those in [x_min, x] while x < u (negative part)."""
    e = o.edges()
    a, b = e[j], e[j + 1]
    h, xc = b - a, 0.5 * (a + b)
    top = u + v - spec.x_min

    def f(x):
        above, below = o.mass_split([x], [u], [v])
        val = 0.0
        if u < x <= top:
            val += above[0]
        if x < u:
            val -= below[0]
        return val

    big, small = max(u, v), min(u, v)
    mfrag = (u + v) * oracle.mfrag_ratio(big / small)
    kinks = [u, top, mfrag, big, u + v - mfrag]
    pts = sorted(set(p for p in kinks if a < p < b)) or None
    out, scale = np.zeros(spec.order_k + 1), np.zeros(spec.order_k + 1)
    for i in range(1, spec.order_k + 1):
        c = np.zeros(i + 1)
        c[i] = 1.0
        dphi = lambda x: (2.0 / h) * npl.legval(2.0 * (x - xc) / h, npl.legder(c))
        out[i] = integrate.quad(lambda x: f(x) * dphi(x), a, b, points=pts, epsabs=0, epsrel=1e-12,
                                limit=400)[0]
        scale[i] = integrate.quad(lambda x: abs(f(x) * dphi(x)), a, b, points=pts, epsabs=0,
                                  epsrel=1e-10, limit=400)[0]
    return out, scale


@pytest.mark.parametrize("cutoff_mode", [0, 1])
def test_appB_pair_terms_match_pointwise_flux_integral(cutoff_mode):
    """App. B per collision pair: the five sub-interval terms (R7: positive terms on
    I_j cap (u, min(u+v-x_min, m_cut or m_left)), negative terms on I_j cap (x_min, u), R10 for
    m_cut <= x_min and remnants below x_min) equal the x-integral of the pair's pointwise flux
    times d_x phi_i over bin j, for every bin and pairs covering each interval end (u, u+v-x_min,
    m_cut and m_left below, inside and above the bin) and both cutoffs.  A wrong interval end
    (e.g. a missing min with u+v-x_min or with m_cut) fails this test."""
    spec = W.coupled_toy_spec(3, 2, flux_mode=0, x_min=1e-2, x_max=1e2).replace(
        cutoff_mode=cutoff_mode, quad_q=24)
    o = oracle.Oracle(spec)
    nonzero = 0
    for u, v in _PAIRS + [(v_, u_) for u_, v_ in _PAIRS[:4]]:
        for j in range(spec.n_bins):
            J = o.appB_pair(j, u, v)
            ref, scale = _pair_flux_integral(o, spec, j, u, v)
            assert J[0] == 0.0
            tol = 1e-10 * max(scale.max(), 1e-300)
            assert np.all(np.abs(J[1:] - ref[1:]) <= tol), (u, v, j, J, ref)
            nonzero += int(np.any(ref[1:] != 0.0))
    assert nonzero >= 20
