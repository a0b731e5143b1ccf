"""Pins of the oracle's ballistic-turbulent kernel (the disk workload's library model, not in the
paper): sigma = pi (a_u + a_v)^2 for compact spheres a = (3 m / (4 pi rho_s))^(1/3), a turbulent
relative velocity dv = c_s sqrt(3 alpha St / (1 + St^2)) with the Epstein Stokes number
St = pi rho_s a / (2 Sigma_g) of the larger grain, and a linear fragmentation ramp
p_frag = clamp((dv - (1 - w) v_f) / (2 w v_f), 0, 1) splitting K = s sigma dv into
K_coag = K (1 - p_frag) and K_frag = K p_frag.

The formula is not re-typed here.  The tests check what the definition fixes: the symmetry in the
two colliders, exact power laws in alpha and in the rate scale, the power laws of K in the grain
mass in the limits St << 1 and St >> 1, the larger grain setting St, the invariance of
St / (1 + St^2) under St -> 1 / St with its maximum 1/2 at St = 1, and the ramp's end points and
mid point.  A dropped factor, a wrong exponent, the smaller grain in St or a shifted ramp fails
one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2607_13740_b300 import workloads as W

RHO, SIG, CS, ALPHA, VF, RW = 1.6, 10.0, 5.0e4, 1e-3, 100.0, 0.2
NO_FRAG = 1e300     # v_f so large that p_frag = 0


def kernels(u, v, rho=RHO, sig=SIG, cs=CS, alpha=ALPHA, vf=VF, rw=RW, scale=1.0):
    p = (rho, sig, cs, alpha, vf, rw, scale)
    spec = W.GroupSpec(4, 0, 1e-12, 1e3, W.FLUX_CONSERVATIVE, W.COAG_BALLISTIC, p, W.FRAG_BALLISTIC, p,
                       W.BREAK_POWERLAW_REMNANT, (-11.0 / 6.0,), 1, 0, 0, 1, 0)
    u, v = np.broadcast_arrays(np.atleast_1d(np.asarray(u, float)), np.atleast_1d(np.asarray(v, float)))
    return oracle.Oracle(spec).kernels(np.ascontiguousarray(u), np.ascontiguousarray(v))


def total(u, v, **kw):
    kc, kf = kernels(u, v, **kw)
    return kc + kf


def radius(m, rho=RHO):
    return (3.0 * m / (4.0 * math.pi * rho)) ** (1.0 / 3.0)


def test_symmetric_in_the_colliders():
    rng = np.random.default_rng(5)
    u, v = 10 ** rng.uniform(-11, 2, 200), 10 ** rng.uniform(-11, 2, 200)
    kc1, kf1 = kernels(u, v)
    kc2, kf2 = kernels(v, u)
    assert np.array_equal(kc1, kc2) and np.array_equal(kf1, kf2)
    assert np.all(kc1 >= 0) and np.all(kf1 >= 0)


def test_total_rate_does_not_depend_on_the_ramp():
    """v_f and the ramp width only split K between coagulation and fragmentation."""
    rng = np.random.default_rng(6)
    u, v = 10 ** rng.uniform(-11, 2, 100), 10 ** rng.uniform(-11, 2, 100)
    K = total(u, v, vf=NO_FRAG)
    for vf, rw in ((1.0, 0.2), (100.0, 0.2), (300.0, 0.05), (1e4, 0.5)):
        kc, kf = kernels(u, v, vf=vf, rw=rw)
        assert np.allclose(kc + kf, K, rtol=1e-14, atol=0)
    assert np.all(kernels(u, v, vf=NO_FRAG)[1] == 0.0)
    assert np.all(kernels(u, v, vf=1e-30)[0] == 0.0)   # every collision fragments


def test_power_laws_in_alpha_and_the_rate_scale():
    rng = np.random.default_rng(7)
    u, v = 10 ** rng.uniform(-11, 2, 50), 10 ** rng.uniform(-11, 2, 50)
    K = total(u, v, vf=NO_FRAG)
    assert np.allclose(total(u, v, vf=NO_FRAG, alpha=4 * ALPHA), 2.0 * K, rtol=1e-14, atol=0)   # dv ~ sqrt(alpha)
    assert np.allclose(total(u, v, vf=NO_FRAG, scale=3.0), 3.0 * K, rtol=1e-14, atol=0)
    assert np.allclose(total(u, v, vf=NO_FRAG, cs=2 * CS), 2.0 * K, rtol=1e-14, atol=0)


@pytest.mark.parametrize("sig,exponent", [(1e15, 5.0 / 6.0), (1e-15, 0.5)])
def test_mass_power_law_in_the_stokes_limits(sig, exponent):
    """Equal grains: sigma ~ m^(2/3), St ~ m^(1/3); dv ~ St^(1/2) for St << 1 (a huge gas surface
    density) and ~ St^(-1/2) for St >> 1, so K ~ m^(5/6) and m^(1/2)."""
    m = np.geomspace(1e-10, 1e1, 12)
    r = total(8 * m, 8 * m, sig=sig, vf=NO_FRAG) / total(m, m, sig=sig, vf=NO_FRAG)
    assert np.allclose(r, 8.0 ** exponent, rtol=1e-9, atol=0)


def test_the_larger_grain_sets_the_stokes_number():
    """Below a fixed larger grain v, changing the smaller one changes only the cross section."""
    v = 1e-3
    u = np.geomspace(1e-10, 5e-4, 20)
    u2 = u / 7.0
    r = total(u, v, vf=NO_FRAG) / total(u2, v, vf=NO_FRAG)
    geom = ((u / v) ** (1 / 3) + 1.0) ** 2 / ((u2 / v) ** (1 / 3) + 1.0) ** 2
    assert np.allclose(r, geom, rtol=1e-13, atol=0)


@pytest.mark.parametrize("m", [1e-9, 1e-4, 1.0])
def test_unit_stokes_number_is_the_velocity_maximum(m):
    """St / (1 + St^2) is invariant under St -> 1/St and peaks at 1/2 for St = 1: with the gas
    surface density that gives St = 1 the rate is s pi (2 a)^2 c_s sqrt(3 alpha / 2), and scaling
    the surface density by lam or 1/lam gives equal, smaller rates."""
    a = radius(m)
    sig1 = math.pi * RHO * a / 2.0          # St = 1
    K1 = total(m, m, sig=sig1, vf=NO_FRAG)[0]
    assert K1 == pytest.approx(math.pi * (2 * a) ** 2 * CS * math.sqrt(1.5 * ALPHA), rel=1e-13)
    for lam in (1.5, 10.0, 1e4):
        up, dn = total(m, m, sig=sig1 * lam, vf=NO_FRAG)[0], total(m, m, sig=sig1 / lam, vf=NO_FRAG)[0]
        assert up == pytest.approx(dn, rel=1e-13)
        assert up < K1
        assert up == pytest.approx(K1 * math.sqrt(2 * lam / (1 + lam * lam)), rel=1e-13)


def test_fragmentation_ramp_end_and_mid_points():
    """At St = 1 the relative velocity is dv* = c_s sqrt(3 alpha / 2): v_f = dv* puts the pair at the
    middle of the ramp (equal split), v_f = dv* / (1 - w) at its start (no fragmentation) and
    v_f = dv* / (1 + w) at its end (fragmentation only); a quarter of the way gives 1/4."""
    m = 1e-4
    a = radius(m)
    sig1 = math.pi * RHO * a / 2.0
    dv = CS * math.sqrt(1.5 * ALPHA)
    kc, kf = kernels(m, m, sig=sig1, vf=dv)
    assert kc[0] == pytest.approx(kf[0], rel=1e-12)
    kc, kf = kernels(m, m, sig=sig1, vf=dv / (1 - RW) * (1 + 1e-12))
    assert kf[0] == 0.0
    kc, kf = kernels(m, m, sig=sig1, vf=dv / (1 + RW) * (1 - 1e-12))
    assert kc[0] == 0.0
    # p = 1/4: dv - (1 - w) vf = (w / 2) vf  ->  vf = dv / (1 - w / 2)
    kc, kf = kernels(m, m, sig=sig1, vf=dv / (1 - RW / 2))
    assert kf[0] / (kc[0] + kf[0]) == pytest.approx(0.25, rel=1e-12)
