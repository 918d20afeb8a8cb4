"""Pins of the oracle's planet growth and gas gaps (Secs. 3.1 and 3.3).

References: the special values Eqs. 13 and 15 fix (the starting mass, the
core mass at tau_c where the two phases meet, the e-folding of the runaway
phase and its final mass), the Hill radius of a circular orbit, the limits of
Eq. 14, and the drag of a disk whose surface density is scaled as a whole
(the gap factor multiplies the gas density only).
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2601_16791_gb300 import workloads as W

MU0 = W.G
ME = W.M_EARTH


def params(gas=True):
    return orc.make_params(W.default_params(10.0, W.default_gas(gas)))


def one_planet(a=10.0, mass=0.0):
    """A planet on a circular orbit at (a, 0, 0), DH state, with its mass."""
    v = math.sqrt(MU0 * (1 + mass) / a)
    return np.array([[a], [0.0], [0.0], [0.0], [v], [0.0]]), np.array([MU0 * mass])


def track(m0=0.01 * ME, mc=15 * ME, mf=300 * ME, tc=1000.0, tg=300.0, dr=0.01):
    return dict(m0=[m0], mc=[mc], mf=[mf], tau_c=[tc], tau_g=[tg], delta_r=[dr], grows=[1])


def mass_at(t, g=None, mu=None):
    g = g or track()
    xv, mu0 = one_planet()
    out = orc.grow_state(params(), 1, xv, mu0 if mu is None else mu, [0.0], g, t)
    return out["mu"][0] / MU0


def test_masses_at_the_special_times():
    g = track()
    m0, mc, mf, tc, tg = 0.01 * ME, 15 * ME, 300 * ME, 1000.0, 300.0
    assert mass_at(0.0) == pytest.approx(m0, rel=1e-15)
    # the two phases meet at M_c (Eq. 13 at t = tau_c: the e/(e-1) factor)
    assert mass_at(tc) == pytest.approx(mc, rel=1e-14)
    assert mass_at(tc * (1 + 1e-12)) == pytest.approx(mc, rel=1e-9)
    # runaway accretion: e-folding time tau_g towards M_f
    assert (mf - mass_at(tc + tg)) / (mf - mc) == pytest.approx(math.exp(-1), rel=1e-13)
    assert (mf - mass_at(tc + 3 * tg)) / (mf - mc) == pytest.approx(math.exp(-3), rel=1e-12)
    assert mass_at(tc + 60 * tg) == pytest.approx(mf, rel=1e-15)
    # the core phase rises monotonically to M_c
    ts = np.linspace(0, tc, 50)
    ms = [mass_at(t) for t in ts]
    assert np.all(np.diff(ms) > 0)


def test_hill_radius_and_changeover_radius_follow_the_mass():
    """Circular orbit at 10 AU (massless before the update, so P = 0): R_H =
    a (M/3 m0)^(1/3) with a = 10, rcrit = 3 R_H, gap half-width 4 R_H after
    tau_c and none before, gap factor exp(-(t - tau_c)/tau_g)."""
    g = track()
    tc, tg = 1000.0, 300.0
    for t, M in ((500.0, None), (tc + 2 * tg, None)):
        M = mass_at(t)
        xv, _ = one_planet(10.0, M)      # circular for the updated mass
        out = orc.grow_state(params(), 1, xv, [0.0], [0.0], g, t)
        rh = 10.0 * (M / 3.0) ** (1.0 / 3.0)
        assert out["rcrit"][0] == pytest.approx(3.0 * rh, rel=1e-12)
        if t > tc:
            assert out["gap_w"][0] == pytest.approx(4.0 * rh, rel=1e-12)
            assert out["gap_f"][0] == pytest.approx(math.exp(-2.0), rel=1e-14)
        else:
            assert out["gap_w"][0] == 0.0 and out["gap_f"][0] == 1.0


def test_bodies_that_do_not_grow_keep_mass_and_radius():
    xv, mu = one_planet(10.0, 1e-5)
    g = track()
    g["grows"] = [0]
    out = orc.grow_state(params(), 1, xv, mu, [0.7], g, 5000.0)
    assert out["mu"][0] == mu[0] and out["rcrit"][0] == 0.7
    assert out["gap_w"][0] == 0.0 and out["radius"][0] == 0.0


def test_radius_limits():
    """Eq. 14: for G M / R_H << c_s^2 the radius tends to the Bondi-like
    G M / c_s^2, for G M / R_H >> c_s^2 to k2 R_H = R_H / 4.  Eq. 16: after
    tau_c the radius falls from R_c by delta_r (1 - exp(-(t - tau_c)/tau_g))."""
    p = params()
    cs = 0.05 * 10.0 ** 0.25 * math.sqrt(MU0 / 10.0)   # H/r v_k at 10 AU
    tiny = 1e-12
    g = track(m0=tiny, mc=tiny, mf=tiny)
    xv, _ = one_planet(10.0, tiny)
    out = orc.grow_state(p, 1, xv, [0.0], [0.0], g, 0.0)
    assert out["radius"][0] == pytest.approx(MU0 * tiny / cs ** 2, rel=1e-6)
    big = 0.5
    g = track(m0=big, mc=big, mf=big)
    xv, _ = one_planet(10.0, big)
    out = orc.grow_state(p, 1, xv, [0.0], [0.0], g, 0.0)
    rh = 10.0 * (big / 3.0) ** (1.0 / 3.0)
    assert out["radius"][0] == pytest.approx(rh / 4.0, rel=5e-3)
    g = track()
    M = mass_at(1000.0)
    xv, _ = one_planet(10.0, 15 * ME)
    rc = orc.grow_state(p, 1, xv, [0.0], [0.0], g, 1000.0)["radius"][0]
    r2 = orc.grow_state(p, 1, xv, [0.0], [0.0], g, 1000.0 + 300.0)["radius"][0]
    assert r2 == pytest.approx(rc - 0.01 * (1 - math.exp(-1)), rel=1e-12)
    assert M == pytest.approx(15 * ME, rel=1e-14)


def _gap_system():
    """One planet at 10 AU with a gap of half-width 1 AU and factor 0.25, and
    planetesimals at cylindrical distances across the band."""
    R = np.array([8.0, 9.2, 9.99, 10.5, 10.999, 11.5, 12.0])
    k = len(R)
    x = np.zeros((6, 1 + k))
    x[0, 0] = 10.0
    x[4, 0] = math.sqrt(MU0 / 10.0)
    x[0, 1:] = R
    x[2, 1:] = 0.01
    x[4, 1:] = np.sqrt(MU0 / R) * 0.999
    mu = np.array([MU0 * 1e-4] + [0.0] * k)
    rp = np.full(k, 10.0)
    rho = np.full(k, 2.0)
    return R, x, mu, rp, rho


def test_gap_scales_the_gas_density_of_the_disk():
    """Inside the band |R - r_p| < W the drag is the drag of the same disk with
    Sigma1 times the factor (Re and the drag both see rho_g); outside it is
    unchanged; the band is open at both ends."""
    R, x, mu, rp, rho = _gap_system()
    p = params()
    acc = orc.gas_drag_gap(p, 1, x, mu, rp, rho, [1.0], [0.25])
    plain = orc.gas_drag(p, 1, x, mu, rp, rho)
    g = W.default_gas(True, sigma1=1700.0 * 0.25)
    scaled = orc.gas_drag(orc.make_params(W.default_params(10.0, g)), 1, x, mu, rp, rho)
    inside = np.abs(R - 10.0) < 1.0
    assert inside.sum() == 4
    assert np.max(np.abs(acc[:, inside] - scaled[:, inside]) / np.abs(scaled[:, inside]).max()) < 1e-14
    assert np.array_equal(acc[:, ~inside], plain[:, ~inside])
    assert np.max(np.abs(scaled[:, inside] - plain[:, inside])) > 0.1 * np.abs(plain).max()
    # a body exactly on the band's edge is outside it
    x2 = x.copy()
    x2[0, 1] = 11.0
    x2[2, 1] = 0.0
    e2 = orc.gas_drag_gap(p, 1, x2, mu, rp, rho, [1.0], [0.25])
    p2 = orc.gas_drag(p, 1, x2, mu, rp, rho)
    assert np.array_equal(e2[:, 0], p2[:, 0])


def test_overlapping_gaps_take_the_last_planet():
    """Two planets whose bands overlap: the planetesimal in both gets the
    factor of the planet with the higher index (the listing's loop order)."""
    R, x, mu, rp, rho = _gap_system()
    x = np.concatenate([x[:, :1], x[:, :1], x[:, 1:]], axis=1)
    x[0, 1] = 10.5                     # second planet at 10.5 AU
    mu = np.concatenate([mu[:1], mu[:1], mu[1:]])
    p = params()
    acc = orc.gas_drag_gap(p, 2, x, mu, rp, rho, [1.0, 1.0], [0.25, 0.5])
    for sig, sel in ((0.5, (R > 9.5) & (R < 11.0)), (0.25, (R > 9.0) & (R <= 9.5))):
        g = W.default_gas(True, sigma1=1700.0 * sig)
        ref = orc.gas_drag(orc.make_params(W.default_params(10.0, g)), 2, x, mu, rp, rho)
        assert sel.any()
        assert np.max(np.abs(acc[:, sel] - ref[:, sel]) / np.abs(ref[:, sel]).max()) < 1e-14


def test_growth_run_follows_the_track():
    """A run with growth: after n steps from step0 the masses are the track's
    at the start of the last step (t = (step0 + n - 1) h) and the changeover
    radii have grown with them; planetesimals keep rcrit 0."""
    w = W.growth_2giant(nsmall=300, tau_c_days=400.0, tau_g_days=200.0)
    p = orc.make_params(w.params)
    xv, mu, rc = orc.init(p, w.nbig, w.nsmall, w.m_big, w.xv_helio)
    n = 30
    out, mu_n, stat, _, rc_n = orc.step_ex(p, w.nbig, xv, mu, rc, w.rp_km, w.rhop, n, step0=10,
                                           growth=w.growth, gap_c=w.gap_c)
    t_last = (10 + n - 1) * 10.0
    for i in range(2):
        g1 = {k: [v[i]] for k, v in w.growth.items()}
        M = mass_at(t_last, g1)
        assert mu_n[i] == pytest.approx(MU0 * M, rel=1e-15)
    assert np.all(mu_n[:2] > mu[:2] * 10)
    assert not stat.any()
    assert np.all(rc_n[2:] == 0.0)
    assert np.all(rc_n[:2] > rc[:2])
