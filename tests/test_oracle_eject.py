"""Pins of the oracle's orbital elements and ejection test (Sec. 3.5).

References are independent of the oracle's element code: states built in this
file from elements (a rotation of the pericentre state, a Newton solve of
Kepler's equation in numpy), the oracle's Kepler drift (itself pinned against
the elliptic closed form) for the time dependence of the mean anomaly, and the
energy criterion of an unbound orbit.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2601_16791_gb300 import workloads as W

MU0 = W.G
TWO_PI = 2.0 * math.pi


def params(dt=8.0, eject_every=0):
    p = W.default_params(dt)
    p["eject_every"] = eject_every
    return orc.make_params(p)


def rot(xo, yo, vxo, vyo, inc, node, peri):
    """R_z(node) R_x(inc) R_z(peri) applied to an orbit-plane state."""
    def Rz(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])

    def Rx(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])

    R = Rz(node) @ Rx(inc) @ Rz(peri)
    return np.concatenate([R @ np.array([xo, yo, 0.0]), R @ np.array([vxo, vyo, 0.0])])


def angdiff(a, b):
    d = (np.asarray(a) - np.asarray(b)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


# ------------------------------------------------------------------ elements
@pytest.mark.parametrize("e", [0.0, 0.05, 0.6, 1.0, 1.7, 4.0])
def test_elements_at_pericentre(e):
    """At pericentre (distance q, speed sqrt(gm (1 + e)/q) perpendicular to
    the radius) every element is known: q, e, i, varpi = Omega + omega,
    Omega and M = 0."""
    q, inc, node, peri = 2.3, 0.4, 1.1, 2.0
    gm = MU0 * 1.001
    xv = rot(q, 0.0, 0.0, math.sqrt(gm * (1 + e) / q), inc, node, peri)[:, None]
    el = orc.elements(gm, xv)[:, 0]
    assert abs(el[0] - q) <= 1e-14 * q
    assert abs(el[1] - e) <= 1e-14
    assert abs(el[2] - inc) <= 1e-14
    assert abs(el[4] - node) <= 1e-14
    if e > 0:
        assert angdiff(el[3], node + peri) <= 1e-13
        assert angdiff(el[5], 0.0) <= 1e-13


def _kepler_state(gm, a, e, inc, node, peri, M):
    """Elliptic state from elements: Newton on E - e sin E = M in numpy."""
    E = M if e < 0.8 else math.pi
    for _ in range(100):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    n = math.sqrt(gm / a ** 3)
    xo, yo = a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E)
    fac = n * a / (1 - e * math.cos(E))
    return rot(xo, yo, -fac * math.sin(E), fac * math.sqrt(1 - e * e) * math.cos(E), inc, node,
               peri)


def _hyper_state(gm, a, e, inc, node, peri, M):
    """Hyperbolic state (a < 0): Newton on e sinh F - F = M in numpy."""
    F = math.asinh(M / e)
    for _ in range(100):
        F -= (e * math.sinh(F) - F - M) / (e * math.cosh(F) - 1)
    A = -a
    n = math.sqrt(gm / A ** 3)
    xo, yo = A * (e - math.cosh(F)), A * math.sqrt(e * e - 1) * math.sinh(F)
    fac = n * A / (e * math.cosh(F) - 1)
    return rot(xo, yo, -fac * math.sinh(F), fac * math.sqrt(e * e - 1) * math.cosh(F), inc, node,
               peri)


def test_elements_round_trip_elliptic():
    rng = np.random.default_rng(11)
    k = 200
    a = rng.uniform(0.5, 30, k)
    e = rng.uniform(0.01, 0.95, k)
    inc = rng.uniform(0.01, 3.1, k)
    node, peri, M = (rng.uniform(0, TWO_PI, k) for _ in range(3))
    xv = np.stack([_kepler_state(MU0, *v) for v in zip(a, e, inc, node, peri, M)], axis=1)
    el = orc.elements(MU0, xv)
    assert np.max(np.abs(el[0] - a * (1 - e)) / (a * (1 - e))) <= 1e-12
    assert np.max(np.abs(el[1] - e)) <= 1e-13
    assert np.max(np.abs(el[2] - inc)) <= 1e-12
    assert np.max(angdiff(el[4], node)) <= 1e-12
    assert np.max(angdiff(el[3], node + peri)) <= 1e-10
    assert np.max(angdiff(el[5], M)) <= 1e-10


def test_elements_round_trip_hyperbolic():
    rng = np.random.default_rng(12)
    k = 100
    e = rng.uniform(1.05, 3.0, k)
    q = rng.uniform(0.5, 10, k)
    a = q / (1 - e)
    inc = rng.uniform(0.01, 3.1, k)
    node, peri = (rng.uniform(0, TWO_PI, k) for _ in range(2))
    M = rng.uniform(-5, 5, k)
    xv = np.stack([_hyper_state(MU0, *v) for v in zip(a, e, inc, node, peri, M)], axis=1)
    el = orc.elements(MU0, xv)
    assert np.max(np.abs(el[0] - q) / q) <= 1e-12
    assert np.max(np.abs(el[1] - e)) <= 1e-12
    assert np.max(np.abs(el[2] - inc)) <= 1e-12
    assert np.max(angdiff(el[3], node + peri)) <= 1e-10
    assert np.max(np.abs(el[5] - M) / np.maximum(1, np.abs(M))) <= 1e-10


def test_equatorial_and_retrograde_conventions():
    """Orbits in the reference plane have Omega = 0 and varpi measured from x;
    a retrograde equatorial orbit has i = pi."""
    gm = MU0
    pro = rot(1.5, 0.0, 0.0, math.sqrt(gm * 1.2 / 1.5), 0.0, 0.0, 0.7)[:, None]
    el = orc.elements(gm, pro)[:, 0]
    assert el[2] == 0.0 and el[4] == 0.0 and angdiff(el[3], 0.7) <= 1e-14
    retro = pro.copy()
    retro[3:] *= -1.0
    el = orc.elements(gm, retro)[:, 0]
    assert abs(el[2] - math.pi) <= 1e-15 and abs(el[1] - 0.2) <= 1e-14


@pytest.mark.parametrize("e", [0.3, 2.0])
def test_mean_anomaly_advances_at_mean_motion(e):
    """Along the exact two-body flow (the oracle's pinned Kepler drift) q, e,
    i, varpi and Omega stay fixed and M advances by n t, n = sqrt(gm/|a|^3)."""
    gm = MU0
    q = 1.7
    xv0 = rot(q, 0.0, 0.0, math.sqrt(gm * (1 + e) / q), 0.3, 0.5, 1.2)[:, None]
    p = params()
    t = 37.0
    xv1, _ = orc.drift(p, xv0, t)
    e0, e1 = orc.elements(gm, xv0)[:, 0], orc.elements(gm, xv1)[:, 0]
    assert np.max(np.abs(e1[:3] - e0[:3])) <= 1e-12
    assert angdiff(e1[3], e0[3]) <= 1e-11 and angdiff(e1[4], e0[4]) <= 1e-12
    n = math.sqrt(gm / abs(q / (1 - e)) ** 3)
    dM = e1[5] - e0[5]
    if e < 1:
        assert angdiff(dM, n * t) <= 1e-11
    else:
        assert abs(dM - n * t) <= 1e-11 * n * t


def test_parabolic_barker_anomaly():
    """A parabola (gm = 1, q = 1/2) at true anomaly 90 degrees: x = (0, 1, 0),
    v = (-1, 1, 0) give e = 1 exactly, q = 1/2 and Barker's D = tan(f/2) = 1,
    so M = D + D^3/3 = 4/3; at pericentre M = 0."""
    el = orc.elements(1.0, np.array([[0.0], [1.0], [0.0], [-1.0], [1.0], [0.0]]))[:, 0]
    assert el[1] == 1.0 and el[0] == 0.5 and el[2] == 0.0
    assert abs(el[5] - 4.0 / 3.0) <= 1e-15 and angdiff(el[3], 0.0) <= 1e-15
    el = orc.elements(1.0, np.array([[0.5], [0.0], [0.0], [0.0], [2.0], [0.0]]))[:, 0]
    assert el[1] == 1.0 and el[5] == 0.0


def test_unbound_iff_eccentricity_at_least_one():
    """e >= 1 exactly when the orbital energy v^2/2 - gm/r is >= 0 (away from
    the rounding band), and e^2 = 1 + p (v^2/gm - 2/r)."""
    rng = np.random.default_rng(13)
    k = 2000
    x = rng.normal(size=(3, k)) * 5
    r = np.linalg.norm(x, axis=0)
    vesc = np.sqrt(2 * MU0 / r)
    v = rng.normal(size=(3, k))
    v *= vesc * rng.uniform(0.2, 1.8, k) / np.linalg.norm(v, axis=0)
    xv = np.concatenate([x, v])
    el = orc.elements(MU0, xv)
    eps = 0.5 * np.sum(v * v, axis=0) - MU0 / r
    keep = np.abs(eps) > 1e-12 * MU0 / r
    assert np.array_equal(el[1][keep] >= 1.0, eps[keep] >= 0)
    h2 = np.sum(np.cross(x.T, v.T) ** 2, axis=1)
    e2 = 1 + h2 / MU0 * (np.sum(v * v, axis=0) / MU0 - 2 / r)
    assert np.max(np.abs(el[1] ** 2 - e2)) <= 1e-12 * np.max(np.abs(e2))


# ------------------------------------------------------------------- ejection
def _scatter(nsmall=400, eject_every=5, seed=5):
    w = W.scatter_2giant(seed=seed, nsmall=nsmall, eject_every=eject_every)
    p = orc.make_params(w.params)
    xv, mu, rc = orc.init(p, w.nbig, w.nsmall, w.m_big, w.xv_helio)
    return w, p, xv, mu, rc


def _helio_e(p, nbig, xv, mu):
    P = orc.momentum(nbig, xv, mu)
    vh = xv[3:] + P[:, None] / (p.G * p.m_star)
    gm = np.full(xv.shape[1], p.G * p.m_star)
    gm[:nbig] += mu[:nbig]
    return orc.elements(gm, np.concatenate([xv[:3], vh]))[1]


def test_eject_test_flags_exactly_the_unbound():
    """One ejection test: the bodies removed are those whose heliocentric e,
    computed here from the momentum and the elements, is >= 1; massive ones
    lose their mass; nothing else changes."""
    w, p, xv, mu, rc = _scatter()
    e = _helio_e(p, w.nbig, xv, mu)
    mu2, stat, k = orc.eject(p, w.nbig, xv, mu)
    assert k == int(np.sum(e >= 1)) and k > w.nsmall // 4
    assert np.array_equal(stat == -3, e >= 1) and set(np.unique(stat)) <= {0, -3}
    assert np.array_equal(mu2, np.where(e >= 1, 0.0, mu))
    # a second test removes nobody new
    _, stat2, k2 = orc.eject(p, w.nbig, xv, mu2, stat)
    assert k2 == 0 and np.array_equal(stat2, stat)


def test_eject_schedule_and_frozen_state():
    """With eject_every = 5 nobody is removed in the first 4 steps; a body
    removed after step 5 keeps its step-5 state; the bodies left move exactly
    as in a run without the test (removed planetesimals are massless)."""
    w, p, xv, mu, rc = _scatter(eject_every=5)
    x4, mu4, st4, _, _ = orc.step_ex(p, w.nbig, xv, mu, rc, None, None, 4)
    assert not st4.any()
    x5, mu5, st5, _, _ = orc.step_ex(p, w.nbig, xv, mu, rc, None, None, 5)
    gone = st5 == -3
    assert gone.sum() > w.nsmall // 4 and not gone[:w.nbig].any()
    x12, _, st12, _, _ = orc.step_ex(p, w.nbig, xv, mu, rc, None, None, 12)
    assert np.array_equal(x12[:, gone], x5[:, gone])
    assert np.all(st12[gone] == -3)
    p0 = params(eject_every=0)
    ref, _, _, _ = orc.step(p0, w.nbig, xv, mu, rc, None, None, 12)
    keep = st12 == 0
    assert np.array_equal(x12[:, keep], ref[:, keep])


def test_step_index_sets_the_schedule():
    """The test follows steps whose global index is a multiple of eject_every:
    from step0 = 3, the first test comes after 2 steps."""
    w, p, xv, mu, rc = _scatter(eject_every=5)
    _, _, st1, _, _ = orc.step_ex(p, w.nbig, xv, mu, rc, None, None, 1, step0=3)
    _, _, st2, _, _ = orc.step_ex(p, w.nbig, xv, mu, rc, None, None, 2, step0=3)
    assert not st1.any() and (st2 == -3).sum() > w.nsmall // 4


def test_removed_massive_body_takes_no_part():
    """A giant on an unbound orbit is removed at the first test.  From then on
    the other bodies move exactly as in a system where that body is absent."""
    w, p, xv, mu, rc = _scatter(nsmall=200, eject_every=1)
    # a third massive body, 1 Earth mass, unbound: e = 1.4 from q = 20 AU
    xb = W.pericentre_to_xv(MU0, 20.0, 1.4, 0.1, 0.2, 0.3)
    m3 = 3.0e-6
    xh = np.concatenate([w.xv_helio[:, :2], xb[:, None], w.xv_helio[:, 2:]], axis=1)
    mb = np.concatenate([w.m_big, [m3]])
    x0, mu0, rc0 = orc.init(p, 3, w.nsmall, mb, xh)
    x1, mu1, st1, _, _ = orc.step_ex(p, 3, x0, mu0, rc0, None, None, 1)
    assert st1[2] == -3 and mu1[2] == 0.0
    x9, mu9, st9, _, _ = orc.step_ex(p, 3, x1, mu1, rc0, None, None, 8, stat=st1, step0=1)
    # the same state without the removed body, as a 2-giant system
    keep = np.ones(x1.shape[1], dtype=bool)
    keep[2] = False
    y9, _, sty, _, _ = orc.step_ex(p, 2, x1[:, keep], mu1[keep], rc0[keep], None, None, 8,
                                stat=st1[keep], step0=1)
    assert np.array_equal(x9[:, keep], y9)
    assert np.array_equal(st9[keep], sty)
    assert np.array_equal(x9[:, 2], x1[:, 2])
    # the energy of the massive bodies no longer counts it
    E9, _ = orc.energy(p, 3, x9, mu9)
    Ey, _ = orc.energy(p, 2, y9, mu1[keep])
    assert E9 == Ey
