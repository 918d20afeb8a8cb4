"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: references are closed forms,
hand-derived values (tests/golden/closed_forms.json), library routines
(mpmath, scipy's DOP853), or invariants of the exact flow.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_2601_16791_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
K = W.GAUSS_K
MU0 = W.G


def rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def params(dt=8.0, gas=False, **kw):
    p = W.default_params(dt, W.default_gas(gas))
    p.update(kw)
    return orc.make_params(p)


# ------------------------------------------------------- disk gravity (Eqs. 10-12)
def _dg_params(gamma=1.0, r_in=0.5, sigma1=1700.0, enabled=True):
    g = W.default_gas(True, sigma1=sigma1, gamma=gamma, disk_gravity=enabled)
    g["r_in_au"] = r_in
    return orc.make_params(W.default_params(10.0, g))


@pytest.mark.parametrize("gamma", [0.3, 0.5, 0.8, 1.2, 1.5, 1.9])
def test_disk_gravity_series_vs_mpmath(gamma):
    """Eq. 10's series S(gamma), summed by mpmath's own convergence acceleration."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    g = mp.mpf(gamma)
    term = lambda n: ((mp.binomial(2 * n, n) / mp.mpf(4) ** n) ** 2 * (1 - g) * (4 * n + 1)
                      / ((2 * n + 2 - g) * (2 * n - 1 + g)))
    ref = float(mp.nsum(term, [0, mp.inf]))
    assert abs(orc.dg_series(gamma) - ref) <= 2e-15 * abs(ref)


@pytest.mark.parametrize("gamma", [0.3, 0.8, 1.5, 1.9])
def test_disk_gravity_series_derivative_vs_mpmath(gamma):
    """dS/dgamma, which the oracle's forward derivative carries through the
    disk's gravity, against mpmath's numerical derivative of its own sum of
    Eq. 10's series."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30

    def S(g):
        term = lambda n: ((mp.binomial(2 * n, n) / mp.mpf(4) ** n) ** 2 * (1 - g) * (4 * n + 1)
                          / ((2 * n + 2 - g) * (2 * n - 1 + g)))
        return mp.nsum(term, [0, mp.inf])
    ref = float(mp.diff(S, mp.mpf(gamma)))
    assert abs(orc.dg_series_dgamma(gamma) - ref) <= 1e-12 * abs(ref)


def test_disk_gravity_units_against_cgs():
    """2 pi G Sigma for Sigma = 1700 g/cm^2 at 1 AU, gamma = 1.5 (force = that x S),
    computed in CGS (G = 6.6743e-8) and converted to AU/day^2: the Gaussian units
    and the solar mass agree with CGS to ~1e-4."""
    p = _dg_params(gamma=1.5, r_in=0.0)
    a = orc.disk_gravity(p, [1.0, 0.0, 0.0])
    cgs = 2 * math.pi * 6.6743e-8 * 1700.0 * orc.dg_series(1.5)          # cm/s^2
    ref = cgs * 86400.0 ** 2 / 1.495978707e13                              # AU/d^2
    assert abs(a[0] - ref) <= 2e-4 * abs(ref) and a[1] == 0.0 and a[2] == 0.0


def test_disk_gravity_geometry_and_scalings():
    """Radial in the plane, zero inside R_in and when off, independent of z,
    outward for the gamma = 1 edge term (Eq. 12) and inward for gamma != 1
    (S < 0), proportional to Sigma1, and for gamma = 1 to R_in / R^2."""
    p = _dg_params(gamma=1.0, r_in=0.5)
    a1 = orc.disk_gravity(p, [3.0, 4.0, 0.0])           # R = 5
    assert a1[2] == 0.0 and a1[0] > 0 and abs(a1[0] / a1[1] - 0.75) < 1e-15
    assert np.allclose(orc.disk_gravity(p, [3.0, 4.0, 0.3]), a1, rtol=1e-15, atol=0)
    assert np.all(orc.disk_gravity(p, [0.3, 0.1, 0.0]) == 0.0)              # R < R_in
    assert np.all(orc.disk_gravity(_dg_params(enabled=False), [3.0, 4.0, 0.0]) == 0.0)
    a2 = orc.disk_gravity(p, [6.0, 8.0, 0.0])           # R = 10
    assert abs(np.linalg.norm(a1) / np.linalg.norm(a2) - 4.0) < 1e-13
    a3 = orc.disk_gravity(_dg_params(gamma=1.0, r_in=1.0), [3.0, 4.0, 0.0])
    assert abs(np.linalg.norm(a3) / np.linalg.norm(a1) - 2.0) < 1e-13
    a4 = orc.disk_gravity(_dg_params(gamma=1.0, r_in=0.5, sigma1=850.0), [3.0, 4.0, 0.0])
    assert abs(np.linalg.norm(a1) / np.linalg.norm(a4) - 2.0) < 1e-13
    b = orc.disk_gravity(_dg_params(gamma=1.5, r_in=0.5), [3.0, 4.0, 0.0])
    assert b[0] < 0 and b[1] < 0
    b2 = orc.disk_gravity(_dg_params(gamma=1.5, r_in=0.5), [6.0, 8.0, 0.0])
    assert abs(np.linalg.norm(b) / np.linalg.norm(b2) - 2.0 ** 1.5) < 1e-13    # Sigma ~ R^-1.5


# ------------------------------------------------------------ changeover K(r)
def test_changeover_endpoints_midpoint_symmetry():
    """Sec. 2.1.3 listing: K=1 for s >= rc, K=0 for s <= 0.1 rc, smooth between."""
    rc = 0.7
    assert orc.changeover(rc, rc) == 1.0
    assert orc.changeover(2.5 * rc, rc) == 1.0
    assert orc.changeover(0.1 * rc, rc) == 0.0
    assert orc.changeover(0.03 * rc, rc) == 0.0
    g = GOLDEN["changeover_midpoint"]
    assert abs(orc.changeover(g["s_over_rc"] * rc, rc) - g["K"]) < 1e-15
    # the quintic is the symmetric smooth step: K(q) + K(1 - q) = 1
    for q in (0.07, 0.23, 0.41):
        s1, s2 = 0.1 * rc + 0.9 * rc * q, 0.1 * rc + 0.9 * rc * (1 - q)
        assert abs(orc.changeover(s1, rc) + orc.changeover(s2, rc) - 1.0) < 1e-14


def test_changeover_c2_contact():
    """K and its first two derivatives vanish at q=0 and match 1 at q=1: K ~ 10 q^3 at both ends."""
    rc = 1.0
    for eps in (1e-3, 1e-4):
        k_lo = orc.changeover(0.1 + 0.9 * eps, rc)
        k_hi = orc.changeover(0.1 + 0.9 * (1 - eps), rc)
        assert abs(k_lo / (10 * eps ** 3) - 1) < 2e-2
        assert abs((1 - k_hi) / (10 * eps ** 3) - 1) < 2e-2


def test_k_over_s3_branches():
    rc = 1.0
    for s in (1.0, 1.3, 4.0):
        assert rel(orc.k_over_s3(s * s, rc), s ** -3) < 1e-15
    assert orc.k_over_s3(0.01, rc) == 0.0          # s^2 = 0.01 rc^2 is inside (inclusive)
    s = 0.55
    assert rel(orc.k_over_s3(s * s, rc), 0.5 / s ** 3) < 1e-14


# ---------------------------------------------------------------- gravity
def _random_cluster(rng, nbig, nsmall, spread=1.0):
    n = nbig + nsmall
    xv = np.zeros((6, n))
    xv[:3] = rng.normal(0, spread, (3, n)) + np.array([[5.0], [0.0], [0.0]])
    xv[3:] = rng.normal(0, 0.01, (3, n))
    mu = np.zeros(n)
    mu[:nbig] = MU0 * rng.uniform(1e-6, 1e-3, nbig)
    rc = np.zeros(n)
    rc[:nbig] = rng.uniform(0.2, 0.8, nbig)
    return xv, mu, rc


def test_gather_equals_triangular():
    """Sec. 2.1.3 prints both loops; they must give the same forces (to rounding)."""
    rng = np.random.default_rng(11)
    xv, mu, rc = _random_cluster(rng, 7, 120, spread=0.4)
    a1 = orc.accel_grav(7, xv, mu, rc, triangular=False)
    a2 = orc.accel_grav(7, xv, mu, rc, triangular=True)
    assert rel(a1, a2) < 1e-13
    # several pairs sit in the changeover zone, so K is exercised
    d = np.linalg.norm(xv[:3, None, :7] - xv[:3, :, None], axis=0)
    zone = (d > 0.1 * rc[None, :7]) & (d < rc[None, :7])
    assert zone.sum() > 5


def test_inverse_square_closed_form():
    mu = np.array([1e-3, 0.0])
    rc = np.array([0.5, 0.0])
    xv = np.zeros((6, 2))
    xv[0] = [1.0, 4.0]
    a = orc.accel_grav(1, xv, mu, rc)
    assert rel(a[0, 1], -1e-3 / 9.0) < 1e-15
    assert a[1, 1] == 0.0 and a[2, 1] == 0.0
    assert np.all(a[:, 0] == 0.0)                   # no self force, massless source
    xv[0, 1] = 1.0 + 0.55 * 0.5                     # changeover midpoint: half the force
    a = orc.accel_grav(1, xv, mu, rc)
    assert rel(a[0, 1], -0.5e-3 / (0.275 ** 2)) < 1e-14


# ------------------------------------------------------------------- gas
def test_drag_coefficient_golden_and_limits():
    g = GOLDEN["cd_re10_ma0"]
    assert abs(orc.drag_cd(g["Re"], g["Ma"], g["cd_mode"]) - g["C_D"]) < 1e-14
    # Stokes: C_D Re / 24 -> 1
    assert abs(orc.drag_cd(1e-7, 0.0) * 1e-7 / 24 - 1) < 1e-6
    # printed exponent -2 gives (24/Re)^2 instead
    assert abs(orc.drag_cd(1e-4, 0.0, 1) / (24e4) ** 2 - 1) < 1e-4
    # Newton regime: C_D -> k = 0.2 above Re = 1e5
    assert abs(orc.drag_cd(1e13, 0.0) - 0.2) < 1e-10
    # supersonic: C_D -> 2
    assert abs(orc.drag_cd(1e6, 1e12) - 2.0) < 1e-9
    # the k switch
    jump = orc.drag_cd(1e5 * (1 - 1e-12), 0.0) - orc.drag_cd(1e5, 0.0)
    assert abs(jump - GOLDEN["cd_switch_jump"]["jump"]) < 1e-9


@pytest.mark.parametrize("key", ["disk_1au", "disk_16au"])
def test_disk_hand_values(key):
    g = GOLDEN[key]
    p = params(10.0, gas=True)
    d = orc.gas_state(p, g["R"])
    for f in ("sigma", "hr", "vk", "eta"):
        assert rel(d[f], g[f]) < 1e-13, f
    if "rho_g" in g:
        assert rel(d["rho_g"], g["rho_g"]) < 1e-13
        assert rel(d["vg"], g["vg"]) < 1e-13


def _disk_nu_cgs(d):
    """Kinematic viscosity (cm^2/s) from the Brasser et al. definitions."""
    au_cm, day_s = 1.495978707e13, 86400.0
    lam = 2.34 * 1.6735575e-24 / (2e-15 * d["rho_g"])
    cs = d["cs"] * au_cm / day_s
    return 0.5 * math.sqrt(8 / math.pi) * cs * lam


def test_drag_zero_when_comoving_and_direction():
    p = params(10.0, gas=True)
    R = 3.0
    d = orc.gas_state(p, R)
    x = np.array([R, 0.0, 0.0])
    acc, _, _ = orc.drag_one(p, x, np.array([0.0, d["vg"], 0.0]), 10.0, 2.0)
    assert np.all(acc == 0.0)
    # circular Keplerian orbit is faster than the gas: drag points backwards (-phi)
    acc, re, ma = orc.drag_one(p, x, np.array([0.0, d["vk"], 0.0]), 10.0, 2.0)
    assert acc[1] < 0 and acc[0] == 0.0 and acc[2] == 0.0


def test_drag_stokes_law():
    """Re << 1, Ma -> 0: Eq. 3 with C_D = 24/Re is Stokes' law a = 9 rho_g nu dv / (2 r_p^2 rho_p)."""
    p = params(10.0, gas=True)
    R = 2.0
    d = orc.gas_state(p, R)
    au_cm, day_s = 1.495978707e13, 86400.0
    dv_cgs = 1e-3                                   # 10 micron/s relative speed
    dv = dv_cgs * day_s / au_cm
    rp_km, rho = 1.0, 2.0
    acc, re, ma = orc.drag_one(p, np.array([R, 0.0, 0.0]), np.array([0.0, d["vg"] + dv, 0.0]),
                               rp_km, rho)
    assert re < 1e-2
    nu = _disk_nu_cgs(d)
    rp_cm = rp_km * 1e5
    stokes_cgs = 4.5 * d["rho_g"] * nu * dv_cgs / (rp_cm ** 2 * rho)
    stokes = stokes_cgs * day_s ** 2 / au_cm
    assert abs(-acc[1] / stokes - 1) < 1e-3
    # dv enters as (v_g + dv) - v_g, which keeps only ~6 digits of a 1e-13 AU/d speed
    assert abs(re - 2 * rp_cm * dv_cgs / nu) / re < 1e-5


def test_drag_quadratic_law():
    """Re >> 1e5, Ma << 1: C_D -> 0.2 and a -> (3/8)(0.2/r_p)(rho_g/rho_p) dv^2."""
    p = params(10.0, gas=True)
    R = 1.0
    d = orc.gas_state(p, R)
    dv = 2e-5 * d["vk"]
    rp_km, rho = 3.0e4, 3.0
    acc, re, ma = orc.drag_one(p, np.array([R, 0.0, 0.0]), np.array([0.0, d["vg"] + dv, 0.0]),
                               rp_km, rho)
    assert re > 1e6 and ma < 1e-3
    quad = 0.375 * 0.2 / (rp_km / 1.495978707e8) * (d["rho_g"] / rho) * dv * dv
    assert abs(-acc[1] / quad - 1) < 1e-2


# ----------------------------------------------------------------- Stumpff
def test_stumpff_vs_closed_forms():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for z in (1e-9, 0.05, 0.3, 2.0, 17.0, 60.0, -0.2, -3.0, -25.0):
        c = orc.stumpff(z)
        zz = mp.mpf(z)
        if z > 0:
            r = mp.sqrt(zz)
            ref = [mp.cos(r), mp.sin(r) / r, (1 - mp.cos(r)) / zz, (r - mp.sin(r)) / r ** 3]
        else:
            r = mp.sqrt(-zz)
            ref = [mp.cosh(r), mp.sinh(r) / r, (mp.cosh(r) - 1) / (-zz), (mp.sinh(r) - r) / r ** 3]
        for k in range(4):
            tol = 1e-14 * max(1.0, abs(z)) ** 1.5
            assert abs(c[k] - float(ref[k])) <= tol * max(abs(float(ref[k])), 1e-2), (z, k)


# ------------------------------------------------------------ Kepler drift
def _kepler_ref(gm, x0, v0, t):
    """Two-body propagation through the classical anomalies, in mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x = [mp.mpf(float(a)) for a in x0]
    v = [mp.mpf(float(a)) for a in v0]
    gm = mp.mpf(gm)
    r = mp.sqrt(sum(a * a for a in x))
    v2 = sum(a * a for a in v)
    rv = sum(a * b for a, b in zip(x, v))
    a = 1 / (2 / r - v2 / gm)
    hvec = [x[1] * v[2] - x[2] * v[1], x[2] * v[0] - x[0] * v[2], x[0] * v[1] - x[1] * v[0]]
    if a > 0:
        n = mp.sqrt(gm / a ** 3)
        ecosE, esinE = 1 - r / a, rv / mp.sqrt(gm * a)
        E0 = mp.atan2(esinE, ecosE)
        e = mp.sqrt(ecosE ** 2 + esinE ** 2)
        M1 = E0 - e * mp.sin(E0) + n * t
        E1 = mp.findroot(lambda E: E - e * mp.sin(E) - M1, M1)
        dE = E1 - E0
        f = 1 - a / r * (1 - mp.cos(dE))
        g = t - (dE - mp.sin(dE)) / n
        r1 = a * (1 - e * mp.cos(E1))
        fd = -mp.sqrt(gm * a) / (r * r1) * mp.sin(dE)
        gd = 1 - a / r1 * (1 - mp.cos(dE))
    else:
        n = mp.sqrt(gm / (-a) ** 3)
        ecoshF, esinhF = 1 - r / a, rv / mp.sqrt(-gm * a)
        F0 = mp.atanh(esinhF / ecoshF)
        e = mp.sqrt(ecoshF ** 2 - esinhF ** 2)
        M1 = e * mp.sinh(F0) - F0 + n * t
        F1 = mp.findroot(lambda F: e * mp.sinh(F) - F - M1, F0 + n * t / e)
        dF = F1 - F0
        f = 1 - a / r * (1 - mp.cosh(dF))
        g = t - (mp.sinh(dF) - dF) / n
        r1 = a * (1 - e * mp.cosh(F1))
        fd = -mp.sqrt(-gm * a) / (r * r1) * mp.sinh(dF)
        gd = 1 - a / r1 * (1 - mp.cosh(dF))
    del hvec
    xn = [float(f * x[k] + g * v[k]) for k in range(3)]
    vn = [float(fd * x[k] + gd * v[k]) for k in range(3)]
    return np.array(xn + vn)


@pytest.mark.parametrize("case", ["circular", "eccentric", "inclined", "hyperbolic"])
def test_drift_vs_classical_anomaly_solution(case):
    p = params(8.0)
    rng = np.random.default_rng(3)
    if case == "circular":
        xv = W.elements_to_xv(MU0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.3)
    elif case == "eccentric":
        xv = W.elements_to_xv(MU0, 5.2, 0.6, 0.1, 1.0, 2.0, 2.5)
    elif case == "inclined":
        xv = W.elements_to_xv(MU0, 0.7, 0.2, 1.2, 0.4, 5.0, 4.0)
    else:
        xv = np.array([1.0, 0.2, 0.05, 0.001, 0.03, 0.002])
    for h in (8.0, 37.0, -5.0, 400.0):
        out, it = orc.drift(p, xv.reshape(6, 1), h)
        ref = _kepler_ref(MU0, xv[:3], xv[3:], h)
        assert rel(out[:3, 0], ref[:3]) < 2e-14, (case, h)
        assert rel(out[3:, 0], ref[3:]) < 2e-14, (case, h)
        assert it < 64                             # converged below the cap
    del rng


def test_drift_one_orbit_closes_and_reverses():
    p = params(8.0)
    a = 2.3
    xv = W.elements_to_xv(MU0, a, 0.3, 0.2, 0.1, 0.5, 1.0).reshape(6, 1)
    period = 2 * math.pi * math.sqrt(a ** 3 / MU0)
    nstep = 37
    cur = xv.copy()
    for _ in range(nstep):
        cur, _ = orc.drift(p, cur, period / nstep)
    assert rel(cur[:3], xv[:3]) < 1e-13
    assert rel(cur[3:], xv[3:]) < 1e-13
    fwd, _ = orc.drift(p, xv, 13.0)
    back, _ = orc.drift(p, fwd, -13.0)
    assert rel(back, xv) < 1e-15 * 10


# ------------------------------------------------------------- detection
def test_hermite_exact_for_straight_lines():
    """Straight relative motion makes d^2(t) quadratic; the cubic reading reproduces it exactly."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        dx0 = rng.normal(0, 1, 3)
        dv = rng.normal(0, 1, 3)
        tstar = -dx0 @ dv / (dv @ dv)
        h = abs(tstar) * rng.uniform(1.2, 3.0)
        if tstar <= 0:
            dv = -dv
            tstar = -tstar
        dx1 = dx0 + dv * h
        d0, d1 = dx0 @ dx0, dx1 @ dx1
        got = orc.hermite_d2min(d0, d1, 2 * dx0 @ dv, 2 * dx1 @ dv, h)
        perp = np.linalg.norm(np.cross(dx0, dv)) ** 2 / (dv @ dv)
        assert abs(got - perp) <= 1e-12 * d0
    # separating at the start, or approaching at the end: no interior minimum
    assert math.isinf(orc.hermite_d2min(1.0, 2.0, 0.5, 1.0, 1.0))
    assert math.isinf(orc.hermite_d2min(2.0, 1.0, -1.0, -0.5, 1.0))


def test_detect_flybys():
    """Flag iff the closest approach of a straight fly-by is within rc (Sec. 2.1.2 mce_snif)."""
    p = params(dt=2.0)
    rc_big = 0.5
    impact = [0.3, 0.49, 0.51, 0.8, 0.45]
    n = 1 + len(impact)
    xv0 = np.zeros((6, n))
    xv1 = np.zeros((6, n))
    xv0[0, 0] = xv1[0, 0] = 10.0                    # big at rest at (10, 0, 0)
    for k, b in enumerate(impact):
        j = k + 1
        x0 = np.array([10.0 - 1.0, b, 0.0])
        v = np.array([1.0, 0.0, 0.0])              # crosses x = 10 at t = 1 (mid-step)
        xv0[:3, j], xv0[3:, j] = x0, v
        xv1[:3, j], xv1[3:, j] = x0 + 2.0 * v, v
    rcrit = np.zeros(n)
    rcrit[0] = rc_big
    flags, pairs = orc.detect(p, 1, xv0, xv1, rcrit)
    want = [j + 1 for j, b in enumerate(impact) if b <= rc_big]
    assert sorted(pairs[:, 1].tolist()) == want
    assert np.all(pairs[:, 0] == 0)
    assert flags[0] == 1 and all(flags[j] == (1 if j in want else 0) for j in range(1, n))


# ------------------------------------------------------------ Bulirsch-Stoer
def test_bs_single_body_is_kepler():
    p = params(8.0)
    xv = W.elements_to_xv(MU0, 1.5, 0.2, 0.1, 0.2, 0.3, 0.4).reshape(6, 1)
    out, nsub = orc.bs_group(p, np.zeros(1), np.zeros(1), xv, 40.0)
    ref = _kepler_ref(MU0, xv[:3, 0], xv[3:, 0], 40.0)
    assert rel(out[:3, 0], ref[:3]) < 1e-11
    assert rel(out[3:, 0], ref[3:]) < 1e-11


def _nbody_rhs(gm_star, mus):
    """Heliocentric N-body equations (textbook form with the indirect term)."""
    mus = np.asarray(mus)

    def rhs(t, y):
        n = len(mus)
        x = y[:3 * n].reshape(3, n)
        v = y[3 * n:].reshape(3, n)
        r = np.linalg.norm(x, axis=0)
        a = -(gm_star + mus) * x / r ** 3
        for j in range(n):
            if mus[j] == 0.0:
                continue
            for i in range(n):
                if i == j:
                    continue
                d = x[:, j] - x[:, i]
                a[:, i] += mus[j] * (d / np.linalg.norm(d) ** 3 - x[:, j] / r[j] ** 3)
        return np.concatenate([v.ravel(), a.ravel()])
    return rhs


def test_bs_deep_encounter_vs_dop853():
    """Inside 0.1 rc the (1-K) weight is 1: BS must follow the plain three-body motion."""
    from scipy.integrate import solve_ivp
    p = params(8.0)
    mu_big = MU0 * 1e-3
    xb = W.elements_to_xv(MU0, 5.2, 0.0, 0.0, 0.0, 0.0, 0.0)
    xs = xb.copy()
    xs[1] += 0.02                                  # 0.02 AU from the planet, rc ~ 1 AU
    xs[3] += np.sqrt(mu_big / 0.02)                # on a planetocentric circular orbit
    xv = np.stack([xb, xs], axis=1)
    # The group integrates in DH variables: star's pull -mu0 x/r^3 on every body
    # plus the pair force; with mu_small = 0 the big body is a pure Kepler orbit.
    rcrit = np.array([1.0, 0.0])
    out, _ = orc.bs_group(p, np.array([mu_big, 0.0]), rcrit, xv, 8.0)

    def rhs(t, y):
        x = y[:6].reshape(3, 2)
        a = -MU0 * x / np.linalg.norm(x, axis=0) ** 3
        d = x[:, 1] - x[:, 0]
        a[:, 1] -= mu_big * d / np.linalg.norm(d) ** 3
        return np.concatenate([y[6:], a.ravel()])
    y0 = np.concatenate([xv[:3].ravel(), xv[3:].ravel()])
    sol = solve_ivp(rhs, (0, 8.0), y0, method="DOP853", rtol=1e-13, atol=1e-16)
    ref = sol.y[:, -1]
    assert rel(out[:3].ravel(), ref[:6]) < 1e-10
    assert rel(out[3:].ravel(), ref[6:]) < 1e-9


# --------------------------------------------------------------- full step
def _two_giants():
    w = W.plain_2big_1k(nsmall=0)
    return w


def test_energy_bounded_and_angular_momentum_conserved():
    w = _two_giants()
    p = orc.make_params(w.params)
    xv, mu, rc = orc.init(p, 2, 0, w.m_big, w.xv_helio)
    E0, L0 = orc.energy(p, 2, xv, mu)
    errs = []
    for _ in range(40):
        xv, _, _, st = orc.step(p, 2, xv, mu, rc, None, None, 100)
        E, L = orc.energy(p, 2, xv, mu)
        errs.append(abs(E / E0 - 1))
        assert rel(L, L0) < 2e-13
    errs = np.array(errs)
    assert errs.max() < 1e-6
    # no secular drift: the second half is no worse than the first
    assert errs[20:].max() < 3 * errs[:20].max() + 1e-12


def test_time_reversibility():
    w = W.plain_2big_1k(nsmall=60)
    p = orc.make_params(w.params)
    xv, mu, rc = orc.init(p, 2, 60, w.m_big, w.xv_helio)
    fwd, ever, _, st = orc.step(p, 2, xv, mu, rc, None, None, 30)
    pb = orc.make_params(dict(w.params, dt=-w.params["dt"]))
    back, ever2, _, st2 = orc.step(pb, 2, fwd, mu, rc, None, None, 30)
    keep = (ever == 0) & (ever2 == 0)
    assert keep.sum() > 40
    if st[0] == 0 and st2[0] == 0:
        assert rel(back, xv) < 1e-13
    d = np.abs(back - xv)[:, keep].max() / np.abs(xv).max()
    assert d < 1e-13


def test_massless_bodies_do_not_act():
    w = W.plain_2big_1k(nsmall=50)
    p = orc.make_params(w.params)
    xv, mu, rc = orc.init(p, 2, 50, w.m_big, w.xv_helio)
    full, _, _, _ = orc.step(p, 2, xv, mu, rc, None, None, 25)
    only, _, _, _ = orc.step(p, 2, xv[:, :2].copy(), mu[:2], rc[:2], None, None, 25)
    assert np.array_equal(full[:, :2], only)
    E1, L1 = orc.energy(p, 2, full, mu)
    E2, L2 = orc.energy(p, 2, only, mu[:2])
    assert E1 == E2 and np.array_equal(L1, L2)


def test_init_readout_round_trip():
    w = W.plain_2big_1k(nsmall=30)
    p = orc.make_params(w.params)
    xv, mu, rc = orc.init(p, 2, 30, w.m_big, w.xv_helio)
    back = orc.readout(p, 2, 30, mu, xv)
    assert rel(back, w.xv_helio) < 1e-15
    # changeover radii: 3 Hill radii of Jupiter and Saturn, about 1.07 and 1.30 AU
    assert abs(rc[0] - 1.07) < 0.03 and abs(rc[1] - 1.30) < 0.03
    assert np.all(rc[2:] == 0.0)


def _hybrid_vs_dop853(mus_big, xv_helio, nsteps, h, tol):
    from scipy.integrate import solve_ivp
    nbig = len(mus_big)
    n = xv_helio.shape[1]
    cfg = W.default_params(h)
    p = orc.make_params(cfg)
    m_big = np.asarray(mus_big) / W.G
    xv, mu, rc = orc.init(p, nbig, n - nbig, m_big, xv_helio)
    out, ever, _, st = orc.step(p, nbig, xv, mu, rc, None, None, nsteps)
    hel = orc.readout(p, nbig, n - nbig, mu, out)
    mus = np.concatenate([np.asarray(mus_big), np.zeros(n - nbig)])
    y0 = np.concatenate([xv_helio[:3].ravel(), xv_helio[3:].ravel()])
    sol = solve_ivp(_nbody_rhs(MU0, mus), (0, nsteps * h), y0, method="DOP853",
                    rtol=1e-13, atol=1e-15)
    ref = sol.y[:, -1]
    refx = ref[:3 * n].reshape(3, n)
    err = np.linalg.norm(hel[:3] - refx, axis=0) / np.linalg.norm(refx, axis=0)
    return err, st


def test_hybrid_matches_brute_force_few_body():
    """Sun + 2 giants + 2 test particles, no encounters: O(h^2) agreement with DOP853."""
    w = W.plain_2big_1k(nsmall=2, seed=7)
    mus = W.G * w.m_big
    err, st = _hybrid_vs_dop853(mus, w.xv_helio, 400, 1.0, None)
    assert st[0] == 0
    assert err.max() < 2e-7


def test_hybrid_close_encounter_vs_brute_force():
    """A test particle passing through Jupiter's changeover zone: BS takes over (Sec. 2)."""
    mu_j = W.G * W.M_JUP
    xj = W.elements_to_xv(MU0 + mu_j, 5.2, 0.0, 0.0, 0.0, 0.0, 0.0)
    xs = W.elements_to_xv(MU0, 5.2, 0.0, 0.0, 0.0, 0.0, -0.12)   # trails Jupiter by ~0.6 AU
    xs[4] *= 0.985                                               # slower: Jupiter pulls away
    xv = np.stack([xj, xs], axis=1)
    err, st = _hybrid_vs_dop853([mu_j], xv, 300, 1.0, None)
    assert st[0] > 0 and st[1] > 0                               # pairs flagged, groups run
    assert err.max() < 1e-6


# ------------------------------------------------------ reference derivative
def test_jvp_matches_central_difference():
    w = W.gas_4core_100k(nsmall=24, nsteps=6)
    p = orc.make_params(w.params)
    rng = np.random.default_rng(2)
    wts = np.full(w.nsmall, 1.0 / w.nsmall)
    dxv = np.zeros((6, w.n))
    dxv[:3] = rng.normal(0, 1e-3, (3, w.n))
    dxv[3:] = rng.normal(0, 1e-5, (3, w.n))
    dpar = np.array([17.0, 0.01, 0.01])
    L, dL = orc.jvp_loss(p, w.nbig, w.m_big, w.xv_helio, w.rp_km, w.rhop, wts, w.nsteps, dxv, dpar)
    eps = 1e-4

    def loss_at(t):
        cfg = dict(w.params)
        gas = dict(cfg["gas"])
        gas["sigma1_gcm2"] += t * dpar[0]
        gas["gamma"] += t * dpar[1]
        gas["cd_scale"] += t * dpar[2]
        cfg["gas"] = gas
        pp = orc.make_params(cfg)
        Lt, _ = orc.jvp_loss(pp, w.nbig, w.m_big, w.xv_helio + t * dxv, w.rp_km, w.rhop, wts,
                             w.nsteps, np.zeros_like(dxv), np.zeros(3))
        return Lt
    fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
    assert abs(fd - dL) <= 1e-5 * abs(dL)
    assert L > 0


@pytest.mark.parametrize("gamma,r_in,dpar", [(1.5, 1.0, (0.0, 0.02, 0.0)),
                                              (1.5, 1.0, (17.0, 0.0, 0.0)),
                                              (1.0, 1.5, (17.0, 0.0, 0.0))])
def test_jvp_with_disk_gravity_matches_central_difference(gamma, r_in, dpar):
    """With the disk's gravity on (Eqs. 10-12): the derivative along gamma
    runs through Sigma and through S(gamma) (for gamma != 1; dropping dS/dgamma
    puts it 85% off here), the one along sigma1 through Sigma.  At gamma = 1 the
    force is the edge form of Eq. 12, a branch in gamma, so only sigma1 is
    checked there.  The loss runs its bodies' encounters through BS, whose
    step choices leave ~1e-6 of noise in the differences."""
    w = W.gas_4core_100k(nsmall=24, nsteps=6)
    w.params = dict(w.params, gas=dict(w.params["gas"], gamma=gamma, r_in_au=r_in,
                                       disk_gravity=True))
    p = orc.make_params(w.params)
    wts = np.full(w.nsmall, 1.0 / w.nsmall)
    dxv = np.zeros((6, w.n))
    dpar = np.array(dpar)
    L, dL = orc.jvp_loss(p, w.nbig, w.m_big, w.xv_helio, w.rp_km, w.rhop, wts, w.nsteps, dxv, dpar)

    def loss_at(t):
        gas = dict(w.params["gas"])
        gas["sigma1_gcm2"] += t * dpar[0]
        gas["gamma"] += t * dpar[1]
        pp = orc.make_params(dict(w.params, gas=gas))
        Lt, _ = orc.jvp_loss(pp, w.nbig, w.m_big, w.xv_helio, w.rp_km, w.rhop, wts, w.nsteps,
                             dxv, np.zeros(3))
        return Lt
    eps = 1e-2
    fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
    assert abs(fd - dL) <= 1e-5 * abs(dL), (fd, dL)
