"""Seeded synthetic inputs shaped like the paper's workloads.

This module feeds both the CUDA path and the CPU oracle and holds none of the
method's arithmetic: it only draws orbital elements from the stated
distributions and turns them into heliocentric Cartesian states with the
textbook two-body transform.  No dataset is involved; these draws stand in for
the paper's planetesimal disks (Sec. 4: giant planets growing inside extended,
gas-rich planetesimal disks).

Units: AU, day, solar mass.  States are ``6 x N`` float64 arrays (x, y, z, vx,
vy, vz rows) with the big bodies first.

Named workloads (sizes can be scaled down for tests with ``nbig=``/``nsmall=``):

* ``plain_2big_1k``: star, Jupiter at 5.2 AU and 0.3 Jupiter masses at
  9.5 AU (e=0.03, i=0.5 deg), 1,000 massless planetesimals with a~U[2,12] AU,
  e~Rayleigh(0.01), i~Rayleigh(0.005) rad; dt=8 d, 1,000 steps, no gas; seed 0.
* ``gas_4core_100k``: 4 cores of 10-30 Earth masses, a~U[3,10] AU, plus
  100,000 planetesimals, a~U[1,15] AU, radius log-uniform 1-100 km, density
  U[1,3] g/cm^3; gas Sigma=1700 g/cm^2 (r/AU)^-1, H/r=0.05 (r/AU)^0.25;
  dt=10 d, 10,000 steps; seed 1.
* ``semiactive_2000big_200k``: 2,000 bigs log-uniform between lunar and Mars
  mass and 200,000 massless bodies, a~U[0.5,4] AU, e~Rayleigh(0.02),
  i~Rayleigh(0.01); no gas; dt=6 d, 2,000 steps; seed 2.
* ``ensemble_256``: 256 independent systems, each with 2-50 big bodies
  (uniform integer) and 1,000-200,000 planetesimals (log-uniform) as in
  ``gas_4core_100k``, gas as there with Sigma scaled by U[0.3,3]; dt=10 d,
  1,000 steps; seed 3.  The big bodies' masses are not fixed by the
  workload's statement; they are drawn log-uniform between lunar and Mars
  mass with a~U[1,15] AU (embryos spread over the disk), so that a 50-body
  system is not an immediately unstable pile of giant cores.
* ``adjoint_4core_50k``: 4 cores + 50,000 planetesimals as in
  ``gas_4core_100k``; 2,000 steps checkpointed every 50; seed 4.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAUSS_K = 0.01720209895              # Gaussian gravitational constant
G = GAUSS_K * GAUSS_K                # AU^3 Msun^-1 d^-2
M_JUP = 9.547919e-4                  # Jupiter mass [Msun]
M_EARTH = 3.003489e-6                # Earth mass [Msun]
M_MOON = 3.69e-8                     # lunar mass [Msun]
M_MARS = 3.23e-7                     # Mars mass [Msun]


def default_gas(enabled=False, sigma1=1700.0, gamma=1.0, disk_gravity=False):
    return dict(sigma1_gcm2=sigma1, gamma=gamma, r_c_au=math.inf, r_in_au=0.0, hr_1au=0.05,
                flare=0.25, gamma_c=1.4, mu_mol=2.34, sigma_mol_cm2=2e-15, cd_scale=1.0,
                enabled=bool(enabled), cd_mode=0, disk_gravity=bool(disk_gravity))


def default_params(dt, gas=None, pair_cap=1 << 20):
    return dict(G=G, m_star=1.0, dt=float(dt), rcrit_hill=3.0, bs_tol=1e-12,
                kepler_max_iter=64, bs_max_sub=4096, pair_cap=int(pair_cap), eject_every=0,
                gas=gas if gas is not None else default_gas(False))


@dataclasses.dataclass
class Workload:
    name: str
    params: dict
    nbig: int
    nsmall: int
    m_big: np.ndarray          # [nbig] solar masses
    xv_helio: np.ndarray       # [6, n] heliocentric
    rp_km: np.ndarray          # [nsmall]
    rhop: np.ndarray           # [nsmall] g/cm^3
    nsteps: int
    checkpoint_every: int = 0
    # growth tracks of the massive bodies (Sec. 3.3), per-big arrays m0, mc,
    # mf [Msun], tau_c, tau_g [d], delta_r [AU], grows; None: fixed masses
    growth: dict = None
    gap_c: float = 4.0         # gap half-width in Hill radii (Eq. 8)

    @property
    def n(self):
        return self.nbig + self.nsmall


def elements_to_xv(gm, a, e, inc, node, peri, M):
    """Heliocentric state from Keplerian elements (elliptic orbits)."""
    gm, a, e, inc, node, peri, M = (np.asarray(v, dtype=np.float64) for v in
                                    np.broadcast_arrays(gm, a, e, inc, node, peri, M))
    E = M.copy()
    for _ in range(60):
        E = E - (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
    cE, sE = np.cos(E), np.sin(E)
    rt = np.sqrt(1.0 - e * e)
    n = np.sqrt(gm / a ** 3)
    xo = a * (cE - e)
    yo = a * rt * sE
    fac = n * a / (1.0 - e * cE)
    vxo = -fac * sE
    vyo = fac * rt * cE
    cO, sO = np.cos(node), np.sin(node)
    cw, sw = np.cos(peri), np.sin(peri)
    ci, si = np.cos(inc), np.sin(inc)
    r11 = cO * cw - sO * sw * ci
    r12 = -cO * sw - sO * cw * ci
    r21 = sO * cw + cO * sw * ci
    r22 = -sO * sw + cO * cw * ci
    r31 = sw * si
    r32 = cw * si
    out = np.empty((6,) + a.shape)
    out[0] = r11 * xo + r12 * yo
    out[1] = r21 * xo + r22 * yo
    out[2] = r31 * xo + r32 * yo
    out[3] = r11 * vxo + r12 * vyo
    out[4] = r21 * vxo + r22 * vyo
    out[5] = r31 * vxo + r32 * vyo
    return out


def pericentre_to_xv(gm, q, e, inc, node, peri):
    """Heliocentric state at pericentre from (q, e, inc, node, peri), for any
    e >= 0 (elliptic, parabolic or hyperbolic orbits)."""
    gm, q, e, inc, node, peri = (np.asarray(v, dtype=np.float64) for v in
                                 np.broadcast_arrays(gm, q, e, inc, node, peri))
    zero = np.zeros_like(q)
    return elements_rotate(q, zero, zero, np.sqrt(gm * (1.0 + e) / q), inc, node, peri)


def elements_rotate(xo, yo, vxo, vyo, inc, node, peri):
    """Orbit-plane position and velocity (pericentre along x) rotated by
    R_z(node) R_x(inc) R_z(peri) into the reference frame."""
    cO, sO = np.cos(node), np.sin(node)
    cw, sw = np.cos(peri), np.sin(peri)
    ci, si = np.cos(inc), np.sin(inc)
    r11 = cO * cw - sO * sw * ci
    r12 = -cO * sw - sO * cw * ci
    r21 = sO * cw + cO * sw * ci
    r22 = -sO * sw + cO * cw * ci
    r31 = sw * si
    r32 = cw * si
    out = np.empty((6,) + np.shape(xo))
    out[0] = r11 * xo + r12 * yo
    out[1] = r21 * xo + r22 * yo
    out[2] = r31 * xo + r32 * yo
    out[3] = r11 * vxo + r12 * vyo
    out[4] = r21 * vxo + r22 * vyo
    out[5] = r31 * vxo + r32 * vyo
    return out


def _angles(rng, k):
    return (rng.uniform(0, 2 * math.pi, k), rng.uniform(0, 2 * math.pi, k),
            rng.uniform(0, 2 * math.pi, k))


def _smalls(rng, k, amin, amax, sig_e, sig_i, gm):
    a = rng.uniform(amin, amax, k)
    e = np.minimum(rng.rayleigh(sig_e, k), 0.9)
    inc = rng.rayleigh(sig_i, k)
    node, peri, M = _angles(rng, k)
    return elements_to_xv(gm, a, e, inc, node, peri, M)


def _assemble(name, params, m_big, xv_big, xv_small, rp, rho, nsteps, ckpt=0):
    xv = np.concatenate([xv_big, xv_small], axis=1)
    return Workload(name=name, params=params, nbig=len(m_big), nsmall=xv_small.shape[1],
                    m_big=np.asarray(m_big, dtype=np.float64), xv_helio=np.ascontiguousarray(xv),
                    rp_km=np.ascontiguousarray(rp, dtype=np.float64),
                    rhop=np.ascontiguousarray(rho, dtype=np.float64), nsteps=int(nsteps),
                    checkpoint_every=int(ckpt))


def plain_2big_1k(seed=0, nsmall=1000, nsteps=1000):
    rng = np.random.default_rng(seed)
    m = np.array([M_JUP, 0.3 * M_JUP])
    a = np.array([5.2, 9.5])
    node, peri, M = _angles(rng, 2)
    xb = elements_to_xv(G * (1.0 + m), a, 0.03, math.radians(0.5), node, peri, M)
    xs = _smalls(rng, nsmall, 2.0, 12.0, 0.01, 0.005, G)
    rp = np.full(nsmall, 1.0)
    rho = np.full(nsmall, 1.0)
    return _assemble("plain_2big_1k", default_params(8.0), m, xb, xs, rp, rho, nsteps)


def _cores(rng, k, amin=3.0, amax=10.0):
    m = rng.uniform(10.0, 30.0, k) * M_EARTH
    a = rng.uniform(amin, amax, k)
    e = rng.rayleigh(0.01, k)
    inc = rng.rayleigh(0.005, k)
    node, peri, M = _angles(rng, k)
    return m, elements_to_xv(G * (1.0 + m), a, e, inc, node, peri, M)


def _gas_smalls(rng, k):
    xs = _smalls(rng, k, 1.0, 15.0, 0.01, 0.005, G)
    rp = np.exp(rng.uniform(math.log(1.0), math.log(100.0), k))
    rho = rng.uniform(1.0, 3.0, k)
    return xs, rp, rho


def gas_4core_100k(seed=1, nbig=4, nsmall=100_000, nsteps=10_000):
    rng = np.random.default_rng(seed)
    m, xb = _cores(rng, nbig)
    xs, rp, rho = _gas_smalls(rng, nsmall)
    params = default_params(10.0, default_gas(True))
    return _assemble("gas_4core_100k", params, m, xb, xs, rp, rho, nsteps)


def semiactive_2000big_200k(seed=2, nbig=2000, nsmall=200_000, nsteps=2000):
    rng = np.random.default_rng(seed)
    m = np.exp(rng.uniform(math.log(M_MOON), math.log(M_MARS), nbig))
    a = rng.uniform(0.5, 4.0, nbig)
    e = rng.rayleigh(0.02, nbig)
    inc = rng.rayleigh(0.01, nbig)
    node, peri, M = _angles(rng, nbig)
    xb = elements_to_xv(G * (1.0 + m), a, e, inc, node, peri, M)
    xs = _smalls(rng, nsmall, 0.5, 4.0, 0.02, 0.01, G)
    rp = np.full(nsmall, 1.0)
    rho = np.full(nsmall, 1.0)
    return _assemble("semiactive_2000big_200k", default_params(6.0), m, xb, xs, rp, rho, nsteps)


def scatter_2giant(seed=5, nsmall=4000, nsteps=500, eject_every=10):
    """Two giants (Jupiter and Saturn masses at 5.2 and 9.5 AU) scattering a
    planetesimal swarm on giant-crossing orbits, with the ejection test of
    Sec. 3.5 every `eject_every` steps: half the planetesimals elliptic with
    a ~ U[4, 12] AU and e ~ U[0.3, 0.95], a quarter near-parabolic (e ~
    U[0.97, 1.03]) and a quarter hyperbolic (e ~ U[1.05, 1.5]), the last two
    started at pericentre q ~ U[3, 8] AU.  No gas; dt = 8 d."""
    rng = np.random.default_rng(seed)
    m = np.array([M_JUP, 0.3 * M_JUP])
    node, peri, M = _angles(rng, 2)
    xb = elements_to_xv(G * (1.0 + m), np.array([5.2, 9.5]), 0.05, math.radians(1.0), node, peri,
                        M)
    k1 = nsmall // 2
    k2 = nsmall // 4
    k3 = nsmall - k1 - k2
    a = rng.uniform(4.0, 12.0, k1)
    e = rng.uniform(0.3, 0.95, k1)
    inc = rng.rayleigh(0.02, k1)
    node, peri, M = _angles(rng, k1)
    x1 = elements_to_xv(G, a, e, inc, node, peri, M)
    parts = [x1]
    for k, lo, hi in ((k2, 0.97, 1.03), (k3, 1.05, 1.5)):
        node, peri, _ = _angles(rng, k)
        parts.append(pericentre_to_xv(G, rng.uniform(3.0, 8.0, k), rng.uniform(lo, hi, k),
                                      rng.rayleigh(0.02, k), node, peri))
    xs = np.concatenate(parts, axis=1)
    params = default_params(8.0)
    params["eject_every"] = int(eject_every)
    rp = np.full(nsmall, 1.0)
    rho = np.full(nsmall, 1.0)
    return _assemble("scatter_2giant", params, m, xb, xs, rp, rho, nsteps)


YEAR = 365.25                        # days


def growth_2giant(seed=6, nsmall=24_000, nsteps=1000, tau_c_days=5.0e3 * YEAR,
                  tau_g_days=1.0e3 * YEAR):
    """Two forming giants in a gas disk (the paper's first use case, Sec. 4.1):
    lunar-mass embryos (0.01 M_earth) at 10 and 20 AU grow to 15 M_earth cores
    in tau_c (Eq. 13), then accrete gas towards 300 and 100 M_earth with
    e-folding time tau_g (Eq. 15) and open gaps (Eqs. 8-9); planetesimals from
    1 to 25 AU, 1,000 per AU, r_p log-uniform 1-100 km, rho ~ U[1, 3] g/cm^3.
    dt = 10 d."""
    rng = np.random.default_rng(seed)
    m0 = np.full(2, 0.01 * M_EARTH)
    node, peri, M = _angles(rng, 2)
    xb = elements_to_xv(G * (1.0 + m0), np.array([10.0, 20.0]), 0.01, math.radians(0.5), node,
                        peri, M)
    xs = _smalls(rng, nsmall, 1.0, 25.0, 0.01, 0.005, G)
    rp = np.exp(rng.uniform(math.log(1.0), math.log(100.0), nsmall))
    rho = rng.uniform(1.0, 3.0, nsmall)
    params = default_params(10.0, default_gas(True))
    w = _assemble("growth_2giant", params, m0, xb, xs, rp, rho, nsteps)
    w.growth = dict(m0=m0.copy(), mc=np.full(2, 15.0 * M_EARTH),
                    mf=np.array([300.0, 100.0]) * M_EARTH, tau_c=np.full(2, float(tau_c_days)),
                    tau_g=np.full(2, float(tau_g_days)), delta_r=np.full(2, 0.01),
                    grows=np.ones(2, dtype=np.int32))
    return w


def adjoint_4core_50k(seed=4, nbig=4, nsmall=50_000, nsteps=2000, checkpoint_every=50):
    rng = np.random.default_rng(seed)
    m, xb = _cores(rng, nbig)
    xs, rp, rho = _gas_smalls(rng, nsmall)
    params = default_params(10.0, default_gas(True))
    return _assemble("adjoint_4core_50k", params, m, xb, xs, rp, rho, nsteps, checkpoint_every)


def ensemble_256(seed=3, nsys=256, nsmall_min=1000, nsmall_max=200_000, nsteps=1000):
    """List of independent systems (one Workload each)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(nsys):
        nb = int(rng.integers(2, 51))
        ns = int(round(math.exp(rng.uniform(math.log(nsmall_min), math.log(nsmall_max)))))
        m = np.exp(rng.uniform(math.log(M_MOON), math.log(M_MARS), nb))
        a = rng.uniform(1.0, 15.0, nb)
        node, peri, M = _angles(rng, nb)
        xb = elements_to_xv(G * (1.0 + m), a, rng.rayleigh(0.01, nb), rng.rayleigh(0.005, nb),
                            node, peri, M)
        xs, rp, rho = _gas_smalls(rng, ns)
        gas = default_gas(True, sigma1=1700.0 * rng.uniform(0.3, 3.0))
        params = default_params(10.0, gas)
        out.append(_assemble(f"ensemble_256[{s}]", params, m, xb, xs, rp, rho, nsteps))
    return out


WORKLOADS = {
    "plain_2big_1k": plain_2big_1k,
    "gas_4core_100k": gas_4core_100k,
    "semiactive_2000big_200k": semiactive_2000big_200k,
    "adjoint_4core_50k": adjoint_4core_50k,
    "scatter_2giant": scatter_2giant,
    "growth_2giant": growth_2giant,
}


def make(name, **kw):
    return WORKLOADS[name](**kw)
