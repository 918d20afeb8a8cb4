"""ctypes loader for the CPU FP64 oracle (``mx_oracle.cpp``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import
this package.  It shares no code with the CUDA path; the two meet only through
the seeded inputs of ``paper_2601_16791_gb300.workloads``, which hold none of
the method's arithmetic.

Arrays are numpy float64 in structure-of-arrays layout (``6 x N`` for states:
x, y, z, vx, vy, vz rows), big bodies first.
"""
import ctypes
import math

import numpy as np

from .build import build

_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.c_void_p


class OrcGas(ctypes.Structure):
    _fields_ = [("sigma1_gcm2", _D), ("gamma", _D), ("r_c_au", _D), ("r_in_au", _D),
                ("hr_1au", _D), ("flare", _D), ("gamma_c", _D), ("mu_mol", _D),
                ("sigma_mol_cm2", _D), ("cd_scale", _D), ("enabled", _I), ("cd_mode", _I),
                ("disk_gravity", _I), ("reserved", _I)]


class OrcParams(ctypes.Structure):
    _fields_ = [("G", _D), ("m_star", _D), ("dt", _D), ("rcrit_hill", _D), ("bs_tol", _D),
                ("kepler_max_iter", _I), ("bs_max_sub", _I), ("pair_cap", _I),
                ("eject_every", _I), ("gas", OrcGas)]


class OrcGrowth(ctypes.Structure):
    _fields_ = [("m0", _D), ("mc", _D), ("mf", _D), ("tau_c", _D), ("tau_g", _D),
                ("delta_r", _D), ("grows", _I), ("reserved", _I)]


def make_growth(g, nbig):
    """OrcGrowth[nbig] from a dict of per-big arrays (m0, mc, mf, tau_c, tau_g,
    delta_r, grows), or None."""
    if g is None:
        return None
    arr = (OrcGrowth * nbig)()
    for i in range(nbig):
        arr[i] = OrcGrowth(float(g["m0"][i]), float(g["mc"][i]), float(g["mf"][i]),
                           float(g["tau_c"][i]), float(g["tau_g"][i]), float(g["delta_r"][i]),
                           int(g["grows"][i]), 0)
    return arr


ERRORS = {0: "ok", 1: "bad argument", 2: "Kepler solve did not converge",
          3: "Bulirsch-Stoer did not converge", 4: "pair list overflow", 5: "non-finite state"}


class OracleError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"oracle {where}: {ERRORS.get(code, code)}")
        self.code = code


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        sig = {
            "orc_set_threads": (None, [_I]),
            "orc_changeover": (_D, [_D, _D]),
            "orc_k_over_s3": (_D, [_D, _D]),
            "orc_init": (_I, [_P, _I, _I, _P, _P, _P, _P, _P]),
            "orc_readout": (_I, [_P, _I, _I, _P, _P, _P]),
            "orc_accel_grav": (_I, [_I, _I, _P, _P, _P, _P, _I]),
            "orc_momentum": (_I, [_I, _I, _P, _P, _P]),
            "orc_gas_drag": (_I, [_P, _I, _I, _P, _P, _P, _P, _P]),
            "orc_gas_state": (_I, [_P, _D, _P]),
            "orc_drag_cd": (_D, [_D, _D, _I]),
            "orc_dg_series": (_D, [_D]),
            "orc_dg_series_dgamma": (_D, [_D]),
            "orc_disk_gravity": (_I, [_P, _P, _P]),
            "orc_drag_one": (_I, [_P, _P, _P, _D, _D, _P, _P]),
            "orc_stumpff": (None, [_D, _P]),
            "orc_drift": (_I, [_P, _I, _P, _D, _P]),
            "orc_hermite_d2min": (_D, [_D, _D, _D, _D, _D]),
            "orc_detect": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _I, _P]),
            "orc_bs_group": (_I, [_P, _I, _P, _P, _P, _D, _P]),
            "orc_build_groups": (_I, [_I, _I, _I, _P, _I, _I, _P, _P, _P, _P]),
            "orc_step": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _I, _P, _P, _I, _P, _P]),
            "orc_step_ex": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _I, ctypes.c_longlong, _P, _P,
                                 _D, _P, _P]),
            "orc_gas_drag_gap": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P, _P]),
            "orc_grow_state": (_I, [_P, _I, _I, _P, _P, _P, _P, _D, _D, _P, _P, _P, _P, _P]),
            "orc_eject": (_I, [_P, _I, _I, _P, _P, _P, _P]),
            "orc_elements": (_I, [_I, _P, _P, _P]),
            "orc_energy": (_I, [_P, _I, _I, _P, _P, _P, _P]),
            "orc_semimajor": (_I, [_P, _I, _I, _P, _P, _P]),
            "orc_jvp_loss": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _I, _P, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(code, where):
    if code != 0:
        raise OracleError(code, where)


def make_params(cfg):
    """OrcParams from a plain parameter dict (see workloads.Workload.params)."""
    g = cfg["gas"]
    gas = OrcGas(g["sigma1_gcm2"], g["gamma"], g["r_c_au"], g["r_in_au"], g["hr_1au"], g["flare"],
                 g["gamma_c"], g["mu_mol"], g["sigma_mol_cm2"], g["cd_scale"], int(g["enabled"]),
                 int(g["cd_mode"]), int(g.get("disk_gravity", False)), 0)
    return OrcParams(cfg["G"], cfg["m_star"], cfg["dt"], cfg["rcrit_hill"], cfg["bs_tol"],
                     int(cfg["kepler_max_iter"]), int(cfg["bs_max_sub"]), int(cfg["pair_cap"]),
                     int(cfg.get("eject_every", 0)), gas)


def set_threads(n):
    lib().orc_set_threads(int(n))


def changeover(s, rc):
    return lib().orc_changeover(float(s), float(rc))


def k_over_s3(s2, rc):
    return lib().orc_k_over_s3(float(s2), float(rc))


def init(p, nbig, nsmall, m_big, xv_helio):
    n = nbig + nsmall
    xv_helio = _f64(xv_helio)
    m_big = _f64(m_big)
    xv = np.empty((6, n))
    mu = np.empty(n)
    rc = np.empty(n)
    _check(lib().orc_init(ctypes.byref(p), nbig, nsmall, _ptr(m_big), _ptr(xv_helio), _ptr(xv),
                          _ptr(mu), _ptr(rc)), "init")
    return xv, mu, rc


def readout(p, nbig, nsmall, mu, xv_dh):
    n = nbig + nsmall
    out = np.empty((6, n))
    xv_dh = _f64(xv_dh)
    mu = _f64(mu)
    _check(lib().orc_readout(ctypes.byref(p), nbig, nsmall, _ptr(mu), _ptr(xv_dh), _ptr(out)),
           "readout")
    return out


def accel_grav(nbig, xv, mu, rcrit, triangular=False):
    xv, mu, rcrit = _f64(xv), _f64(mu), _f64(rcrit)
    n = xv.shape[1]
    acc = np.empty((3, n))
    _check(lib().orc_accel_grav(nbig, n, _ptr(xv), _ptr(mu), _ptr(rcrit), _ptr(acc),
                                int(triangular)), "accel_grav")
    return acc


def momentum(nbig, xv, mu):
    xv, mu = _f64(xv), _f64(mu)
    P = np.empty(3)
    _check(lib().orc_momentum(nbig, xv.shape[1], _ptr(xv), _ptr(mu), _ptr(P)), "momentum")
    return P


def gas_drag(p, nbig, xv, mu, rp_km, rhop):
    xv, mu, rp_km, rhop = _f64(xv), _f64(mu), _f64(rp_km), _f64(rhop)
    nsmall = xv.shape[1] - nbig
    acc = np.empty((3, nsmall))
    _check(lib().orc_gas_drag(ctypes.byref(p), nbig, nsmall, _ptr(xv), _ptr(mu), _ptr(rp_km),
                              _ptr(rhop), _ptr(acc)), "gas_drag")
    return acc


GAS_STATE_KEYS = ("sigma", "rho_g", "H_au", "cs", "vk", "eta", "vg", "hr")


def gas_drag_gap(p, nbig, xv, mu, rp_km, rhop, gap_w, gap_f):
    """Drag on the small bodies (3 x nsmall) with gaps around the massive ones."""
    xv, mu, rp_km, rhop = _f64(xv), _f64(mu), _f64(rp_km), _f64(rhop)
    gap_w, gap_f = _f64(gap_w), _f64(gap_f)
    nsmall = xv.shape[1] - nbig
    acc = np.empty((3, nsmall))
    _check(lib().orc_gas_drag_gap(ctypes.byref(p), nbig, nsmall, _ptr(xv), _ptr(mu), _ptr(rp_km),
                                  _ptr(rhop), _ptr(gap_w), _ptr(gap_f), _ptr(acc)), "gas_drag_gap")
    return acc


def gas_state(p, R):
    out = np.empty(8)
    _check(lib().orc_gas_state(ctypes.byref(p), float(R), _ptr(out)), "gas_state")
    return dict(zip(GAS_STATE_KEYS, out))


def drag_cd(Re, Ma, mode=0):
    return lib().orc_drag_cd(float(Re), float(Ma), int(mode))


def dg_series(gamma):
    """S(gamma) of Eq. 10: F_DG = 2 pi G Sigma(r) S(gamma) for gamma != 1."""
    return lib().orc_dg_series(float(gamma))


def dg_series_dgamma(gamma):
    """dS/dgamma of the disk-gravity series S(gamma) of Eq. 10, summed term by term."""
    return lib().orc_dg_series_dgamma(float(gamma))


def disk_gravity(p, x3):
    x3 = _f64(x3)
    acc = np.empty(3)
    _check(lib().orc_disk_gravity(ctypes.byref(p), _ptr(x3), _ptr(acc)), "disk_gravity")
    return acc


def drag_one(p, x3, vh3, rp_km, rhop):
    x3, vh3 = _f64(x3), _f64(vh3)
    acc = np.empty(3)
    rm = np.empty(2)
    _check(lib().orc_drag_one(ctypes.byref(p), _ptr(x3), _ptr(vh3), float(rp_km), float(rhop),
                              _ptr(acc), _ptr(rm)), "drag_one")
    return acc, rm[0], rm[1]


def stumpff(z):
    c = np.empty(4)
    lib().orc_stumpff(float(z), _ptr(c))
    return c


def drift(p, xv, h):
    xv = _f64(xv).copy()
    it = ctypes.c_int(0)
    _check(lib().orc_drift(ctypes.byref(p), xv.shape[1], _ptr(xv), float(h), ctypes.byref(it)),
           "drift")
    return xv, it.value


def hermite_d2min(d0, d1, d0t, d1t, h):
    return lib().orc_hermite_d2min(float(d0), float(d1), float(d0t), float(d1t), float(h))


def detect(p, nbig, xv0, xv1, rcrit, cap=1 << 20):
    xv0, xv1, rcrit = _f64(xv0), _f64(xv1), _f64(rcrit)
    n = xv0.shape[1]
    flags = np.empty(n, dtype=np.uint8)
    pairs = np.empty((cap, 2), dtype=np.int32)
    npairs = ctypes.c_int(0)
    _check(lib().orc_detect(ctypes.byref(p), nbig, n, _ptr(xv0), _ptr(xv1), _ptr(rcrit),
                            _ptr(flags), _ptr(pairs), cap, ctypes.byref(npairs)), "detect")
    return flags, pairs[:npairs.value].copy()


def bs_group(p, mu, rcrit, xv, h):
    mu, rcrit = _f64(mu), _f64(rcrit)
    xv = _f64(xv).copy()
    nsub = ctypes.c_int(0)
    _check(lib().orc_bs_group(ctypes.byref(p), xv.shape[1], _ptr(mu), _ptr(rcrit), _ptr(xv),
                              float(h), ctypes.byref(nsub)), "bs_group")
    return xv, nsub.value


def build_groups(nbig, nsmall, pairs):
    """Encounter groups of one step from its flagged (i, j) pairs.  Returns a
    list of (members, write_from): members bigs ascending then the
    planetesimal, write_from the index of the first member written back."""
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    ng = ctypes.c_int(0)
    cap_g = max(1, nbig + nsmall)
    cap_m = max(1, len(pr) * (nbig + 1) + nbig)
    mem = np.empty(cap_m, dtype=np.int32)
    off = np.empty(cap_g + 1, dtype=np.int32)
    wf = np.empty(cap_g, dtype=np.int32)
    _check(lib().orc_build_groups(int(nbig), int(nsmall), len(pr), _ptr(pr), cap_g, cap_m,
                                  _ptr(mem), _ptr(off), _ptr(wf), ctypes.byref(ng)),
           "build_groups")
    return [(mem[off[g]:off[g + 1]].tolist(), int(wf[g])) for g in range(ng.value)]


def step(p, nbig, xv, mu, rcrit, rp_km, rhop, nsteps, log_cap=0):
    """Run nsteps hybrid steps.  Returns (xv, ever_flag, pair_log, stats)."""
    xv = _f64(xv).copy()
    n = xv.shape[1]
    nsmall = n - nbig
    mu, rcrit = _f64(mu), _f64(rcrit)
    rp = None if rp_km is None else _f64(rp_km)
    rh = None if rhop is None else _f64(rhop)
    ever = np.zeros(n, dtype=np.uint8)
    log = np.zeros((max(log_cap, 1), 3), dtype=np.int32)
    lc = ctypes.c_int(0)
    stats = np.zeros(4, dtype=np.int64)
    _check(lib().orc_step(ctypes.byref(p), nbig, nsmall, _ptr(xv), _ptr(mu), _ptr(rcrit),
                          _ptr(rp), _ptr(rh), int(nsteps), _ptr(ever),
                          _ptr(log) if log_cap > 0 else None, int(log_cap), ctypes.byref(lc),
                          _ptr(stats)), "step")
    return xv, ever, log[:min(lc.value, log_cap)].copy(), stats


def step_ex(p, nbig, xv, mu, rcrit, rp_km, rhop, nsteps, stat=None, step0=0, growth=None,
            gap_c=4.0):
    """nsteps hybrid steps with the ejection test of Sec. 3.5 on the schedule
    p.eject_every and, with growth (a dict of per-big arrays, see make_growth),
    the growth tracks and gaps of Secs. 3.1 and 3.3, from global step index
    step0.  Returns (xv, mu, stat, ever, rcrit): stat is int8, 0 for bodies in
    the integration and -3 for removed ones; removed massive bodies have mu 0."""
    xv = _f64(xv).copy()
    n = xv.shape[1]
    mu = _f64(mu).copy()
    rcrit = _f64(rcrit).copy()
    gr = make_growth(growth, nbig)
    stat = np.zeros(n, dtype=np.int8) if stat is None else np.ascontiguousarray(stat, np.int8).copy()
    rp = None if rp_km is None else _f64(rp_km)
    rh = None if rhop is None else _f64(rhop)
    ever = np.zeros(n, dtype=np.uint8)
    _check(lib().orc_step_ex(ctypes.byref(p), nbig, n - nbig, _ptr(xv), _ptr(mu), _ptr(rcrit),
                             _ptr(rp), _ptr(rh), int(nsteps), int(step0), _ptr(stat), gr,
                             float(gap_c), _ptr(ever), None), "step_ex")
    return xv, mu, stat, ever, rcrit


def grow_state(p, nbig, xv, mu, rcrit, growth, t, gap_c=4.0):
    """Growth quantities at time t (orc_grow_state): dict of per-big arrays
    mu, rcrit, gap_w, gap_f, radius."""
    xv, mu, rcrit = _f64(xv), _f64(mu), _f64(rcrit)
    out = {k: np.zeros(nbig) for k in ("mu", "rcrit", "gap_w", "gap_f", "radius")}
    _check(lib().orc_grow_state(ctypes.byref(p), nbig, xv.shape[1], _ptr(xv), _ptr(mu),
                                _ptr(rcrit), make_growth(growth, nbig), float(gap_c), float(t),
                                _ptr(out["mu"]), _ptr(out["rcrit"]), _ptr(out["gap_w"]),
                                _ptr(out["gap_f"]), _ptr(out["radius"])), "grow_state")
    return out


def eject(p, nbig, xv, mu, stat=None):
    """The ejection test on a DH state.  Returns (mu, stat, removed)."""
    xv = _f64(xv)
    n = xv.shape[1]
    mu = _f64(mu).copy()
    stat = np.zeros(n, dtype=np.int8) if stat is None else np.ascontiguousarray(stat, np.int8).copy()
    k = ctypes.c_int(0)
    _check(lib().orc_eject(ctypes.byref(p), nbig, n, _ptr(xv), _ptr(mu), _ptr(stat),
                           ctypes.byref(k)), "eject")
    return mu, stat, k.value


def elements(gm, xv_helio):
    """Osculating elements (6 x n rows q, e, i, varpi, Omega, M) of heliocentric
    states about gm (scalar or per body)."""
    xv_helio = _f64(xv_helio)
    n = xv_helio.shape[1]
    gm = _f64(np.broadcast_to(np.asarray(gm, dtype=np.float64), (n,)))
    out = np.empty((6, n))
    _check(lib().orc_elements(n, _ptr(gm), _ptr(xv_helio), _ptr(out)), "elements")
    return out


def energy(p, nbig, xv, mu):
    xv, mu = _f64(xv), _f64(mu)
    E = ctypes.c_double(0.0)
    L = np.empty(3)
    _check(lib().orc_energy(ctypes.byref(p), nbig, xv.shape[1], _ptr(xv), _ptr(mu),
                            ctypes.byref(E), _ptr(L)), "energy")
    return E.value, L


def semimajor(p, nbig, mu, xv_helio):
    xv_helio, mu = _f64(xv_helio), _f64(mu)
    a = np.empty(xv_helio.shape[1])
    _check(lib().orc_semimajor(ctypes.byref(p), nbig, xv_helio.shape[1], _ptr(mu),
                               _ptr(xv_helio), _ptr(a)), "semimajor")
    return a


def jvp_loss(p, nbig, m_big, xv_helio, rp_km, rhop, w, nsteps, dxv, dpar):
    xv_helio = _f64(xv_helio)
    n = xv_helio.shape[1]
    nsmall = n - nbig
    m_big, rp_km, rhop, w = _f64(m_big), _f64(rp_km), _f64(rhop), _f64(w)
    dxv, dpar = _f64(dxv), _f64(dpar)
    L = ctypes.c_double(0.0)
    dL = ctypes.c_double(0.0)
    _check(lib().orc_jvp_loss(ctypes.byref(p), nbig, nsmall, _ptr(m_big), _ptr(xv_helio),
                              _ptr(rp_km), _ptr(rhop), _ptr(w), int(nsteps), _ptr(dxv),
                              _ptr(dpar), ctypes.byref(L), ctypes.byref(dL)), "jvp_loss")
    return L.value, dL.value


INF = math.inf
