"""Thin ctypes binding of include/mx.h (argument marshalling only).

Every function here has the C name and calls straight into libmx.so; all
arithmetic on bodies runs in the library's CUDA kernels.  Device buffers are
passed as torch CUDA tensors (float64, contiguous) or raw integer pointers;
host buffers as numpy arrays.  If libmx.so cannot be built or loaded, the
import of the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.c_void_p

MX_OK = 0
STATUS = {0: "MX_OK", 1: "MX_ERR_ARG", 2: "MX_ERR_CUDA", 3: "MX_ERR_OOM", 4: "MX_ERR_KEPLER_NOCONV",
          5: "MX_ERR_BS_NOCONV", 6: "MX_ERR_PAIR_OVERFLOW", 7: "MX_ERR_NONFINITE",
          8: "MX_ERR_BARRIER_TIMEOUT", 9: "MX_ERR_ENCOUNTER_IN_ADJOINT",
          10: "MX_ERR_GROUP_TOO_LARGE"}
MX_COORD_HELIO = 0
MX_COORD_DH = 1
MX_MAX_GROUP = 16


class MxGas(ctypes.Structure):
    _fields_ = [("sigma1_gcm2", _D), ("gamma", _D), ("r_c_au", _D), ("r_in_au", _D),
                ("hr_1au", _D), ("flare", _D), ("gamma_c", _D), ("mu_mol", _D),
                ("sigma_mol_cm2", _D), ("cd_scale", _D), ("enabled", _I), ("cd_mode", _I),
                ("disk_gravity", _I), ("reserved", _I)]


class MxParams(ctypes.Structure):
    _fields_ = [("G", _D), ("m_star", _D), ("dt", _D), ("rcrit_hill", _D), ("bs_tol", _D),
                ("kepler_max_iter", _I), ("bs_max_sub", _I), ("pair_cap", _I),
                ("eject_every", _I), ("gas", MxGas)]


class MxGrowth(ctypes.Structure):
    _fields_ = [("m0", _D), ("mc", _D), ("mf", _D), ("tau_c", _D), ("tau_g", _D),
                ("delta_r", _D), ("grows", _I), ("reserved", _I)]


class MxError(RuntimeError):
    def __init__(self, code, where, msg=""):
        super().__init__(f"{where}: {STATUS.get(code, code)} {msg}".strip())
        self.code = code
        self.status = STATUS.get(code, str(code))


_lib = None

_SIGS = {
    "mx_init_system": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P]),
    "mx_destroy": (None, [_P]),
    "mx_step": (_I, [_P, _I]),
    "mx_step_profiled": (_I, [_P, _I, _P, _P, _P]),
    "mx_step_timed": (_I, [_P, _I, _P, ctypes.c_size_t, _P, _P, _P]),
    "mx_step_wall": (_I, [_P, _I, _P, ctypes.c_size_t, _P, _P]),
    "mx_catchup_work": (_I, [_P, _P, _I]),
    "mx_set_persistent": (_I, [_P, _I, ctypes.c_longlong]),
    "mx_last_encounters": (_I, [_P, _P, _I, _P]),
    "mx_accel": (_I, [_P, _P]),
    "mx_gas_drag": (_I, [_P, _P]),
    "mx_detect_encounters": (_I, [_P, _P, _P, _P, _P, _I, _P]),
    "mx_kepler_drift": (_I, [_P, _P, _D]),
    "mx_energy": (_I, [_P, _P, _P]),
    "mx_get_state": (_I, [_P, _P, _I, _P]),
    "mx_set_state": (_I, [_P, _P, _I, ctypes.c_longlong]),
    "mx_get_state_device": (_I, [_P, _P]),
    "mx_set_state_device": (_I, [_P, _P]),
    "mx_sizes": (_I, [_P, _P, _P]),
    "mx_last_error": (ctypes.c_char_p, []),
    "mx_fp64_peak": (_I, [_P, _D, _P]),
    "mx_detect_encounters_noalloc": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _I, _P, _P]),
    "mx_init_batch": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "mx_batch_offsets": (_I, [_P, _P]),
    "mx_batch_size": (_I, [_P, _P, _P]),
    "mx_energy_batch": (_I, [_P, _P, _P]),
    "mx_tiling": (_I, [_P, _P, _P]),
    "mx_set_tiling": (_I, [_P, _I, _I]),
    "mx_set_defer_window": (_I, [_P, _I]),
    "mx_defer_stats": (_I, [_P, _P, _P, _P, _P]),
    "mx_set_gas_params": (_I, [_P, _I, _D, _D, _D]),
    "mx_kick_branches": (_I, [_P, _I, ctypes.c_longlong]),
    "mx_encounter_log": (_I, [_P, _P, _P, _I]),
    "mx_set_step_index": (_I, [_P, ctypes.c_longlong]),
    "mx_loss_semimajor": (_I, [_P, _P, _P, _P, _P, _P]),
    "mx_adjoint_step": (_I, [_P, _P, ctypes.c_longlong, _P, _P]),
    "mx_adjoint_init": (_I, [_P, _P, _P]),
    "mx_check_ejections": (_I, [_P, _P]),
    "mx_body_status": (_I, [_P, _P, _P]),
    "mx_elements": (_I, [_P, _P]),
    "mx_set_growth": (_I, [_P, _I, _P, _D]),
    "mx_adjoint_encounters": (_I, [_P, _I]),
    "mx_adjoint_store": (_I, [_P, ctypes.c_longlong]),
    "mx_adjoint_merge": (_I, [_P, _I]),
    "mx_predrift_state": (_I, [_P, _P]),
    "mx_adjoint_step_predrift": (_I, [_P, _P, _P, ctypes.c_longlong, _P, _P]),
    "mx_adjoint_flush": (_I, [_P]),
    "mx_planets": (_I, [_P, _P, _P]),
}


def lib_path():
    return _build.LIB


def load():
    """Build (if stale) and load libmx.so; raises if either fails."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(code, where):
    if code != MX_OK:
        raise MxError(code, where, load().mx_last_error().decode())


def _host(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _hptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dptr(t):
    """Device pointer of a torch CUDA tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def make_params(cfg) -> MxParams:
    g = cfg["gas"]
    gas = MxGas(g["sigma1_gcm2"], g["gamma"], g["r_c_au"], g["r_in_au"], g["hr_1au"], g["flare"],
                g["gamma_c"], g["mu_mol"], g["sigma_mol_cm2"], g["cd_scale"], int(g["enabled"]),
                int(g["cd_mode"]), int(g.get("disk_gravity", False)), 0)
    return MxParams(cfg["G"], cfg["m_star"], cfg["dt"], cfg["rcrit_hill"], cfg["bs_tol"],
                    int(cfg["kepler_max_iter"]), int(cfg["bs_max_sub"]), int(cfg["pair_cap"]),
                    int(cfg.get("eject_every", 0)), gas)


# ------------------------------------------------------------ C-named calls
def mx_init_system(params, n_big, n_small, m_big, xv_helio, rp_km=None, rho_gcm3=None,
                   stream=None):
    L = load()
    out = ctypes.c_void_p()
    m_big = _host(m_big)
    xv = _host(xv_helio)
    rp = None if rp_km is None else _host(rp_km)
    rho = None if rho_gcm3 is None else _host(rho_gcm3)
    st = ctypes.c_void_p(stream) if stream else None
    _check(L.mx_init_system(ctypes.byref(params), int(n_big), int(n_small), _hptr(m_big), _hptr(xv),
                            _hptr(rp), _hptr(rho), st, ctypes.byref(out)), "mx_init_system")
    return out


def mx_destroy(sys):
    load().mx_destroy(sys)


def mx_step(sys, n_steps):
    _check(load().mx_step(sys, int(n_steps)), "mx_step")


KERNELS = ("k_prep", "k_jump_kick", "k_jump_drift", "k_detect", "k_sort_keys", "k_groups", "k_bs",
           "k_catchup", "k_catchup_side", "k_eject")


def mx_step_profiled(sys, n_steps):
    """Returns (per-kernel ms dict, per-kernel launch counts dict, total ms)."""
    ms = np.zeros(len(KERNELS))
    cnt = np.zeros(len(KERNELS), dtype=np.int32)
    tot = ctypes.c_double(0.0)
    _check(load().mx_step_profiled(sys, int(n_steps), _hptr(ms), _hptr(cnt), ctypes.byref(tot)),
           "mx_step_profiled")
    return dict(zip(KERNELS, ms.tolist())), dict(zip(KERNELS, cnt.tolist())), tot.value


def mx_step_timed(sys, n_steps, dev_flush=None, per_kernel=True):
    """mx_step_profiled with dev_flush (a CUDA tensor, e.g. larger than L2)
    overwritten before every step, outside the timed spans.  per_kernel=False
    runs the production graphs with events only around each step (the
    per-kernel dicts come back empty)."""
    ms = np.zeros(len(KERNELS))
    cnt = np.zeros(len(KERNELS), dtype=np.int32)
    tot = ctypes.c_double(0.0)
    nbytes = 0 if dev_flush is None else dev_flush.numel() * dev_flush.element_size()
    _check(load().mx_step_timed(sys, int(n_steps), _dptr(dev_flush), nbytes,
                                _hptr(ms) if per_kernel else None,
                                _hptr(cnt) if per_kernel else None,
                                ctypes.byref(tot)), "mx_step_timed")
    if not per_kernel:
        return {}, {}, tot.value
    return dict(zip(KERNELS, ms.tolist())), dict(zip(KERNELS, cnt.tolist())), tot.value


def mx_step_wall(sys, n_steps, dev_flush=None):
    """n_steps production steps plus the settling catch-up, enqueued without
    host waits, dev_flush overwritten before every step.  Returns (wall_ms,
    flush_ms): the span from the first flush to the end of the catch-up, and
    the same flushes timed alone afterwards."""
    wall, fl = ctypes.c_double(0.0), ctypes.c_double(0.0)
    nbytes = 0 if dev_flush is None else dev_flush.numel() * dev_flush.element_size()
    _check(load().mx_step_wall(sys, int(n_steps), _dptr(dev_flush), nbytes, ctypes.byref(wall),
                               ctypes.byref(fl)), "mx_step_wall")
    return wall.value, fl.value


def mx_set_persistent(sys, on=True, spin_limit=-1):
    """Interior steps as one cooperative launch per step (grid barriers
    between the phases); spin_limit < 0 keeps the default barrier patience."""
    _check(load().mx_set_persistent(sys, 1 if on else 0, int(spin_limit)), "mx_set_persistent")


def mx_catchup_work(sys, reset=False):
    """Catch-up work counters: ((body-slots, half kicks, two-body BS force
    evaluations) of the main-stream catch-ups, the same of the side stream's)."""
    ops = np.zeros(6, dtype=np.int64)
    _check(load().mx_catchup_work(sys, _hptr(ops), 1 if reset else 0), "mx_catchup_work")
    return tuple(int(v) for v in ops[:3]), tuple(int(v) for v in ops[3:])


def mx_last_encounters(sys, cap=1 << 16):
    pairs = np.empty((max(cap, 1), 2), dtype=np.int32)
    n = ctypes.c_int(0)
    _check(load().mx_last_encounters(sys, _hptr(pairs), int(cap), ctypes.byref(n)),
           "mx_last_encounters")
    return pairs[:min(n.value, cap)].copy()


def mx_accel(sys, dev_acc):
    _check(load().mx_accel(sys, _dptr(dev_acc)), "mx_accel")


def mx_gas_drag(sys, dev_acc):
    _check(load().mx_gas_drag(sys, _dptr(dev_acc)), "mx_gas_drag")


def mx_detect_encounters(sys, dev_xv0, dev_xv1, dev_flags=None, dev_pairs=None, cap=0):
    n = ctypes.c_int(0)
    _check(load().mx_detect_encounters(sys, _dptr(dev_xv0), _dptr(dev_xv1), _dptr(dev_flags),
                                       _dptr(dev_pairs), int(cap), ctypes.byref(n)),
           "mx_detect_encounters")
    return n.value


def mx_kepler_drift(sys, dev_xv, h):
    _check(load().mx_kepler_drift(sys, _dptr(dev_xv), float(h)), "mx_kepler_drift")


def mx_energy(sys):
    E = ctypes.c_double(0.0)
    L3 = np.empty(3)
    _check(load().mx_energy(sys, ctypes.byref(E), _hptr(L3)), "mx_energy")
    return E.value, L3


def mx_get_state(sys, n, coords=MX_COORD_HELIO):
    out = np.empty((6, n))
    step = ctypes.c_longlong(0)
    _check(load().mx_get_state(sys, _hptr(out), int(coords), ctypes.byref(step)), "mx_get_state")
    return out, step.value


def mx_set_state(sys, xv, coords=MX_COORD_HELIO, step=0):
    xv = _host(xv)
    _check(load().mx_set_state(sys, _hptr(xv), int(coords), int(step)), "mx_set_state")


def mx_get_state_device(sys, dev_xv):
    _check(load().mx_get_state_device(sys, _dptr(dev_xv)), "mx_get_state_device")


def mx_set_state_device(sys, dev_xv):
    _check(load().mx_set_state_device(sys, _dptr(dev_xv)), "mx_set_state_device")


def mx_sizes(sys):
    nb, ns = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().mx_sizes(sys, ctypes.byref(nb), ctypes.byref(ns)), "mx_sizes")
    return nb.value, ns.value


def mx_fp64_peak(stream=None, ms_target=200.0):
    t = ctypes.c_double(0.0)
    st = ctypes.c_void_p(stream) if stream else None
    _check(load().mx_fp64_peak(st, float(ms_target), ctypes.byref(t)), "mx_fp64_peak")
    return t.value


def mx_init_batch(workloads, stream=None):
    """One mx_system holding every workload of the list (the batched ensemble)."""
    L = load()
    k = len(workloads)
    params = (MxParams * k)(*[make_params(w.params) for w in workloads])
    nb = (ctypes.c_int * k)(*[w.nbig for w in workloads])
    ns = (ctypes.c_int * k)(*[w.nsmall for w in workloads])
    keep = []

    def ptrs(arrs):
        arr = (ctypes.c_void_p * k)()
        for q, a in enumerate(arrs):
            a = _host(a)
            keep.append(a)
            arr[q] = a.ctypes.data
        return arr
    m = ptrs([w.m_big for w in workloads])
    xv = ptrs([w.xv_helio for w in workloads])
    rp = ptrs([w.rp_km for w in workloads])
    rh = ptrs([w.rhop for w in workloads])
    out = ctypes.c_void_p()
    st = ctypes.c_void_p(stream) if stream else None
    _check(L.mx_init_batch(k, params, nb, ns, m, xv, rp, rh, st, ctypes.byref(out)),
           "mx_init_batch")
    return out


def mx_batch_offsets(sys, n_sys):
    off = np.empty(n_sys + 1, dtype=np.int32)
    _check(load().mx_batch_offsets(sys, _hptr(off)), "mx_batch_offsets")
    return off


def mx_energy_batch(sys, n_sys):
    E = np.empty(n_sys)
    L3 = np.empty((n_sys, 3))
    _check(load().mx_energy_batch(sys, _hptr(E), _hptr(L3)), "mx_energy_batch")
    return E, L3


def mx_tiling(sys):
    t, o = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().mx_tiling(sys, ctypes.byref(t), ctypes.byref(o)), "mx_tiling")
    return t.value, o.value


def mx_set_tiling(sys, tile, order):
    _check(load().mx_set_tiling(sys, int(tile), int(order)), "mx_set_tiling")


def mx_set_defer_window(sys, window):
    """Steps per catch-up of deferred planetesimals (0: every body on the direct path)."""
    _check(load().mx_set_defer_window(sys, int(window)), "mx_set_defer_window")


def mx_defer_stats(sys):
    """(window in effect, history length, bodies deferred so far, catch-up launches)."""
    w, mw = ctypes.c_int(0), ctypes.c_int(0)
    n, c = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(load().mx_defer_stats(sys, ctypes.byref(w), ctypes.byref(mw), ctypes.byref(n),
                                 ctypes.byref(c)), "mx_defer_stats")
    return w.value, mw.value, n.value, c.value


MX_STAT_EJECTED = -3


def mx_check_ejections(sys):
    """Runs the ejection test (Sec. 3.5) now; returns the bodies it removed."""
    k = ctypes.c_int(0)
    _check(load().mx_check_ejections(sys, ctypes.byref(k)), "mx_check_ejections")
    return k.value


def mx_body_status(sys, n, n_sys=1):
    """(stat [n] int8: 0 or MX_STAT_EJECTED, removed bodies per system [n_sys])."""
    stat = np.zeros(n, dtype=np.int8)
    cnt = np.zeros(n_sys, dtype=np.int32)
    _check(load().mx_body_status(sys, _hptr(stat), _hptr(cnt)), "mx_body_status")
    return stat, cnt


def mx_elements(sys, dev_el):
    """Osculating heliocentric elements into dev_el (6 x N CUDA float64 tensor):
    q, e, i, longitude of pericentre, node, mean anomaly."""
    _check(load().mx_elements(sys, _dptr(dev_el)), "mx_elements")


def mx_set_growth(sys, k, growth, n_big, gap_c=4.0):
    """Growth tracks of system k from a dict of per-big arrays (m0, mc, mf
    [Msun], tau_c, tau_g [d], delta_r [AU], grows)."""
    arr = (MxGrowth * max(1, n_big))()
    for i in range(n_big):
        arr[i] = MxGrowth(float(growth["m0"][i]), float(growth["mc"][i]), float(growth["mf"][i]),
                          float(growth["tau_c"][i]), float(growth["tau_g"][i]),
                          float(growth["delta_r"][i]), int(growth["grows"][i]), 0)
    _check(load().mx_set_growth(sys, int(k), arr, float(gap_c)), "mx_set_growth")


def mx_planets(sys, nb_total):
    """(masses [Msun], radii [AU]) of all massive bodies."""
    m = np.zeros(nb_total)
    r = np.zeros(nb_total)
    _check(load().mx_planets(sys, _hptr(m), _hptr(r)), "mx_planets")
    return m, r


class Batch:
    """Owns one mx_system with many systems (mx_init_batch)."""

    def __init__(self, workloads, stream=None):
        self.ws = list(workloads)
        self.h = mx_init_batch(self.ws, stream)
        self.offsets = mx_batch_offsets(self.h, len(self.ws))
        self.n = int(self.offsets[-1])

    def step(self, n):
        mx_step(self.h, n)

    def state(self, coords=MX_COORD_HELIO):
        return mx_get_state(self.h, self.n, coords)[0]

    def system_state(self, k, coords=MX_COORD_HELIO):
        xv = self.state(coords)
        return xv[:, self.offsets[k]:self.offsets[k + 1]]

    def close(self):
        if self.h:
            mx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """Owns one mx_system; a convenience wrapper over the C-named calls."""

    def __init__(self, workload, stream=None):
        self.w = workload
        self.params = make_params(workload.params)
        self.nbig, self.nsmall = workload.nbig, workload.nsmall
        self.n = workload.n
        self.h = mx_init_system(self.params, self.nbig, self.nsmall, workload.m_big,
                                workload.xv_helio, workload.rp_km, workload.rhop, stream)
        if getattr(workload, "growth", None) is not None:
            mx_set_growth(self.h, 0, workload.growth, self.nbig, workload.gap_c)

    def step(self, n):
        mx_step(self.h, n)

    def state(self, coords=MX_COORD_HELIO):
        return mx_get_state(self.h, self.n, coords)[0]

    def set_state(self, xv, coords=MX_COORD_HELIO, step=0):
        mx_set_state(self.h, xv, coords, step)

    def energy(self):
        return mx_energy(self.h)

    def close(self):
        if self.h:
            mx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


INF = math.inf


# ----------------------------------------------------------- differentiation
def mx_set_gas_params(sys, k, sigma1, gamma, cd_scale):
    _check(load().mx_set_gas_params(sys, int(k), float(sigma1), float(gamma), float(cd_scale)),
           "mx_set_gas_params")


def mx_kick_branches(sys, mode, max_kicks=0):
    _check(load().mx_kick_branches(sys, int(mode), int(max_kicks)), "mx_kick_branches")


def mx_encounter_log(sys, dev_ever=None, reset=False):
    nbb = ctypes.c_longlong(0)
    _check(load().mx_encounter_log(sys, _dptr(dev_ever), ctypes.byref(nbb), int(bool(reset))),
           "mx_encounter_log")
    return nbb.value


def mx_set_step_index(sys, step):
    _check(load().mx_set_step_index(sys, int(step)), "mx_set_step_index")


def mx_loss_semimajor(sys, dev_xv_helio0, dev_w, dev_seed_final, dev_seed_init, n_sys=1):
    L = np.zeros(n_sys)
    _check(load().mx_loss_semimajor(sys, _dptr(dev_xv_helio0), _dptr(dev_w), _hptr(L),
                                    _dptr(dev_seed_final), _dptr(dev_seed_init)),
           "mx_loss_semimajor")
    return L


def mx_adjoint_step(sys, dev_state_k, step_k, dev_lambda, dev_dparams):
    _check(load().mx_adjoint_step(sys, _dptr(dev_state_k), int(step_k), _dptr(dev_lambda),
                                  _dptr(dev_dparams)), "mx_adjoint_step")


def mx_predrift_state(sys, dev_xv):
    _check(load().mx_predrift_state(sys, _dptr(dev_xv)), "mx_predrift_state")


def mx_adjoint_step_predrift(sys, dev_state_k, dev_predrift_k, step_k, dev_lambda, dev_dparams):
    _check(load().mx_adjoint_step_predrift(sys, _dptr(dev_state_k), _dptr(dev_predrift_k),
                                           int(step_k), _dptr(dev_lambda), _dptr(dev_dparams)),
           "mx_adjoint_step_predrift")


def mx_adjoint_merge(sys, on):
    _check(load().mx_adjoint_merge(sys, int(bool(on))), "mx_adjoint_merge")


def mx_adjoint_flush(sys):
    _check(load().mx_adjoint_flush(sys), "mx_adjoint_flush")


def mx_adjoint_init(sys, dev_lambda, dev_grad_helio):
    _check(load().mx_adjoint_init(sys, _dptr(dev_lambda), _dptr(dev_grad_helio)),
           "mx_adjoint_init")
