"""Disk gravity (Eqs. 10-12) on the GPU against the oracle.

The kick adds the disk's radial force on planetesimals to the big bodies'
gravity.  Checked: the acceleration of mx_accel / mx_gas_drag at 1e-12 for the
gamma = 1 edge form and for gamma != 1 (the series S(gamma), which the library
and the oracle sum by different methods); positions after a run; the deferred
path bit for bit; and the adjoint through the disk's gravity.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2601_16791_gb300 import mx, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _workload(gamma, r_in, nsmall=20_000, nsteps=10):
    w = W.gas_4core_100k(nsmall=nsmall, nsteps=nsteps)
    gas = dict(w.params["gas"], gamma=gamma, r_in_au=r_in, disk_gravity=True)
    w.params = dict(w.params, gas=gas)
    return w


def rel_rows(a, b):
    num = np.linalg.norm(np.asarray(a) - np.asarray(b), axis=0)
    den = np.linalg.norm(np.asarray(b), axis=0)
    return float(np.max(num / np.maximum(den, 1e-300)))


@pytest.mark.parametrize("gamma,r_in", [(1.0, 1.5), (1.5, 1.0), (0.7, 0.0)])
def test_accel_with_disk_gravity(gamma, r_in):
    w = _workload(gamma, r_in)
    g = mx.System(w)
    p = orc.make_params(w.params)
    xv, mu, rc = orc.init(p, w.nbig, w.nsmall, w.m_big, w.xv_helio)
    acc = torch.zeros((3, w.n), dtype=torch.float64, device="cuda")
    mx.mx_accel(g.h, acc)
    ref = orc.accel_grav(w.nbig, xv, mu, rc)
    gas = orc.gas_drag(p, w.nbig, xv, mu, w.rp_km, w.rhop)
    ref[:, w.nbig:] += gas
    assert rel_rows(acc.cpu().numpy(), ref) <= 1e-12
    # the disk's share is not negligible: it changes the acceleration
    off = orc.make_params(dict(w.params, gas=dict(w.params["gas"], disk_gravity=False)))
    drag_only = orc.gas_drag(off, w.nbig, xv, mu, w.rp_km, w.rhop)
    assert np.max(np.linalg.norm(gas - drag_only, axis=0)) > 0
    sm = torch.zeros((3, w.nsmall), dtype=torch.float64, device="cuda")
    mx.mx_gas_drag(g.h, sm)
    inside = np.linalg.norm(gas, axis=0) == 0
    assert rel_rows(sm.cpu().numpy()[:, ~inside], gas[:, ~inside]) <= 1e-12
    g.close()


@pytest.mark.parametrize("gamma,r_in", [(1.0, 1.5), (1.5, 1.0)])
def test_run_with_disk_gravity(gamma, r_in):
    w = _workload(gamma, r_in, nsmall=3000, nsteps=200)
    g = mx.System(w)
    g.step(w.nsteps)
    out = g.state(mx.MX_COORD_DH)
    g.close()
    p = orc.make_params(w.params)
    xv, mu, rc = orc.init(p, w.nbig, w.nsmall, w.m_big, w.xv_helio)
    ref, ever, _, _ = orc.step(p, w.nbig, xv, mu, rc, w.rp_km, w.rhop, w.nsteps)
    keep = ever == 0
    err = np.linalg.norm(out[:3] - ref[:3], axis=0) / np.linalg.norm(ref[:3], axis=0)
    assert keep.sum() > 2000 and err[keep].max() <= 1e-9


def test_deferred_path_with_disk_gravity_is_bit_identical():
    w = _workload(1.5, 1.0, nsmall=60_000, nsteps=30)
    out = []
    for window in (0, 8):
        g = mx.System(w)
        mx.mx_set_defer_window(g.h, window)
        n0 = mx.mx_defer_stats(g.h)[2]
        g.step(w.nsteps)
        out.append((g.state(mx.MX_COORD_DH), mx.mx_defer_stats(g.h)[2] - n0))
        g.close()
    assert out[1][1] > 0
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("gamma,r_in", [(1.5, 1.0), (1.0, 1.5)])
def test_adjoint_with_disk_gravity_vs_oracle_jvp(gamma, r_in):
    """The adjoint through the disk's gravity (a radial force on planetesimals
    in the gas: position and, through Sigma and S(gamma), sigma1 and gamma)
    against the oracle's dual-number JVP, encountered planetesimals masked as
    in the plain adjoint test; relative <= 1e-8.  At gamma = 1 the force is the
    edge form of Eq. 12, a branch in gamma, so gamma is not perturbed there."""
    from paper_2601_16791_gb300.autograd import Trajectory, semimajor_loss
    w = W.adjoint_4core_50k(nsmall=300, nsteps=40, checkpoint_every=10)
    w.params = dict(w.params, gas=dict(w.params["gas"], gamma=gamma, r_in_au=r_in,
                                       disk_gravity=True))
    traj = Trajectory(w)
    g = w.params["gas"]
    xv0 = torch.tensor(w.xv_helio, dtype=torch.float64, device="cuda", requires_grad=True)
    gas = torch.tensor([g["sigma1_gcm2"], g["gamma"], g["cd_scale"]], dtype=torch.float64,
                       device="cuda", requires_grad=True)
    wts = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    wts[w.nbig:] = 1.0 / w.nsmall
    L = semimajor_loss(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every, mask_encounters=True)
    L.backward()
    gx, gp = xv0.grad.cpu().numpy(), gas.grad.cpu().numpy()
    ever = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    mx.mx_encounter_log(traj.h, ever)
    traj.close()
    w_small = (1.0 / w.nsmall) * (1 - ever.cpu().numpy()[w.nbig:].astype(float))
    p = orc.make_params(w.params)
    rng = np.random.default_rng(21)
    for _ in range(3):
        dxv = np.zeros((6, w.n))
        dxv[:3] = rng.normal(0, 1e-4, (3, w.n))
        dxv[3:] = rng.normal(0, 1e-6, (3, w.n))
        dpar = np.array([17.0, 0.01 if gamma != 1.0 else 0.0, 0.01]) * rng.normal(0, 1, 3)
        Lo, jvp = orc.jvp_loss(p, w.nbig, w.m_big, w.xv_helio, w.rp_km, w.rhop, w_small,
                               w.nsteps, dxv, dpar)
        ours = float((gx * dxv).sum() + (gp * dpar).sum())
        assert abs(Lo - float(L.detach())) <= 1e-9 * abs(Lo)
        assert abs(ours - jvp) <= 1e-8 * abs(jvp), (ours, jvp)
