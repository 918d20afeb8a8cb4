"""The batched ensemble (mx_init_batch) and the tiling autotuner.

A batch runs every kernel once over all systems; each system's arithmetic is
the same as when it runs alone, so batched and one-by-one results must agree
bit for bit, whatever tile size and order the autotuner picks.  One member is
also checked against the oracle.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2601_16791_gb300 import mx, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _members():
    ens = W.ensemble_256(nsys=5, nsmall_min=300, nsmall_max=3000)
    ens[1].params = dict(ens[1].params, dt=7.0)                       # different step
    g0 = dict(ens[2].params["gas"], enabled=False)
    ens[2].params = dict(ens[2].params, gas=g0)                       # one without gas
    ens.append(W.plain_2big_1k(nsmall=257))
    return ens


def test_batch_equals_systems_run_alone():
    ws = _members()
    b = mx.Batch(ws)
    b.step(15)
    for k, w in enumerate(ws):
        alone = mx.System(w)
        alone.step(15)
        ref = alone.state(mx.MX_COORD_DH)
        alone.close()
        assert np.array_equal(b.system_state(k, mx.MX_COORD_DH), ref), k
    E, L = mx.mx_energy_batch(b.h, len(ws))
    for k, w in enumerate(ws):
        alone = mx.System(w)
        alone.step(15)
        e1, l1 = alone.energy()
        alone.close()
        assert E[k] == e1 and np.array_equal(L[k], l1)
    b.close()


def test_tiling_does_not_change_results():
    ws = _members()
    outs = []
    for tile in (64, 96, 128, 224, 256):
        for order in (0, 1):
            b = mx.Batch(ws)
            mx.mx_set_tiling(b.h, tile, order)
            assert mx.mx_tiling(b.h) == (tile, order)
            b.step(8)
            outs.append(b.state(mx.MX_COORD_DH))
            b.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_batch_member_vs_oracle():
    ws = _members()
    b = mx.Batch(ws)
    nsteps = 40
    b.step(nsteps)
    for k in (0, 1, 5):
        w = ws[k]
        p = orc.make_params(w.params)
        xv, mu, rc = orc.init(p, w.nbig, w.nsmall, w.m_big, w.xv_helio)
        ref, ever, _, _ = orc.step(p, w.nbig, xv, mu, rc, w.rp_km, w.rhop, nsteps)
        got = b.system_state(k, mx.MX_COORD_DH)
        keep = ever == 0
        err = np.linalg.norm(got[:3] - ref[:3], axis=0) / np.linalg.norm(ref[:3], axis=0)
        assert err[keep].max() <= 1e-9, (k, err[keep].max())
    b.close()


def test_batch_with_ejection_schedule():
    """Two scattering swarms on the same ejection schedule: in a batch and
    alone they take the same steps, so states and removals agree bit for bit,
    and the per-system removal counts are each system's own."""
    ws = [W.scatter_2giant(seed=s, nsmall=600, eject_every=5) for s in (5, 7)]
    b = mx.Batch(ws)
    b.step(23)
    stat_b, cnt_b = mx.mx_body_status(b.h, b.n, len(ws))
    for k, w in enumerate(ws):
        alone = mx.System(w)
        alone.step(23)
        assert np.array_equal(b.system_state(k, mx.MX_COORD_DH), alone.state(mx.MX_COORD_DH))
        stat, cnt = mx.mx_body_status(alone.h, w.n)
        alone.close()
        lo, hi = b.offsets[k], b.offsets[k + 1]
        assert np.array_equal(stat_b[lo:hi], stat) and cnt_b[k] == cnt[0] > 100
    b.close()


def test_batch_with_one_growing_system():
    """Growth tracks on system 0 only (mx_set_growth with its index): system 0
    matches its run alone bit for bit (both end every step with their own half
    kick), system 1 runs the same map with split kicks (positions of bodies
    that met no planet within 1e-12), and the masses are the growing system's."""
    g = W.growth_2giant(nsmall=500, tau_c_days=400.0, tau_g_days=200.0)
    p = W.plain_2big_1k(nsmall=300)
    p.params = dict(p.params, dt=10.0)
    b = mx.Batch([g, p])
    mx.mx_set_growth(b.h, 0, g.growth, g.nbig, g.gap_c)
    b.step(60)
    alone = mx.System(g)
    alone.step(60)
    assert np.array_equal(b.system_state(0, mx.MX_COORD_DH), alone.state(mx.MX_COORD_DH))
    m_alone, _ = mx.mx_planets(alone.h, g.nbig)
    alone.close()
    m_b, _ = mx.mx_planets(b.h, g.nbig + p.nbig)
    assert np.array_equal(m_b[:g.nbig], m_alone) and m_b[0] > 10 * g.m_big[0]
    assert np.allclose(m_b[g.nbig:], p.m_big, rtol=1e-15, atol=0)
    other = mx.System(p)
    other.step(60)
    ref = other.state(mx.MX_COORD_DH)
    ever = torch.zeros(p.n, dtype=torch.uint8, device="cuda")
    mx.mx_encounter_log(other.h, ever)
    other.close()
    got = b.system_state(1, mx.MX_COORD_DH)
    err = np.linalg.norm(got[:3] - ref[:3], axis=0) / np.linalg.norm(ref[:3], axis=0)
    quiet = ever.cpu().numpy() == 0
    assert quiet.sum() > 200 and err[quiet].max() <= 1e-12
    b.close()
