"""The persistent step (mx_set_persistent): every interior step as one
cooperative launch over all systems, with grid barriers between the phases.
It runs the per-kernel step's device functions on the same tiles, so the
state, the encounter log and the last pair list must be the per-kernel
step's bit for bit, for one system and for a batch, across calls and
deferral windows.  A barrier that gives up (a spin limit of 0) must end the
launch and come back as MX_ERR_BARRIER_TIMEOUT, with no hang, leaving the
device usable."""
import numpy as np
import pytest

from paper_2601_16791_gb300 import mx, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _log(h, n):
    ev = torch.zeros(n, dtype=torch.uint8, device="cuda")
    mx.mx_encounter_log(h, ev)
    return ev.cpu().numpy()


def _run_system(w, persist, calls):
    s = mx.System(w)
    if persist:
        mx.mx_set_persistent(s.h, True)
    else:
        mx.mx_set_tiling(s.h, 256, 0)
    for n in calls:
        s.step(n)
    out = (s.state(mx.MX_COORD_DH), _log(s.h, w.n), mx.mx_last_encounters(s.h))
    s.close()
    return out


def test_persistent_step_bitwise_one_system():
    w = W.gas_4core_100k(nsmall=20_000)
    a = _run_system(w, False, [17, 13, 1, 9])
    b = _run_system(w, True, [17, 13, 1, 9])
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1]) and a[1][w.nbig:].sum() > 20
    assert np.array_equal(a[2], b[2])


def test_persistent_step_bitwise_semiactive():
    """Big-big groups, more than 32 big bodies (the kick's momentum tree)."""
    w = W.semiactive_2000big_200k(nbig=300, nsmall=3000)
    a = _run_system(w, False, [12, 8])
    b = _run_system(w, True, [12, 8])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_persistent_step_bitwise_batch():
    ws = W.ensemble_256(nsys=24, nsmall_max=20_000)
    outs = []
    for persist in (False, True):
        b = mx.Batch(ws)
        if persist:
            mx.mx_set_persistent(b.h, True)
        else:
            mx.mx_set_tiling(b.h, 256, 1)
        b.step(14)
        b.step(7)
        outs.append((b.state(mx.MX_COORD_DH), _log(b.h, b.n)))
        b.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_persistent_barrier_gives_up_without_hanging():
    w = W.gas_4core_100k(nsmall=5_000)
    s = mx.System(w)
    mx.mx_set_persistent(s.h, True, 0)        # a barrier polls once, then gives up
    with pytest.raises(mx.MxError) as exc:
        s.step(2)                              # head, one persistent step, last step
    assert exc.value.status == "MX_ERR_BARRIER_TIMEOUT"
    s.close()
    # the device is still usable: a fresh system steps as the per-kernel path does
    a = _run_system(w, False, [6])
    b = _run_system(w, True, [6])
    assert np.array_equal(a[0], b[0])
