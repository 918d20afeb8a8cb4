"""Deferred planetesimals (mx_set_defer_window) against the direct path.

A planetesimal whose Bulirsch-Stoer group outlasts the packed phase leaves
the step and is brought to the end of the window by the catch-up launch,
which replays the direct path's arithmetic on the recorded big-body states.
Every test here runs the same workload with deferral on and off and requires
the states, the encounter log and the last step's pair list to agree exactly;
each one also checks that bodies were in fact deferred, so none of them
passes vacuously.
"""
import numpy as np
import pytest

from paper_2601_16791_gb300 import mx, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _run(w, window, calls):
    s = mx.System(w)
    mx.mx_set_defer_window(s.h, window)
    st0 = mx.mx_defer_stats(s.h)      # (the autotuner's trial steps may have deferred)
    for n in calls:
        s.step(n)
    state = s.state(mx.MX_COORD_DH)
    ever = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    nbb = mx.mx_encounter_log(s.h, ever)
    pairs = mx.mx_last_encounters(s.h)
    E, L = s.energy()
    st1 = mx.mx_defer_stats(s.h)
    stats = (st1[0], st1[1], st1[2] - st0[2], st1[3] - st0[3])
    s.close()
    return state, ever.cpu().numpy(), nbb, pairs, (float(E), tuple(np.ravel(L).tolist())), stats


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert a[2] == b[2]
    assert np.array_equal(np.asarray(a[3]), np.asarray(b[3]))
    assert a[4] == b[4]


def test_gas_disk_deferred_equals_direct():
    w = W.gas_4core_100k(nsmall=100_000)
    direct = _run(w, 0, [40])
    deferred = _run(w, 16, [40])
    assert direct[5][2] == 0 and direct[5][0] == 0
    assert deferred[5][0] == 16
    assert deferred[5][2] > 0, "no body was deferred: the test is vacuous"
    # 41 history slots (the leading half kick and 40 steps): window ends after
    # slots 16 and 32 and, for the last 9, a settle when the state is read
    assert deferred[5][3] == 3
    _same(direct, deferred)


@pytest.mark.parametrize("window", [1, 5, 32])
def test_windows_and_call_boundaries(window):
    # windows span calls: a body deferred in one call is replayed through the
    # next call's leading half kick
    w = W.gas_4core_100k(nsmall=60_000)
    calls = [7, 1, 13, 19, 1, 1, 1]
    direct = _run(w, 0, calls)
    deferred = _run(w, window, calls)
    assert deferred[5][2] > 0
    _same(direct, deferred)


def test_many_big_bodies():
    # 40 giant cores (up to 64 big bodies defer), so the replayed kick and
    # detection loop over many sources and groups often have several bigs
    w = W.gas_4core_100k(nbig=40, nsmall=60_000)
    direct = _run(w, 0, [30])
    deferred = _run(w, 8, [30])
    assert deferred[5][2] > 0
    _same(direct, deferred)


def test_no_deferral_beyond_64_big_bodies():
    w = W.semiactive_2000big_200k(nbig=200, nsmall=20_000)
    direct = _run(w, 0, [30])
    deferred = _run(w, 8, [30])
    assert deferred[5][2] == 0
    _same(direct, deferred)


def test_batch_deferred_equals_direct():
    ws = W.ensemble_256(nsys=6, nsmall_min=2000, nsmall_max=30_000)
    out = []
    for window in (0, 10):
        b = mx.Batch(ws)
        mx.mx_set_defer_window(b.h, window)
        n0 = mx.mx_defer_stats(b.h)[2]
        b.step(25)
        out.append((b.state(mx.MX_COORD_DH), mx.mx_defer_stats(b.h)[2] - n0))
        b.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == 0


def test_profiled_path_defers_too():
    w = W.gas_4core_100k(nsmall=50_000)
    s = mx.System(w)
    mx.mx_set_defer_window(s.h, 8)
    n0 = mx.mx_defer_stats(s.h)[2]
    ms, cnt, tot = mx.mx_step_profiled(s.h, 20)
    assert mx.mx_defer_stats(s.h)[2] > n0
    # 21 slots: window ends after slots 8 and 16 (a side-stream launch
    # each; on the main stream one launch at the first, two at the second,
    # where the bodies deferred in the window go before the wait for the
    # side stream and the carried ones after it), the last 5 slots wait for a
    # reader; side launches are counted once they have completed, at the
    # latest by the settling call (two main-stream launches, as at a window
    # end with the side stream busy)
    assert cnt["k_jump_drift"] == 20 and cnt["k_catchup"] == 3
    ms0, cnt0, _ = mx.mx_step_profiled(s.h, 0)
    assert cnt0["k_catchup"] == 2 and cnt0["k_jump_drift"] == 0
    assert cnt["k_catchup_side"] + cnt0["k_catchup_side"] == 2
    a = s.state(mx.MX_COORD_DH)
    s.close()
    ref = _run(w, 0, [20])
    assert np.array_equal(a, ref[0])


def test_branch_recording_turns_deferral_off():
    w = W.gas_4core_100k(nsmall=5_000)
    s = mx.System(w)
    assert mx.mx_defer_stats(s.h)[0] > 0
    mx.mx_kick_branches(s.h, 1, 64)
    assert mx.mx_defer_stats(s.h)[0] == 0
    mx.mx_kick_branches(s.h, 0, 0)
    assert mx.mx_defer_stats(s.h)[0] > 0
    s.close()


def test_window_limits():
    w = W.plain_2big_1k(nsmall=100)
    s = mx.System(w)
    _, max_window, _, _ = mx.mx_defer_stats(s.h)
    assert 1 <= max_window <= 64
    with pytest.raises(mx.MxError):
        mx.mx_set_defer_window(s.h, max_window + 1)
    with pytest.raises(mx.MxError):
        mx.mx_set_defer_window(s.h, -1)
    mx.mx_set_defer_window(s.h, max_window)
    s.step(max_window + 3)
    s.close()


def test_timed_path_with_flush_matches_step():
    w = W.gas_4core_100k(nsmall=30_000)
    flush = torch.empty(8 * 1024 * 1024, dtype=torch.float32, device="cuda")
    s = mx.System(w)
    ms, cnt, tot = mx.mx_step_timed(s.h, 25, flush)
    ms0, cnt0, tot0 = mx.mx_step_timed(s.h, 0, flush)
    a = s.state(mx.MX_COORD_DH)
    s.close()
    assert tot > 0 and cnt["k_jump_drift"] == 25 and cnt["k_jump_kick"] == 26
    assert np.array_equal(a, _run(w, 32, [25])[0])


def test_production_graph_spans_match_step():
    """mx_step_timed with no per-kernel outputs runs the production graphs
    with events only around each step: the same states as mx_step."""
    w = W.gas_4core_100k(nsmall=30_000)
    flush = torch.empty(8 * 1024 * 1024, dtype=torch.float32, device="cuda")
    s = mx.System(w)
    ms, cnt, tot = mx.mx_step_timed(s.h, 25, flush, per_kernel=False)
    _, _, tot0 = mx.mx_step_timed(s.h, 0, flush, per_kernel=False)
    a = s.state(mx.MX_COORD_DH)
    s.close()
    assert tot > 0 and ms == {} and cnt == {}
    assert np.array_equal(a, _run(w, 32, [25])[0])
