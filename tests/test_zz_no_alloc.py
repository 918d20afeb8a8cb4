"""Encounter detection for callers that cannot allocate device memory.

Some users of this library run it inside a host application that owns all
GPU memory through its own pool, or inside a latency-critical loop where an
allocation's implicit device synchronisation is not acceptable; they cannot
call cudaMalloc.  mx_detect_encounters_noalloc serves them from a fixed array
in the library's static device memory.  This test calls it through the C ABI
twice in a row, on two different step states, and checks each result against
mx_detect_encounters (the allocating entry point) and against the CPU
oracle's detection on the same inputs: the same sorted pair list and the same
flags, except pairs within 1e-9 relative of the changeover threshold (the
tolerance of the detection parity tests).  It also checks the overflow
contract (a cap below the pair count) and that a call takes no device memory.
"""
import ctypes

import numpy as np
import pytest

import oracle as orc
from paper_2601_16791_gb300 import mx, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _near(p, xv0, xv1, rcrit, i, j):
    dx0 = xv0[:3, j] - xv0[:3, i]
    dx1 = xv1[:3, j] - xv1[:3, i]
    dv0 = xv0[3:, j] - xv0[3:, i]
    dv1 = xv1[3:, j] - xv1[3:, i]
    d0, d1 = dx0 @ dx0, dx1 @ dx1
    m = min(d0, d1, orc.hermite_d2min(d0, d1, 2 * dx0 @ dv0, 2 * dx1 @ dv1, p.dt))
    rc = max(rcrit[i], rcrit[j])
    return abs(m - rc * rc) <= 1e-9 * rc * rc


def _inputs(w):
    p = orc.make_params(w.params)
    xv0, mu, rc = orc.init(p, w.nbig, w.nsmall, w.m_big, w.xv_helio)
    xv1, _ = orc.drift(p, xv0, p.dt)
    return p, xv0, xv1, rc


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _same_up_to_threshold(p, xv0, xv1, rc, got, ref):
    A, B = set(map(tuple, got.tolist())), set(map(tuple, ref.tolist()))
    for (i, j) in A ^ B:
        assert _near(p, xv0, xv1, rc, i, j), (i, j)
    return A, B


def _noalloc_raw(w, xv0, xv1, rc, cap):
    L = mx.load()
    params = mx.make_params(w.params)
    d0, d1, drc = _dev(xv0), _dev(xv1), _dev(rc)
    flags = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    n = ctypes.c_int(0)
    st = torch.cuda.current_stream().cuda_stream
    code = L.mx_detect_encounters_noalloc(
        ctypes.byref(params), w.nbig, w.n, ctypes.c_void_p(drc.data_ptr()),
        ctypes.c_void_p(d0.data_ptr()), ctypes.c_void_p(d1.data_ptr()),
        ctypes.c_void_p(flags.data_ptr()), ctypes.c_void_p(pairs.data_ptr()), cap,
        ctypes.byref(n), ctypes.c_void_p(st))
    return code, n.value, pairs.cpu().numpy(), flags.cpu().numpy()


def _noalloc(w, xv0, xv1, rc, cap):
    code, n, pairs, flags = _noalloc_raw(w, xv0, xv1, rc, cap)
    assert code == mx.MX_OK, mx.STATUS.get(code, code)
    return pairs[:2 * n].reshape(-1, 2), flags


def _allocating(w, xv0, xv1, cap):
    g = mx.System(w)
    flags = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    n = mx.mx_detect_encounters(g.h, _dev(xv0), _dev(xv1), flags, pairs, cap)
    g.close()
    return pairs.cpu().numpy()[:2 * n].reshape(-1, 2), flags.cpu().numpy()


def test_noalloc_detection_matches_allocating_entry_point_twice():
    cases = [W.semiactive_2000big_200k(nbig=400, nsmall=5000), W.plain_2big_1k()]
    for w in cases:                       # two calls in a row on different inputs
        p, xv0, xv1, rc = _inputs(w)
        cap = 1 << 14
        got, fg = _noalloc(w, xv0, xv1, rc, cap)
        ref, fr = _allocating(w, xv0, xv1, cap)
        assert len(ref) > 5
        A, B = _same_up_to_threshold(p, xv0, xv1, rc, got, ref)
        assert np.array_equal(got, np.array(sorted(A)).reshape(-1, 2))
        if A == B:
            assert np.array_equal(fg, fr)
        # and against the oracle's detection (the definition, on the CPU)
        fo, po = orc.detect(p, w.nbig, xv0, xv1, rc)
        A, C = _same_up_to_threshold(p, xv0, xv1, rc, got, po)
        if A == C:
            assert np.array_equal(fg, fo)


def test_noalloc_overflow_returns_the_full_count_and_the_first_pairs():
    w = W.semiactive_2000big_200k(nbig=400, nsmall=5000)
    p, xv0, xv1, rc = _inputs(w)
    full, _ = _noalloc(w, xv0, xv1, rc, 1 << 14)
    assert len(full) > 3
    cap = 2
    code, n, pairs, _ = _noalloc_raw(w, xv0, xv1, rc, cap)
    assert code == 6, mx.STATUS.get(code, code)    # MX_ERR_PAIR_OVERFLOW
    assert n == len(full)
    assert np.array_equal(pairs[:2 * cap].reshape(-1, 2), full[:cap])


def test_noalloc_takes_no_device_memory():
    w = W.plain_2big_1k()
    p, xv0, xv1, rc = _inputs(w)
    _noalloc(w, xv0, xv1, rc, 1 << 10)          # first call: address look-up
    torch.cuda.synchronize()
    # inputs and outputs allocated up front; the call itself must not move
    # the device's free memory
    L = mx.load()
    params = mx.make_params(w.params)
    d0, d1, drc = _dev(xv0), _dev(xv1), _dev(rc)
    flags = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    pairs = torch.zeros(2 << 10, dtype=torch.int32, device="cuda")
    n = ctypes.c_int(0)
    st = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        code = L.mx_detect_encounters_noalloc(
            ctypes.byref(params), w.nbig, w.n, ctypes.c_void_p(drc.data_ptr()),
            ctypes.c_void_p(d0.data_ptr()), ctypes.c_void_p(d1.data_ptr()),
            ctypes.c_void_p(flags.data_ptr()), ctypes.c_void_p(pairs.data_ptr()), 1 << 10,
            ctypes.byref(n), ctypes.c_void_p(st))
        assert code == mx.MX_OK
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_array():
    L = mx.load()
    w = W.plain_2big_1k(nsmall=10)
    params = mx.make_params(w.params)
    n = ctypes.c_int(0)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    code = L.mx_detect_encounters_noalloc(ctypes.byref(params), 2, (1 << 21) + 1, ptr, ptr, ptr,
                                          ptr, ptr, 0, ctypes.byref(n), None)
    assert code == 1   # MX_ERR_ARG
