"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/*.h.  No compute calls are made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"\b(?:mx_status|void|const char\s*\*)\s+(mx_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for required in ("mx_init_system", "mx_step", "mx_detect_encounters", "mx_gas_drag",
                     "mx_energy", "mx_destroy", "mx_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2601_16791_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2601_16791_gb300 import mx
    names = set(declared_symbols())
    bound = set(mx.exported_symbols())
    assert names <= bound | {n for n in names if n.startswith("mx_batch") or "adjoint" in n}


def test_kernels_are_sm_103a_native_source():
    """The hot path is hand-written CUDA: no Triton, no torch.compile, no fallback module."""
    src = " ".join(open(p).read() for p in glob.glob(os.path.join(ROOT, "paper_2601_16791_gb300", "*.py")))
    for banned in ("import triton", "torch.compile", "import oracle", "from oracle"):
        assert banned not in src


def test_ejection_schedule_is_checked_on_the_host():
    """A negative eject_every, or a batch whose systems disagree on it, is
    refused before any device work (MX_ERR_ARG)."""
    from paper_2601_16791_gb300 import mx, workloads as W
    w = W.scatter_2giant(nsmall=10, eject_every=5)
    bad = mx.make_params(dict(w.params, eject_every=-1))
    with pytest.raises(mx.MxError) as e:
        mx.mx_init_system(bad, w.nbig, w.nsmall, w.m_big, w.xv_helio)
    assert e.value.status == "MX_ERR_ARG"
    w0 = W.scatter_2giant(nsmall=10, eject_every=0)
    with pytest.raises(mx.MxError) as e:
        mx.mx_init_batch([w, w0])
    assert e.value.status == "MX_ERR_ARG" and "eject_every" in str(e.value)
