"""GB300 (sm_103a) FP64 hot path of the Mercury-style hybrid symplectic step
(arXiv 2601.16791): K-weighted kick with gas drag, Kepler drift, encounter
detection and grouped Bulirsch-Stoer, behind the C ABI of include/mx.h.

``mx`` is the thin ctypes binding (same names as the C entry points);
``workloads`` draws the seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["mx", "workloads"]
