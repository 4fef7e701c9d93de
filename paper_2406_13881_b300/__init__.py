"""B300-native host/device validity data-flow (OMPDart, SC24) -- Python side.

The analysis runs in ``libompdart.so`` (hand-written CUDA for sm_103a plus a
C++ host ingestion layer), reached through ``_native`` (ctypes marshalling
only).  ``workload`` draws the seeded synthetic CFGs.
"""
from . import workload  # noqa: F401

__all__ = ["workload", "analyze", "analyze_batch", "Plan", "Batch", "Server", "OmpdartError"]


def __getattr__(name):
    if name in ("analyze", "analyze_batch", "Plan", "Batch", "Server", "OmpdartError", "load"):
        from . import _native
        return getattr(_native, name)
    raise AttributeError(name)
