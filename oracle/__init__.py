"""CPU oracle for the OMPDart validity data-flow -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product library never imports, links or
calls it, and it shares no code with the CUDA path: both sides read the
same documented input format (CSR CFG + packed access words) with their own
decoders.

``solve(cfg)`` runs ``oracle.c`` (plain C11, single-threaded FIFO worklists)
and returns every intermediate and final plane as numpy arrays.  The method
is the paper's forward host/device validity analysis (Marzen et al., SC24,
Sec. IV-D and Algorithm 1); ``oracle.c`` documents each step.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain C11, -O2)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC) \
            or os.path.getmtime(_SO) < os.path.getmtime(os.path.join(_HERE, "oracle.h")):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


class _Cfg(C.Structure):
    _fields_ = [("n_blocks", C.c_int32), ("n_vars", C.c_int32), ("entry", C.c_int32),
                ("succ_off", C.c_void_p), ("succ", C.c_void_p), ("acc_off", C.c_void_p),
                ("acc", C.c_void_p), ("entry_host_valid", C.c_void_p),
                ("entry_dev_valid", C.c_void_p), ("exit_host_live", C.c_void_p),
                ("call_planes", C.c_void_p), ("n_calls", C.c_int32), ("region", C.c_void_p),
                ("data_region", C.c_int32), ("eager_to", C.c_int32)]


_OUT_FIELDS = [
    ("reachable", "N", np.uint8), ("is_header", "N", np.uint8), ("is_loop_entry", "E", np.uint8),
    ("gen_h", "NW", np.uint64), ("kill_h", "NW", np.uint64), ("gen_d", "NW", np.uint64),
    ("kill_d", "NW", np.uint64), ("ue_h", "NW", np.uint64), ("ue_d", "NW", np.uint64),
    ("def", "NW", np.uint64), ("ant_h_in", "NW", np.uint64), ("ant_d_in", "NW", np.uint64),
    ("live_in", "NW", np.uint64), ("hp_in", "NW", np.uint64), ("hp_out", "NW", np.uint64),
    ("mask_h", "NW", np.uint64), ("mask_d", "NW", np.uint64), ("d_in", "NW", np.uint64),
    ("d_out", "NW", np.uint64), ("hm", "NW", np.uint64), ("h_in", "NW", np.uint64),
    ("h_out", "NW", np.uint64), ("to_edge", "EW", np.uint64), ("from_edge", "EW", np.uint64),
    ("from_exit", "NW", np.uint64), ("acc_flag", "A", np.uint8),
    ("call_to", "SW", np.uint64), ("call_from", "SW", np.uint64), ("call_entry_h", "SW", np.uint64),
    ("call_entry_d", "SW", np.uint64), ("call_exit_live", "SW", np.uint64),
    ("in_region", "N", np.uint8), ("region_exit", "E", np.uint8), ("ant_dm_in", "NW", np.uint64),
]


class _Out(C.Structure):
    _fields_ = [(name, C.c_void_p) for name, _, _ in _OUT_FIELDS]


class OracleError(RuntimeError):
    pass


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.oracle_solve.argtypes = [C.POINTER(_Cfg), C.POINTER(_Out)]
            lib.oracle_solve.restype = C.c_int
            lib.oracle_summarize.argtypes = [C.POINTER(_Cfg), C.c_void_p]
            lib.oracle_summarize.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _cfg_struct(g):
    n, nv = int(g["n_blocks"]), int(g["n_vars"])
    W = (nv + 63) // 64
    keep = {
        "so": np.ascontiguousarray(g["succ_off"], dtype=np.int32),
        "s": np.ascontiguousarray(g["succ"], dtype=np.int32),
        "ao": np.ascontiguousarray(g["acc_off"], dtype=np.int32),
        "acc": np.ascontiguousarray(g["acc"], dtype=np.uint32),
    }
    for key in ("entry_host_valid", "entry_dev_valid", "exit_host_live", "call_planes"):
        v = g.get(key)
        keep[key] = None if v is None else np.ascontiguousarray(v, dtype=np.uint64)
    calls = keep["call_planes"]
    c = _Cfg(n, nv, int(g.get("entry", 0)), _ptr(keep["so"]), _ptr(keep["s"]), _ptr(keep["ao"]),
             _ptr(keep["acc"]), _ptr(keep["entry_host_valid"]), _ptr(keep["entry_dev_valid"]),
             _ptr(keep["exit_host_live"]), _ptr(calls), 0 if calls is None else int(calls.size // (7 * W)))
    return c, keep


def summarize(cfg) -> np.ndarray:
    """Side-effect summary of a callee in its own variable numbering:
    [7, W] planes ReqH, ReqD, GenH, KillH, GenD, KillD, MustDef (see
    oracle_summarize in oracle.h)."""
    lib = _load()
    g = cfg if isinstance(cfg, dict) else cfg.__dict__
    W = (int(g["n_vars"]) + 63) // 64
    c, _keep = _cfg_struct(g)
    out = np.zeros((7, W), dtype=np.uint64)
    rc = lib.oracle_summarize(C.byref(c), out.ctypes.data)
    if rc != 0:
        raise OracleError("oracle_summarize returned %d" % rc)
    return out


def solve(cfg, want=None, data_region=False, eager_to=False) -> dict:
    """Run the oracle on ``cfg`` (an object with the CSR fields of
    ``paper_2406_13881_b300.workload.CFG`` or a dict with the same keys).

    ``want``: iterable of output names to produce (default: all).  Returns a
    dict of numpy arrays; plane outputs are shaped [rows, W].
    ``data_region``: the single target data region of Sec. IV-D around the
    kernels given by ``cfg.region`` (see oracle_cfg.data_region).
    ``eager_to``: eager `to' placement after the producing host write
    (Sec. IV-E; see oracle_cfg.eager_to)."""
    lib = _load()
    g = cfg if isinstance(cfg, dict) else cfg.__dict__
    n, nv = int(g["n_blocks"]), int(g["n_vars"])
    W = (nv + 63) // 64
    so = np.ascontiguousarray(g["succ_off"], dtype=np.int32)
    s = np.ascontiguousarray(g["succ"], dtype=np.int32)
    ao = np.ascontiguousarray(g["acc_off"], dtype=np.int32)
    acc = np.ascontiguousarray(g["acc"], dtype=np.uint32)
    E, A = int(so[-1]), int(ao[-1])

    def opt(key):
        v = g.get(key)
        return None if v is None else np.ascontiguousarray(v, dtype=np.uint64)

    ehv, edv, xhl = opt("entry_host_valid"), opt("entry_dev_valid"), opt("exit_host_live")
    calls = opt("call_planes")
    reg = g.get("region")
    reg = None if reg is None else np.ascontiguousarray(reg, dtype=np.int32)
    c = _Cfg(n, nv, int(g.get("entry", 0)), _ptr(so), _ptr(s), _ptr(ao), _ptr(acc),
             _ptr(ehv), _ptr(edv), _ptr(xhl), _ptr(calls),
             0 if calls is None else int(calls.size // (7 * W)), _ptr(reg),
             int(bool(data_region) and reg is not None), int(bool(eager_to)))
    S = int(np.count_nonzero(acc >> np.uint32(31)))
    sizes = {"N": (n,), "E": (E,), "A": (A,), "NW": (n, W), "EW": (E, W), "SW": (S, W)}
    res, ptrs = {}, {}
    want = None if want is None else set(want)
    for name, kind, dt in _OUT_FIELDS:
        if want is None or name in want:
            res[name] = np.zeros(sizes[kind], dtype=dt)
            ptrs[name] = res[name].ctypes.data
        else:
            ptrs[name] = None
    o = _Out(**ptrs)
    rc = lib.oracle_solve(C.byref(c), C.byref(o))
    if rc != 0:
        raise OracleError("oracle_solve returned %d" % rc)
    return res
