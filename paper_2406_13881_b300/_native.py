"""ctypes binding of libompdart.so (argument marshalling only).

Every step of the analysis runs in the library's CUDA kernels; this module
only converts numpy inputs to the C structs of ``include/ompdart.h`` and the
results back to numpy.  There is no fallback: if the shared library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libompdart.so")
_lock = threading.Lock()
_lib = None

OK = 0
E_INVALID, E_NOMEM, E_BUDGET, E_NOCONVERGE, E_CUDA, E_TIMEOUT = -1, -2, -3, -4, -5, -6
ERROR_NAMES = {-1: "E_INVALID", -2: "E_NOMEM", -3: "E_BUDGET", -4: "E_NOCONVERGE", -5: "E_CUDA",
               -6: "E_TIMEOUT"}


class OmpdartError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "error"), code, msg))
        self.code = code


class Cfg(C.Structure):
    _fields_ = [("n_blocks", C.c_int32), ("n_vars", C.c_int32), ("entry", C.c_int32),
                ("succ_off", C.c_void_p), ("succ", C.c_void_p), ("acc_off", C.c_void_p),
                ("acc", C.c_void_p), ("entry_host_valid", C.c_void_p),
                ("entry_dev_valid", C.c_void_p), ("exit_host_live", C.c_void_p),
                ("call_planes", C.c_void_p), ("n_calls", C.c_int32), ("mem", C.c_int32),
                ("region", C.c_void_p), ("scalar_vars", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("max_sweeps", C.c_int32), ("keep_states", C.c_int32), ("path", C.c_int32),
                ("chunk_target", C.c_int32), ("device", C.c_int32), ("warps_per_cta", C.c_int32),
                ("tune", C.c_int32), ("no_graph", C.c_int32), ("data_region", C.c_int32),
                ("eager_to", C.c_int32)]


class EdgeXfer(C.Structure):
    _fields_ = [("edge", C.c_int32), ("word", C.c_int32), ("to_bits", C.c_uint64),
                ("from_bits", C.c_uint64)]


XFER_DTYPE = np.dtype([("edge", np.int32), ("word", np.int32), ("to_bits", np.uint64),
                       ("from_bits", np.uint64)])


class Result(C.Structure):
    _fields_ = [("n_blocks", C.c_int32), ("n_vars", C.c_int32), ("n_words", C.c_int32),
                ("n_edges", C.c_int32), ("n_acc", C.c_int32), ("n_exits", C.c_int32),
                ("mem", C.c_int32), ("h_in", C.c_void_p), ("d_in", C.c_void_p),
                ("h_out", C.c_void_p), ("d_out", C.c_void_p), ("acc_flag", C.c_void_p),
                ("n_edge_xfers", C.c_int32), ("edge_xfers", C.c_void_p),
                ("exit_blocks", C.c_void_p), ("from_exit", C.c_void_p), ("path", C.c_int32),
                ("sweeps", C.c_int32), ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64),
                ("live_in", C.c_void_p), ("n_call_sites", C.c_int32), ("call_site_acc", C.c_void_p),
                ("call_to", C.c_void_p), ("call_from", C.c_void_p), ("call_entry_h", C.c_void_p),
                ("call_entry_d", C.c_void_p), ("call_exit_live", C.c_void_p),
                ("in_region", C.c_void_p), ("map_to", C.c_void_p), ("map_from", C.c_void_p),
                ("map_alloc", C.c_void_p), ("n_kernels", C.c_int32), ("kernel_to", C.c_void_p),
                ("kernel_from", C.c_void_p), ("firstprivate", C.c_void_p), ("acc_point", C.c_void_p),
                ("n_region_entries", C.c_int32), ("n_region_exits", C.c_int32),
                ("region_entry_edges", C.c_void_p), ("region_exit_edges", C.c_void_p),
                ("host_block", C.c_void_p)]


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_batch", C.c_int32), ("max_inflight", C.c_int32),
                ("device", C.c_int32), ("keep_results", C.c_int32), ("opts", Opts), ("resident", C.c_int32),
                ("workers", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("batches", C.c_int64), ("mean_batch", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("max_ms", C.c_double), ("peak_bytes", C.c_int64),
                ("bytes_in_use", C.c_int64), ("cache_hits", C.c_int64), ("cache_misses", C.c_int64),
                ("cached_plans", C.c_int64)]


class Program(C.Structure):
    _fields_ = [("n_funcs", C.c_int32), ("funcs", C.POINTER(Cfg)), ("site_off", C.c_void_p),
                ("site_callee", C.c_void_p), ("map_off", C.c_void_p), ("var_map", C.c_void_p),
                ("max_contexts", C.c_int32)]


class Instance(C.Structure):
    _fields_ = [("func", C.c_int32), ("status", C.c_int32), ("entry_h", C.c_void_p), ("entry_d", C.c_void_p),
                ("exit_live", C.c_void_p), ("result", C.POINTER(Result))]


class ProgramResult(C.Structure):
    _fields_ = [("n_instances", C.c_int32), ("inst", C.POINTER(Instance)), ("levels", C.c_int32),
                ("height", C.c_void_p), ("status", C.c_void_p), ("summaries", C.c_void_p),
                ("summary_off", C.c_void_p)]


class Timing(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int32), ("ms", C.c_double)]


EXPORTS = {
    "ompdart_plan_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "ompdart_plan_graph": (C.c_int, [C.c_void_p, C.c_int]),
    "ompdart_plan_timings": (C.c_int, [C.c_void_p, C.POINTER(Timing), C.c_int32, C.POINTER(C.c_int32)]),
    "ompdart_batch_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "ompdart_batch_timings": (C.c_int, [C.c_void_p, C.POINTER(Timing), C.c_int32, C.POINTER(C.c_int32)]),
    "ompdart_plan_create": (C.c_int, [C.POINTER(Cfg), C.POINTER(Opts), C.POINTER(C.c_void_p)]),
    "ompdart_plan_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ompdart_plan_sync": (C.c_int, [C.c_void_p]),
    "ompdart_plan_view": (C.c_int, [C.c_void_p, C.POINTER(Result)]),
    "ompdart_plan_fetch": (C.c_int, [C.c_void_p, C.POINTER(C.POINTER(Result))]),
    "ompdart_plan_launches": (C.c_int, [C.c_void_p]),
    "ompdart_plan_destroy": (None, [C.c_void_p]),
    "ompdart_analyze": (C.c_int, [C.POINTER(Cfg), C.POINTER(Opts), C.POINTER(C.POINTER(Result))]),
    "ompdart_result_free": (None, [C.POINTER(Result)]),
    "ompdart_host_cache_trim": (C.c_size_t, []),
    "ompdart_last_error": (C.c_char_p, []),
    "ompdart_batch_create": (C.c_int, [C.POINTER(Cfg), C.c_int32, C.POINTER(Opts), C.POINTER(C.c_void_p),
                                       C.c_void_p]),
    "ompdart_batch_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ompdart_batch_sync": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ompdart_batch_view": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Result)]),
    "ompdart_batch_fetch": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.POINTER(Result))]),
    "ompdart_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "ompdart_batch_destroy": (None, [C.c_void_p]),
    "ompdart_analyze_batch": (C.c_int, [C.POINTER(Cfg), C.c_int32, C.POINTER(Opts),
                                        C.POINTER(C.POINTER(Result)), C.c_void_p]),
    "ompdart_summarize_batch": (C.c_int, [C.POINTER(Cfg), C.c_int32, C.POINTER(Opts), C.c_void_p, C.c_void_p]),
    "ompdart_summarize_callee": (C.c_int, [C.POINTER(Cfg), C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(Opts)]),
    "ompdart_analyze_program": (C.c_int, [C.POINTER(Program), C.POINTER(Opts), C.POINTER(C.POINTER(ProgramResult))]),
    "ompdart_program_result_free": (None, [C.POINTER(ProgramResult)]),
    "ompdart_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(C.c_void_p)]),
    "ompdart_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Cfg), C.POINTER(C.c_int64)]),
    "ompdart_server_replay": (C.c_int, [C.c_void_p, C.POINTER(Cfg), C.c_int32, C.c_void_p, C.c_void_p]),
    "ompdart_server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.POINTER(Result)),
                                      C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "ompdart_server_drain": (C.c_int, [C.c_void_p, C.c_int32]),
    "ompdart_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "ompdart_server_destroy": (None, [C.c_void_p]),
    "ompdart_liveness_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}


def load():
    """Load libompdart.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise OSError("libompdart.so not built: run `python -m paper_2406_13881_b300.build`")
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in EXPORTS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(rc):
    if rc != OK:
        raise OmpdartError(rc, load().ompdart_last_error().decode())


MEM_HOST, MEM_DEVICE = 0, 1


class DeviceCfg:
    """A CFG whose arrays already sit in device memory (``ompdart_cfg.mem``
    = OMPDART_MEM_DEVICE): integer device addresses (``None`` for an
    omitted optional array) and the sizes.  ``owner`` keeps whatever holds
    that memory alive while the CFG is in use."""

    def __init__(self, n_blocks, n_vars, entry, succ_off, succ, acc_off, acc, entry_host_valid=None,
                 entry_dev_valid=None, exit_host_live=None, call_planes=None, n_calls=0, owner=None,
                 region=None, scalar_vars=None):
        self.n_blocks, self.n_vars, self.entry = int(n_blocks), int(n_vars), int(entry)
        self.ptrs = (succ_off, succ, acc_off, acc, entry_host_valid, entry_dev_valid, exit_host_live, call_planes)
        self.n_calls = int(n_calls)
        self.region, self.scalar_vars = region, scalar_vars
        self.owner = owner

    @property
    def W(self):
        return (self.n_vars + 63) // 64


class _Inputs:
    """Keeps the contiguous numpy copies alive while the C struct points at
    them (or, for a DeviceCfg, passes its device addresses through)."""

    def __init__(self, cfg):
        if isinstance(cfg, DeviceCfg):
            self.n, self.nv, self.W = cfg.n_blocks, cfg.n_vars, cfg.W
            self.dev = cfg
            self.c = Cfg(cfg.n_blocks, cfg.n_vars, cfg.entry, *cfg.ptrs, cfg.n_calls, MEM_DEVICE, cfg.region,
                         cfg.scalar_vars)
            return
        g = cfg if isinstance(cfg, dict) else cfg.__dict__
        self.n, self.nv = int(g["n_blocks"]), int(g["n_vars"])
        self.W = (self.nv + 63) // 64
        self.so = np.ascontiguousarray(g["succ_off"], dtype=np.int32)
        self.s = np.ascontiguousarray(g["succ"], dtype=np.int32)
        self.ao = np.ascontiguousarray(g["acc_off"], dtype=np.int32)
        self.acc = np.ascontiguousarray(g["acc"], dtype=np.uint32)

        def opt(k):
            v = g.get(k)
            return None if v is None else np.ascontiguousarray(v, dtype=np.uint64)

        self.ehv, self.edv, self.xhl = opt("entry_host_valid"), opt("entry_dev_valid"), opt("exit_host_live")
        self.calls = opt("call_planes")
        self.scal = opt("scalar_vars")
        reg = g.get("region")
        self.reg = None if reg is None else np.ascontiguousarray(reg, dtype=np.int32)
        p = lambda a: None if a is None else a.ctypes.data  # noqa: E731
        self.c = Cfg(self.n, self.nv, int(g.get("entry", 0)), p(self.so), p(self.s), p(self.ao),
                     p(self.acc), p(self.ehv), p(self.edv), p(self.xhl), p(self.calls),
                     0 if self.calls is None else int(self.calls.size // (7 * self.W)), MEM_HOST,
                     p(self.reg), p(self.scal))


def _opts(max_sweeps=0, keep_states=False, path=0, chunk_target=0, device=0, warps_per_cta=0, tune=False,
          no_graph=False, data_region=False, eager_to=False):
    return Opts(int(max_sweeps), int(bool(keep_states)), int(path), int(chunk_target), int(device),
                int(warps_per_cta), int(bool(tune)), int(bool(no_graph)), int(bool(data_region)),
                int(bool(eager_to)))


class _Owned:
    """A library-owned host result, freed (ompdart_result_free) once the
    last numpy view into its arrays is gone."""

    __slots__ = ("_free", "_ptr")

    def __init__(self, lib, ptr):
        self._free, self._ptr = lib.ompdart_result_free, ptr

    def __del__(self):
        try:
            self._free(self._ptr)
        except Exception:  # interpreter shutdown
            pass


def _owned_result(lib, ptr) -> dict:
    """Numpy views (no copy) of a host result that ``ptr`` owns."""
    return _result_to_numpy(ptr.contents, _Owned(lib, ptr))


def _result_to_numpy(r: Result, owner: "_Owned | None" = None) -> dict:
    """Arrays of a host result: views that keep ``owner`` alive when given,
    else copies (the caller frees the result)."""
    n, W = r.n_blocks, r.n_words

    def arr(ptr, count, dt, shape=None):
        if not ptr or count == 0:
            a = np.zeros(count, dtype=dt)
        else:
            buf = (C.c_char * (count * np.dtype(dt).itemsize)).from_address(ptr)
            if owner is not None:
                buf._owner = owner
                a = np.frombuffer(buf, dtype=dt)
            else:
                a = np.frombuffer(buf, dtype=dt).copy()
        return a.reshape(shape) if shape else a

    out = {
        "h_in": arr(r.h_in, n * W, np.uint64, (n, W)),
        "d_in": arr(r.d_in, n * W, np.uint64, (n, W)),
        "acc_flag": arr(r.acc_flag, r.n_acc, np.uint8),
        "edge_xfers": arr(r.edge_xfers, r.n_edge_xfers, XFER_DTYPE),
        "exit_blocks": arr(r.exit_blocks, r.n_exits, np.int32),
        "from_exit": arr(r.from_exit, r.n_exits * W, np.uint64, (r.n_exits, W)),
        "path": r.path, "sweeps": r.sweeps, "h2d_bytes": int(r.h2d_bytes), "d2h_bytes": int(r.d2h_bytes),
    }
    if r.h_out:
        out["h_out"] = arr(r.h_out, n * W, np.uint64, (n, W))
        out["d_out"] = arr(r.d_out, n * W, np.uint64, (n, W))
    if r.live_in:
        out["live_in"] = arr(r.live_in, n * W, np.uint64, (n, W))
    S = r.n_call_sites
    out["call_site_acc"] = arr(r.call_site_acc, S, np.int32)
    for k in ("call_to", "call_from", "call_entry_h", "call_entry_d", "call_exit_live"):
        out[k] = arr(getattr(r, k), S * W, np.uint64, (S, W))
    if r.in_region:  # data region and directives
        K = r.n_kernels
        out["in_region"] = arr(r.in_region, n, np.uint8)
        for k in ("map_to", "map_from", "map_alloc"):
            out[k] = arr(getattr(r, k), W, np.uint64)
        for k in ("kernel_to", "kernel_from", "firstprivate"):
            out[k] = arr(getattr(r, k), K * W, np.uint64, (K, W))
        out["acc_point"] = arr(r.acc_point, r.n_acc, np.int32)
        out["region_entry_edges"] = arr(r.region_entry_edges, r.n_region_entries, np.int32)
        out["region_exit_edges"] = arr(r.region_exit_edges, r.n_region_exits, np.int32)
    return out


def analyze(cfg, **opts) -> dict:
    """One-shot analysis through ``ompdart_analyze`` (host buffers in and out)."""
    lib = load()
    inp = _Inputs(cfg)
    o = _opts(**opts)
    res = C.POINTER(Result)()
    _check(lib.ompdart_analyze(C.byref(inp.c), C.byref(o), C.byref(res)))
    return _owned_result(lib, res)


def liveness_noalloc(n_blocks, n_vars, entry, succ_off, succ, acc_off, acc, exit_host_live, live_in,
                     stream=0):
    """``ompdart_liveness_noalloc``: every array argument is a device
    pointer (int); the call allocates nothing."""
    _check(load().ompdart_liveness_noalloc(int(n_blocks), int(n_vars), int(entry), succ_off, succ, acc_off, acc,
                                           exit_host_live, live_in, C.c_void_p(stream or 0)))


class Plan:
    """A resident analysis: ingest once (``ompdart_plan_create``), then run
    the device solver as often as wanted (``run`` enqueues, ``sync`` waits)."""

    def __init__(self, cfg, **opts):
        self._lib = load()
        self._inp = _Inputs(cfg)
        self._h = C.c_void_p()
        _check(self._lib.ompdart_plan_create(C.byref(self._inp.c), C.byref(_opts(**opts)),
                                             C.byref(self._h)))

    def run(self, stream: int | None = None):
        _check(self._lib.ompdart_plan_run(self._h, C.c_void_p(stream or 0)))

    def sync(self):
        _check(self._lib.ompdart_plan_sync(self._h))

    def graph(self, enable: bool = True):
        """Replay later runs as one captured CUDA graph."""
        _check(self._lib.ompdart_plan_graph(self._h, int(bool(enable))))

    def view(self) -> Result:
        r = Result()
        _check(self._lib.ompdart_plan_view(self._h, C.byref(r)))
        return r

    def fetch(self) -> dict:
        res = C.POINTER(Result)()
        _check(self._lib.ompdart_plan_fetch(self._h, C.byref(res)))
        return _owned_result(self._lib, res)

    def profile(self, enable: bool = True):
        _check(self._lib.ompdart_plan_profile(self._h, int(bool(enable))))

    def timings(self) -> dict:
        """{kernel name: (launches, total ms)} accumulated since profile(True)."""
        n = C.c_int32()
        _check(self._lib.ompdart_plan_timings(self._h, None, 0, C.byref(n)))
        arr = (Timing * max(1, n.value))()
        _check(self._lib.ompdart_plan_timings(self._h, arr, n.value, C.byref(n)))
        return {arr[i].name.decode(): (arr[i].launches, arr[i].ms) for i in range(n.value)}

    @property
    def launches(self) -> int:
        return int(self._lib.ompdart_plan_launches(self._h))

    def close(self):
        if self._h:
            self._lib.ompdart_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _BatchInputs:
    """The C structs of many CFGs (and the numpy arrays they point at)."""

    def __init__(self, cfgs):
        self.inp = [_Inputs(c) for c in cfgs]
        self.arr = (Cfg * max(1, len(self.inp)))()
        for i, x in enumerate(self.inp):
            self.arr[i] = x.c
        self.n = len(self.inp)


class Batch:
    """Many independent CFGs analysed per device run (``ompdart_batch_*``):
    ``status`` after construction holds each CFG's ingestion code, ``run``
    enqueues one run of every CFG (a replayed CUDA graph unless
    ``no_graph``), ``sync`` waits and returns the per-CFG status array."""

    def __init__(self, cfgs, **opts):
        self._lib = load()
        self._inp = _BatchInputs(cfgs)
        self._h = C.c_void_p()
        self.status = np.zeros(max(1, self._inp.n), dtype=np.int32)[: self._inp.n]
        _check(self._lib.ompdart_batch_create(self._inp.arr, self._inp.n, C.byref(_opts(**opts)),
                                              C.byref(self._h), self.status.ctypes.data))

    def __len__(self):
        return self._inp.n

    def run(self, stream: int | None = None):
        _check(self._lib.ompdart_batch_run(self._h, C.c_void_p(stream or 0)))

    def sync(self) -> np.ndarray:
        st = np.zeros(max(1, self._inp.n), dtype=np.int32)
        _check(self._lib.ompdart_batch_sync(self._h, st.ctypes.data))
        self.status = st[: self._inp.n]
        return self.status

    def view(self, i: int) -> Result:
        r = Result()
        _check(self._lib.ompdart_batch_view(self._h, int(i), C.byref(r)))
        return r

    def fetch(self, i: int) -> dict:
        res = C.POINTER(Result)()
        _check(self._lib.ompdart_batch_fetch(self._h, int(i), C.byref(res)))
        return _owned_result(self._lib, res)

    def profile(self, enable: bool = True):
        """Per-kernel CUDA events on every later run (plans one after
        another on the run's stream, no graph)."""
        _check(self._lib.ompdart_batch_profile(self._h, int(bool(enable))))

    def timings(self) -> dict:
        """{kernel name: (launches, total ms)} summed over the arenas since profile(True)."""
        n = C.c_int32()
        _check(self._lib.ompdart_batch_timings(self._h, None, 0, C.byref(n)))
        arr = (Timing * max(1, n.value))()
        _check(self._lib.ompdart_batch_timings(self._h, arr, n.value, C.byref(n)))
        return {arr[i].name.decode(): (arr[i].launches, arr[i].ms) for i in range(n.value)}

    def info(self) -> dict:
        na, ns, nl = C.c_int32(), C.c_int32(), C.c_int32()
        _check(self._lib.ompdart_batch_info(self._h, C.byref(na), C.byref(ns), C.byref(nl), 0, None, None, None,
                                            None))
        k = max(1, na.value)
        w, n, ch, wp = (np.zeros(k, np.int32) for _ in range(4))
        _check(self._lib.ompdart_batch_info(self._h, C.byref(na), C.byref(ns), C.byref(nl), k, w.ctypes.data,
                                            n.ctypes.data, ch.ctypes.data, wp.ctypes.data))
        arenas = [dict(W=int(w[i]), cfgs=int(n[i]), chunk_target=int(ch[i]), warps_per_cta=int(wp[i]))
                  for i in range(na.value)]
        return {"arenas": arenas, "solo": ns.value, "launches": nl.value}

    def close(self):
        if self._h:
            self._lib.ompdart_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def analyze_batch(cfgs, **opts):
    """``ompdart_analyze_batch``: host buffers in and out.  Returns
    (results, status): results[i] is a dict as from ``analyze`` or None
    where status[i] is an error code."""
    lib = load()
    inp = _BatchInputs(cfgs)
    outs = (C.POINTER(Result) * max(1, inp.n))()
    st = np.zeros(max(1, inp.n), dtype=np.int32)
    _check(lib.ompdart_analyze_batch(inp.arr, inp.n, C.byref(_opts(**opts)), outs, st.ctypes.data))
    owners = [_Owned(lib, outs[i]) if outs[i] else None for i in range(inp.n)]
    res = [_result_to_numpy(o._ptr.contents, o) if o is not None else None for o in owners]
    return res, st[: inp.n]


class Server:
    """The serving loop (``ompdart_server_*``): ``submit`` queues a CFG and
    returns its ticket, ``wait`` returns (status, latency ms, result dict or
    None), ``replay`` submits many CFGs at given arrival times."""

    def __init__(self, hbm_budget_bytes=0, max_batch=0, max_inflight=0, device=0, keep_results=True, resident=False,
                 workers=0, **opts):
        self._lib = load()
        so = ServerOpts(int(hbm_budget_bytes), int(max_batch), int(max_inflight), int(device),
                        int(bool(keep_results)), _opts(device=device, **opts), int(bool(resident)), int(workers))
        self._h = C.c_void_p()
        self._keep = []
        _check(self._lib.ompdart_server_create(C.byref(so), C.byref(self._h)))

    def submit(self, cfg) -> int:
        inp = _Inputs(cfg)
        t = C.c_int64()
        _check(self._lib.ompdart_server_submit(self._h, C.byref(inp.c), C.byref(t)))
        return t.value

    def replay(self, cfgs, arrival_us) -> np.ndarray:
        """Submit cfgs[i] at arrival_us[i] microseconds from now (native
        timing loop; releases the GIL)."""
        bi = _BatchInputs(cfgs)
        arr = np.ascontiguousarray(arrival_us, dtype=np.float64)
        tickets = np.zeros(max(1, bi.n), dtype=np.int64)
        _check(self._lib.ompdart_server_replay(self._h, bi.arr, bi.n, arr.ctypes.data, tickets.ctypes.data))
        return tickets[: bi.n]

    def wait(self, ticket, timeout_ms=-1, want_result=True):
        res = C.POINTER(Result)()
        st, lat = C.c_int32(), C.c_double()
        _check(self._lib.ompdart_server_wait(self._h, int(ticket), int(timeout_ms),
                                             C.byref(res) if want_result else None, C.byref(st), C.byref(lat)))
        out = None
        if want_result and res:
            out = _owned_result(self._lib, res)
        return st.value, lat.value, out

    def drain(self, timeout_ms=-1):
        _check(self._lib.ompdart_server_drain(self._h, int(timeout_ms)))

    def stats(self) -> dict:
        s = ServerStats()
        _check(self._lib.ompdart_server_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            self._lib.ompdart_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def summarize_batch(cfgs, **opts):
    """``ompdart_summarize_batch``: ([7, W_i] summary or None, status) per callee."""
    lib = load()
    bi = _BatchInputs(cfgs)
    outs = [np.zeros((7, x.W), dtype=np.uint64) for x in bi.inp]
    ptrs = (C.c_void_p * max(1, bi.n))(*[o.ctypes.data for o in outs])
    st = np.zeros(max(1, bi.n), dtype=np.int32)
    _check(lib.ompdart_summarize_batch(bi.arr, bi.n, C.byref(_opts(**opts)), ptrs, st.ctypes.data))
    return [o if s == 0 else None for o, s in zip(outs, st[: bi.n])], st[: bi.n]


def summarize_callee(cfg, var_map, caller_n_vars, **opts) -> np.ndarray:
    """``ompdart_summarize_callee``: the callee's summary as a [7, W_caller]
    call-table row of the caller (var_map: caller variable per callee
    variable, -1 to drop; None = identity)."""
    lib = load()
    inp = _Inputs(cfg)
    row = np.zeros((7, (int(caller_n_vars) + 63) // 64), dtype=np.uint64)
    vm = None if var_map is None else np.ascontiguousarray(var_map, dtype=np.int32)
    _check(lib.ompdart_summarize_callee(C.byref(inp.c), None if vm is None else vm.ctypes.data, int(caller_n_vars),
                                        row.ctypes.data, C.byref(_opts(**opts))))
    return row


def _u64(ptr, n):
    if not ptr or n == 0:
        return np.zeros(n, dtype=np.uint64)
    return np.frombuffer((C.c_char * (8 * n)).from_address(ptr), dtype=np.uint64).copy()


def analyze_program(funcs, site_off, site_callee, var_maps, max_contexts=0, **opts) -> dict:
    """``ompdart_analyze_program``: funcs are CFGs whose call accesses name
    their k-th call site (site_off[f] + k); var_maps[s] maps site s's callee
    variables to caller variables (-1 for a local).  Returns
    {"instances": [(func, (entry_h, entry_d, exit_live), status, result)],
     "summaries": [[7, W_f] per function], "height": [...], "levels": n}."""
    lib = load()
    bi = _BatchInputs(funcs)
    so = np.ascontiguousarray(site_off, dtype=np.int32)
    sc = np.ascontiguousarray(site_callee, dtype=np.int32)
    mo = np.zeros(len(var_maps) + 1, dtype=np.int32)
    mo[1:] = np.cumsum([len(m) for m in var_maps])
    vm = np.ascontiguousarray(np.concatenate([np.asarray(m, dtype=np.int32) for m in var_maps])
                              if var_maps else np.zeros(0, np.int32))
    prog = Program(bi.n, C.cast(bi.arr, C.POINTER(Cfg)), so.ctypes.data, sc.ctypes.data, mo.ctypes.data,
                   vm.ctypes.data, int(max_contexts))
    res = C.POINTER(ProgramResult)()
    _check(lib.ompdart_analyze_program(C.byref(prog), C.byref(_opts(**opts)), C.byref(res)))
    try:
        r = res.contents
        F = bi.n
        height = np.frombuffer((C.c_char * (4 * max(F, 1))).from_address(r.height), dtype=np.int32)[:F].copy()
        soff = np.frombuffer((C.c_char * (8 * max(F, 1))).from_address(r.summary_off), dtype=np.int64)[:F].copy()
        sums = [_u64(r.summaries + 8 * int(soff[f]), 7 * bi.inp[f].W).reshape(7, -1) if r.summaries else None
                for f in range(F)]
        inst = []
        for i in range(r.n_instances):
            x = r.inst[i]
            W = bi.inp[x.func].W
            ctx = (_u64(x.entry_h, W), _u64(x.entry_d, W), _u64(x.exit_live, W))
            inst.append((x.func, ctx, x.status, _result_to_numpy(x.result.contents) if x.result else None))
        return {"instances": inst, "summaries": sums, "height": height, "levels": r.levels}
    finally:
        lib.ompdart_program_result_free(res)
