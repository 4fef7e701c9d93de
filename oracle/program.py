"""Interprocedural oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product library never does.  It is plain Python
over ``oracle.summarize`` / ``oracle.solve`` (both pinned in
``tests/test_oracle_calls.py``) and shares no code with the library.

Sec. IV-C of the paper: a function's side effects on globals and on the
data its pointer parameters denote are recorded once per function and
applied at every call site.  This module states how a summary in the
callee's numbering becomes a call-table row of a caller, how the contexts a
callee is analysed in are formed, and the whole-program driver:

* ``map_summary``: callee variable v denotes caller variable var_map[v]
  (a global, or the actual argument of a pointer parameter) or nothing
  (-1: a callee local, dropped).  Several callee variables may denote one
  caller variable (the same array passed twice, a global also passed as a
  parameter).  Their rows combine into the tightest row that is sound for
  every callee whose per-variable summaries are the given ones: a caller
  variable is required (Req) or killed (Kill) or must-written (MustDef) if
  one of its aliases is, and generated (Gen) if one of its aliases is and
  none kills it.  (``tests/test_oracle_program.py`` derives exactly this
  bound by brute force over all interleavings of alias event sequences.)
* ``map_context``: the caller's state right before the call (validity
  after the requirement transfers, liveness right after the call) in the
  callee's numbering; a callee local starts valid on the host only and is
  dead after the exit.
* ``merge_contexts``: a call site passes on at most ``max_contexts``
  distinct contexts.  Sorted, the first max_contexts - 1 are kept and the
  rest are merged into the last one by the meet (validity AND, liveness
  OR), which is below every context it absorbs, so the merged instance's
  transfers serve each of them.  A context whose meet with the merged one
  would leave a variable valid nowhere that one of them holds somewhere is
  not merged (no single placement serves a host-only and a device-only
  copy) and stays a context of its own.
* ``reference_program``: summaries bottom-up (a function after all its
  callees), then contexts top-down (a function nobody calls runs in its own
  boundary rows; a called function runs once per distinct context its call
  sites pass on).
"""
from functools import lru_cache

import numpy as np

from . import solve, summarize

REQ_H, REQ_D, GEN_H, KILL_H, GEN_D, KILL_D, MUST_DEF = range(7)


def _bit(row, v):
    return (int(row[v >> 6]) >> (v & 63)) & 1


def _set(row, v):
    row[v >> 6] |= np.uint64(1) << np.uint64(v & 63)


def map_summary(summ, callee_vars, var_map, caller_vars):
    """[7, W_caller] call-table row from a [7, W_callee] summary."""
    Wr = (caller_vars + 63) // 64
    row = np.zeros((7, Wr), dtype=np.uint64)
    for v in range(callee_vars):
        t = int(var_map[v])
        if t < 0 or t >= caller_vars:
            continue  # a callee local: no effect on the caller
        for k in range(7):
            if _bit(summ[k], v):
                _set(row[k], t)
    # an alias that may leave the copy stale wins over one that makes it valid
    row[GEN_H] &= ~row[KILL_H]
    row[GEN_D] &= ~row[KILL_D]
    return row


def map_context(eh, ed, xl, var_map, callee_vars):
    W = (callee_vars + 63) // 64
    out = [np.zeros(W, dtype=np.uint64) for _ in range(3)]
    for v in range(callee_vars):
        t = int(var_map[v])
        if t < 0:
            _set(out[0], v)
            continue
        for r, src in zip(out, (eh, ed, xl)):
            if _bit(src, t):
                _set(r, v)
    return tuple(out)


def ctx_key(c):
    return tuple(tuple(int(x) for x in r) for r in c)


def merge_groups(contexts, max_contexts):
    """The contexts a call site passes on, each with the distinct contexts
    it stands for: [(context, [absorbed contexts])] (see the module
    docstring)."""
    d = {ctx_key(c): c for c in contexts}
    keys = sorted(d)
    if len(keys) <= max_contexts:
        return [(d[k], [d[k]]) for k in keys]
    out = [(d[k], [d[k]]) for k in keys[: max_contexts - 1]]
    m = [np.array(r, dtype=np.uint64, copy=True) for r in d[keys[max_contexts - 1]]]
    absorbed = [d[keys[max_contexts - 1]]]
    alone = []
    for k in keys[max_contexts:]:
        c = d[k]
        eh, ed, xl = m[0] & c[0], m[1] & c[1], m[2] | c[2]
        held = m[0] | m[1] | c[0] | c[1]
        if (held & ~(eh | ed)).any():
            alone.append((c, [c]))
            continue
        m = [eh, ed, xl]
        absorbed.append(c)
    return out + [(tuple(m), absorbed)] + alone


def merge_contexts(contexts, max_contexts):
    return [m for m, _ in merge_groups(contexts, max_contexts)]


def with_table(g, table, ctx=None):
    h = type(g)(g.n_blocks, g.n_vars, g.entry, g.succ_off, g.succ, g.acc_off, g.acc)
    h.call_planes = table if table is not None and len(table) else None
    if ctx is not None:
        h.entry_host_valid, h.entry_dev_valid, h.exit_host_live = ctx
    else:
        h.entry_host_valid, h.entry_dev_valid, h.exit_host_live = g.entry_host_valid, g.entry_dev_valid, \
            g.exit_host_live
    return h


def root_context(g):
    """A function nobody calls: its own boundary rows (defaults: every
    variable valid on the host, nothing on the device, all live at exit)."""
    W = g.W
    top = np.full(W, ~np.uint64(0), dtype=np.uint64)
    if g.n_vars % 64:
        top[-1] = np.uint64((1 << (g.n_vars % 64)) - 1)
    eh = (g.entry_host_valid if g.entry_host_valid is not None else top) & top
    ed = (g.entry_dev_valid if g.entry_dev_valid is not None else np.zeros(W, np.uint64)) & top
    xl = (g.exit_host_live if g.exit_host_live is not None else top) & top
    return (np.asarray(eh, np.uint64), np.asarray(ed, np.uint64), np.asarray(xl, np.uint64))


def reference_program(prog, max_contexts=4):
    """(summaries, {(f, ctx_key): (cfg, oracle result)}, heights)."""
    funcs, so, sc, vms = prog.funcs, prog.site_off, prog.site_callee, prog.var_maps
    F = len(funcs)

    @lru_cache(maxsize=None)
    def height(f):
        return max([height(int(sc[s])) + 1 for s in range(so[f], so[f + 1])], default=0)

    H = [height(f) for f in range(F)]
    summary, table = [None] * F, [None] * F
    for f in sorted(range(F), key=lambda x: H[x]):
        g = funcs[f]
        rows = [map_summary(summary[int(sc[s])], funcs[int(sc[s])].n_vars, vms[s], g.n_vars)
                for s in range(so[f], so[f + 1])]
        table[f] = np.stack(rows) if rows else None
        summary[f] = summarize(with_table(g, table[f]))
    callers = np.zeros(F, dtype=bool)
    callers[sc] = True
    ctxs = {f: {} for f in range(F)}
    for f in range(F):
        if not callers[f]:
            c = root_context(funcs[f])
            ctxs[f][ctx_key(c)] = c
    results = {}
    for h in sorted(set(H), reverse=True):
        per_site = {}
        for f in [x for x in range(F) if H[x] == h]:
            g = funcs[f]
            calls = np.flatnonzero(np.asarray(g.acc, np.uint32) >> np.uint32(31))
            for key, c in ctxs[f].items():
                r = solve(with_table(g, table[f], c))
                results[(f, key)] = (with_table(g, table[f], c), r)
                for j, a in enumerate(calls):
                    s = int(so[f]) + int(g.acc[a] & 0x7FFFFFFF)
                    callee = int(sc[s])
                    cc = map_context(r["call_entry_h"][j], r["call_entry_d"][j], r["call_exit_live"][j], vms[s],
                                     funcs[callee].n_vars)
                    per_site.setdefault(s, []).append(cc)
        for s, lst in per_site.items():
            callee = int(sc[s])
            for c in merge_contexts(lst, max_contexts):
                ctxs[callee][ctx_key(c)] = c
    return summary, results, H
