"""Reference interprocedural driver on the CPU oracle (test infrastructure).

Follows the steps the library documents for ompdart_analyze_program, in
plain Python over ``oracle.summarize`` / ``oracle.solve`` (both pinned in
test_oracle_calls.py), sharing no code with the library:
  * summaries bottom-up (a function after all its callees), each call
    site's row = the callee's summary mapped into the caller's numbering
    (Req, Kill, MustDef by OR over callee variables denoting the same caller
    variable, Gen by AND, a kill overriding a gen);
  * contexts top-down: a function nobody calls runs in its own boundary
    rows; otherwise once per distinct context its sites pass on: the
    caller's call_entry_h / call_entry_d / call_exit_live at the call mapped
    into the callee's numbering (a callee local starts host-valid only, dead
    after the exit); per site the distinct contexts sorted, at most
    max_contexts kept, the excess merged into the last (validity AND,
    liveness OR).
"""
from functools import lru_cache

import numpy as np

import oracle


def _bit(row, v):
    return (int(row[v >> 6]) >> (v & 63)) & 1


def _set(row, v):
    row[v >> 6] |= np.uint64(1) << np.uint64(v & 63)


def map_summary(summ, callee_vars, var_map, caller_vars):
    Wr = (caller_vars + 63) // 64
    row = np.zeros((7, Wr), dtype=np.uint64)
    gen = {2: {}, 4: {}}
    for v in range(callee_vars):
        t = int(var_map[v])
        if t < 0 or t >= caller_vars:
            continue
        for k in range(7):
            x = _bit(summ[k], v)
            if k in gen:
                gen[k][t] = gen[k].get(t, 1) & x
            elif x:
                _set(row[k], t)
    for k in gen:
        for t, x in gen[k].items():
            if x:
                _set(row[k], t)
    row[2] &= ~row[3]
    row[4] &= ~row[5]
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


def with_table(g, table, ctx=None):
    h = type(g)(g.n_blocks, g.n_vars, g.entry, g.succ_off, g.succ, g.acc_off, g.acc)
    h.call_planes = table if table is not None and len(table) else None
    if ctx is not None:
        h.entry_host_valid, h.entry_dev_valid, h.exit_host_live = ctx
    else:
        h.entry_host_valid, h.entry_dev_valid, h.exit_host_live = g.entry_host_valid, g.entry_dev_valid, \
            g.exit_host_live
    return h


def reference_program(prog, max_contexts=4):
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
        summary[f] = oracle.summarize(with_table(g, table[f]))
    callers = np.zeros(F, dtype=bool)
    callers[sc] = True
    ctxs = {f: {} for f in range(F)}
    for f in range(F):
        if not callers[f]:
            g = funcs[f]
            W = g.W
            top = np.full(W, ~np.uint64(0), dtype=np.uint64)
            if g.n_vars % 64:
                top[-1] = np.uint64((1 << (g.n_vars % 64)) - 1)
            eh = (g.entry_host_valid if g.entry_host_valid is not None else top) & top
            ed = (g.entry_dev_valid if g.entry_dev_valid is not None else np.zeros(W, np.uint64)) & top
            xl = (g.exit_host_live if g.exit_host_live is not None else top) & top
            c = (np.asarray(eh, np.uint64), np.asarray(ed, np.uint64), np.asarray(xl, np.uint64))
            ctxs[f][ctx_key(c)] = c
    results = {}
    for h in sorted(set(H), reverse=True):
        per_site = {}
        for f in [x for x in range(F) if H[x] == h]:
            g = funcs[f]
            calls = np.flatnonzero(np.asarray(g.acc, np.uint32) >> np.uint32(31))
            for key, c in ctxs[f].items():
                r = oracle.solve(with_table(g, table[f], c))
                results[(f, key)] = (with_table(g, table[f], c), r)
                for j, a in enumerate(calls):
                    s = int(so[f]) + int(g.acc[a] & 0x7FFFFFFF)
                    callee = int(sc[s])
                    cc = map_context(r["call_entry_h"][j], r["call_entry_d"][j], r["call_exit_live"][j], vms[s],
                                     funcs[callee].n_vars)
                    per_site.setdefault(s, {})[ctx_key(cc)] = cc
        for s, d in per_site.items():
            keys = sorted(d)
            if len(keys) > max_contexts:
                m = [r.copy() for r in d[keys[max_contexts - 1]]]
                for k in keys[max_contexts:]:
                    m[0] &= d[k][0]
                    m[1] &= d[k][1]
                    m[2] |= d[k][2]
                keep = [d[k] for k in keys[: max_contexts - 1]] + [tuple(m)]
            else:
                keep = [d[k] for k in keys]
            callee = int(sc[s])
            for c in keep:
                ctxs[callee][ctx_key(c)] = c
    return summary, results, H
