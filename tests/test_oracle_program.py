"""Pins of the interprocedural oracle (``oracle/program.py``, Sec. IV-C:
callee side effects applied at call sites), each against something other
than the module's own formulas:

* alias combination: the mapped row of callee variables that denote one
  caller variable is the tightest row sound for every callee with the given
  per-variable summaries -- derived here by brute force over all event
  sequences (up to 3 events per variable) and all their interleavings;
* renaming: with an injective map the mapped row is the summary of the
  callee whose variables are renamed into the caller's numbering (locals'
  accesses dropped), computed by ``oracle.summarize`` (itself pinned by path
  enumeration); with aliases the mapped row is a sound bound of that exact
  summary (requirements and kills over, gens and must-writes under);
* the call scheme end to end: the caller analysed with the mapped row, the
  callee analysed in the context the call passes on, and the callee's body
  written in place of the call (renamed, its locals fresh variables) --
  replaying every path with all those transfers reads no stale value and
  copies no stale value (path simulation);
* context merging: a merged context lies below every context it absorbed
  (validity under, liveness over) and leaves no variable valid nowhere that
  an absorbed context holds; the callee instance analysed in the merged
  context serves every absorbed context (path simulation from each);
* planted mistakes in copies of these functions each fail one of the above.
"""
import itertools

import numpy as np
import pytest

import oracle
import refsim as rs
from oracle import program as P
from paper_2406_13881_b300 import workload as wl

H, D = 0, 1
KR, KW, KRW = 1, 2, 3
ALPHABET = [("r", H), ("r", D), ("w", H), ("w", D)]


# --------------------------------------------------------------------------
# per-variable event semantics (Sec. IV-D local rule), by simulation
# --------------------------------------------------------------------------

def simulate(evs, start):
    """[valid on host, valid on device] after the events from a state where
    both copies are `start` (a read makes its space valid: the transfer it
    needs; a write makes its space valid and the other stale)."""
    val = [start, start]
    for t, s in evs:
        val[s] = 1
        if t == "w":
            val[1 - s] = 0
    return val


def first_is_read(evs, S):
    for t, s in evs:
        if t == "r" and s == S:
            return 1
        if t == "w":
            return 0
    return 0


def exact_row(evs):
    """(ReqH, ReqD, GenH, KillH, GenD, KillD, MustDef) of one straight-line
    event sequence."""
    st, sv = simulate(evs, 0), simulate(evs, 1)
    return (first_is_read(evs, H), first_is_read(evs, D), st[H], 1 - sv[H], st[D], 1 - sv[D],
            int(any(t == "w" for t, _ in evs)))


def interleavings(a, b):
    if not a or not b:
        yield list(a) + list(b)
        return
    for r in interleavings(a[1:], b):
        yield [a[0]] + r
    for r in interleavings(a, b[1:]):
        yield [b[0]] + r


def _row_of(bits7):
    return np.array([[np.uint64(x)] for x in bits7], dtype=np.uint64)


def _classes(max_len=3):
    by = {}
    for n in range(max_len + 1):
        for seq in itertools.product(ALPHABET, repeat=n):
            by.setdefault(exact_row(list(seq)), []).append(list(seq))
    return by


def tightest_pair_bounds():
    """For every pair of per-variable summaries (s1, s2): the most precise
    row that is still sound for every pair of event sequences with those
    summaries and every interleaving of them (Req, Kill: any case;
    Gen, MustDef: every case)."""
    by = _classes()
    out = {}
    for s1, s2 in itertools.product(by, repeat=2):
        acc = [0, 0, 1, 0, 1, 0, 1]
        for a in by[s1]:
            for b in by[s2]:
                for it in interleavings(a, b):
                    x = exact_row(it)
                    for k in (0, 1, 3, 5):
                        acc[k] |= x[k]
                    for k in (2, 4, 6):
                        acc[k] &= x[k]
        out[s1, s2] = tuple(acc)
    return out


_TIGHT = None


def _tight():
    global _TIGHT
    if _TIGHT is None:
        _TIGHT = tightest_pair_bounds()
    return _TIGHT


def alias_pair_rows(map_summary):
    """{(s1, s2): row} of a map_summary for two callee variables (summaries
    s1, s2) that denote caller variable 0."""
    out = {}
    for s1, s2 in _tight():
        summ = np.array([[np.uint64(s1[k] | (s2[k] << 1))] for k in range(7)], dtype=np.uint64)
        row = map_summary(summ, 2, np.array([0, 0], np.int32), 1)
        out[s1, s2] = tuple(int(row[k][0]) & 1 for k in range(7))
    return out


def test_alias_rule_is_the_tightest_sound_one():
    got = alias_pair_rows(P.map_summary)
    tight = _tight()
    assert len(tight) == 225
    for key, want in tight.items():
        assert got[key] == want, (key, got[key], want)


def test_alias_rule_three_aliases_sound_and_tight():
    """Three aliases: the mapped row equals the bound over every triple of
    sequences (up to 2 events each) and every interleaving."""
    by = _classes(2)
    keys = list(by)
    rng = np.random.default_rng(1)
    for _ in range(60):
        ss = [keys[int(i)] for i in rng.integers(0, len(keys), 3)]
        acc = [0, 0, 1, 0, 1, 0, 1]
        for a in by[ss[0]]:
            for b in by[ss[1]]:
                for c in by[ss[2]]:
                    for ab in interleavings(a, b):
                        for it in interleavings(ab, c):
                            x = exact_row(it)
                            for k in (0, 1, 3, 5):
                                acc[k] |= x[k]
                            for k in (2, 4, 6):
                                acc[k] &= x[k]
        summ = np.array([[np.uint64(ss[0][k] | (ss[1][k] << 1) | (ss[2][k] << 2))] for k in range(7)],
                        dtype=np.uint64)
        row = P.map_summary(summ, 3, np.array([0, 0, 0], np.int32), 1)
        assert tuple(int(row[k][0]) & 1 for k in range(7)) == tuple(acc), ss


# --------------------------------------------------------------------------
# renaming against the summary of the renamed callee
# --------------------------------------------------------------------------

def random_callee(rng, nv):
    """A small callee: random graph (possibly cyclic, some blocks without
    successors), 0-4 accesses per block."""
    return wl.random_graph(None, int(rng.integers(1, 7)), nv, max_out=2, acc_max=4, rng=rng)


def renamed(g, var_map, caller_vars):
    """The callee with every access of variable v turned into one of
    var_map[v] (accesses of locals, var_map[v] < 0, dropped)."""
    var, kind, space = wl.unpack_access(g.acc)
    keep = np.array([var_map[v] >= 0 for v in var], dtype=bool)
    blk = np.repeat(np.arange(g.n_blocks), np.diff(g.acc_off))
    ao = np.zeros(g.n_blocks + 1, dtype=np.int32)
    ao[1:] = np.cumsum(np.bincount(blk[keep], minlength=g.n_blocks))
    acc = wl.pack_access(np.asarray(var_map, np.int64)[var[keep]], kind[keep], space[keep]) if keep.any() \
        else np.zeros(0, np.uint32)
    return wl.CFG(g.n_blocks, caller_vars, g.entry, g.succ_off, g.succ, ao, acc)


@pytest.mark.parametrize("seed", range(30))
def test_injective_map_equals_renamed_callee(seed):
    rng = np.random.default_rng(500 + seed)
    cv = int(rng.choice([3, 7, 70]))
    caller_vars = int(cv + rng.integers(0, 80))
    g = random_callee(rng, cv)
    targets = rng.permutation(caller_vars)[:cv]
    vm = np.where(rng.random(cv) < 0.25, -1, targets).astype(np.int32)  # some locals
    got = P.map_summary(oracle.summarize(g), cv, vm, caller_vars)
    np.testing.assert_array_equal(got, oracle.summarize(renamed(g, vm, caller_vars)))


def _sound(row, exact):
    """Requirements, kills over; gens, must-writes under; gen and kill never
    both (a copy valid at every exit is stale at none)."""
    r = [row[k] for k in range(7)]
    e = [exact[k] for k in range(7)]
    for k in (P.REQ_H, P.REQ_D, P.KILL_H, P.KILL_D):
        if (e[k] & ~r[k]).any():
            return False
    for k in (P.GEN_H, P.GEN_D, P.MUST_DEF):
        if (r[k] & ~e[k]).any():
            return False
    return not ((r[P.GEN_H] & r[P.KILL_H]).any() or (r[P.GEN_D] & r[P.KILL_D]).any())


@pytest.mark.parametrize("seed", range(40))
def test_aliased_map_is_a_sound_bound_of_the_renamed_callee(seed):
    rng = np.random.default_rng(600 + seed)
    cv = int(rng.choice([3, 6, 9]))
    caller_vars = int(rng.integers(1, 4))
    g = random_callee(rng, cv)
    vm = rng.integers(-1, caller_vars, size=cv).astype(np.int32)  # aliases and locals
    row = P.map_summary(oracle.summarize(g), cv, vm, caller_vars)
    assert _sound(row, oracle.summarize(renamed(g, vm, caller_vars)))


# --------------------------------------------------------------------------
# the call scheme end to end, by path simulation
# --------------------------------------------------------------------------

def _body(rng, cv):
    return [(int(rng.integers(0, cv)), int(rng.integers(1, 4)), int(rng.integers(0, 2)))
            for _ in range(int(rng.integers(1, 7)))]


def compose(caller, b, pos, row_planes, body, vm, caller_vars, r_caller, r_callee):
    """The caller with block b cut at access `pos' into [before] -> [the
    callee's body, renamed, its locals fresh variables] -> [after], and the
    transfers of both analyses placed on it.  Every call declares its
    locals anew: the body starts with a host write of each (the value a
    local starts with lives on the host).  Returns (cfg, transfers)."""
    n = caller.n_blocks
    locals_ = {v: caller_vars + i for i, v in enumerate(sorted({v for v in range(len(vm)) if vm[v] < 0}))}
    name = lambda v: int(vm[v]) if vm[v] >= 0 else locals_[v]  # noqa: E731
    nv = caller_vars + len(locals_)
    ao, acc = caller.acc_off, caller.acc
    succs = [list(caller.succ[caller.succ_off[i]:caller.succ_off[i + 1]]) for i in range(n)]
    blocks = [list(acc[ao[i]:ao[i + 1]]) for i in range(n)]
    c, d = n, n + 1
    decl = [np.uint32(wl.pack_access([x], [KW], [H])[0]) for x in sorted(locals_.values())]
    inl = decl + [np.uint32(wl.pack_access([name(v)], [k], [s])[0]) for v, k, s in body]
    succ2 = [s[:] for s in succs] + [[d], succs[b][:]]
    succ2[b] = [c]
    blocks2 = [x[:] for x in blocks] + [inl, blocks[b][pos - ao[b] + 1:]]
    blocks2[b] = blocks[b][: pos - ao[b]]
    so = np.zeros(n + 3, dtype=np.int32)
    so[1:] = np.cumsum([len(s) for s in succ2])
    ao2 = np.zeros(n + 3, dtype=np.int32)
    ao2[1:] = np.cumsum([len(x) for x in blocks2])
    g = wl.CFG(n + 2, nv, caller.entry, so, np.array([t for s in succ2 for t in s], dtype=np.int32), ao2,
               np.array([w for x in blocks2 for w in x], dtype=np.uint32))
    t = {"to_edge": {}, "from_edge": {}, "flag": {}, "from_exit": {}}
    # the caller's transfers, moved to the composed CFG's edge and access ids
    new_edge = {}
    for i in range(n):
        src = d if i == b else i
        for k, e in enumerate(range(caller.succ_off[i], caller.succ_off[i + 1])):
            new_edge[e] = int(so[src]) + k
    for e in range(caller.n_edges):
        for key in ("to_edge", "from_edge"):
            x = rs.word(r_caller[key][e, 0])
            if x:
                t[key][new_edge[e]] = x
    for i in range(n):
        for j in range(int(ao[i]), int(ao[i + 1])):
            f = int(r_caller["acc_flag"][j])
            if not f or j == pos:
                continue
            if i == b and j > pos:
                t["flag"][int(ao2[d]) + j - pos - 1] = f
            elif i == b:
                t["flag"][int(ao2[b]) + j - int(ao[b])] = f
            else:
                t["flag"][int(ao2[i]) + j - int(ao[i])] = f
        x = rs.word(r_caller["from_exit"][i, 0])
        if x:
            t["from_exit"][d if i == b else i] = x
    # the call's requirement transfers, on the edge into the body
    e_in, e_out = int(so[b]), int(so[c])
    if rs.word(r_caller["call_to"][0, 0]):
        t["to_edge"][e_in] = rs.word(r_caller["call_to"][0, 0])
    if rs.word(r_caller["call_from"][0, 0]):
        t["from_edge"][e_in] = rs.word(r_caller["call_from"][0, 0])
    # the callee instance's own transfers: its access flags, and its exit
    # `from' on the edge out of the body
    for j in range(len(body)):
        f = int(r_callee["acc_flag"][j])
        if f:
            t["flag"][int(ao2[c]) + len(decl) + j] = f
    fx = 0
    for v in range(len(vm)):
        if (int(r_callee["from_exit"][0, v >> 6]) >> (v & 63)) & 1:
            fx |= 1 << name(v)
    if fx:
        t["from_edge"][e_out] = fx
    return g, t


def _end_to_end(seed, map_summary=P.map_summary, map_context=P.map_context):
    rng = np.random.default_rng(seed)
    caller_vars = int(rng.integers(1, 6))
    cv = int(rng.integers(1, 6))
    caller = wl.random_graph(None, int(rng.integers(1, 6)), caller_vars, max_out=2, acc_max=3, rng=rng)
    body = _body(rng, cv)
    targets = rng.permutation(caller_vars + cv)[:cv]
    vm = np.where(targets < caller_vars, targets, -1).astype(np.int32)  # injective, some locals
    callee = wl.from_lists([[]], [body], cv)
    row = map_summary(oracle.summarize(callee), cv, vm, caller_vars)
    b = int(rng.integers(0, caller.n_blocks))
    ao, acc = caller.acc_off, caller.acc
    pos = int(rng.integers(ao[b], ao[b + 1] + 1))
    call_acc = np.concatenate([acc[:pos], [np.uint32(0x80000000)], acc[pos:]]).astype(np.uint32)
    call_ao = ao.copy()
    call_ao[b + 1:] += 1
    gc = wl.CFG(caller.n_blocks, caller_vars, caller.entry, caller.succ_off, caller.succ, call_ao, call_acc)
    gc.call_planes = row.reshape(1, 7, -1)
    rc = oracle.solve(gc)
    if not rc["reachable"][b]:
        return None
    ctx = map_context(rc["call_entry_h"][0], rc["call_entry_d"][0], rc["call_exit_live"][0], vm, cv)
    callee.entry_host_valid, callee.entry_dev_valid, callee.exit_host_live = ctx
    ri = oracle.solve(callee)
    g, t = compose(gc, b, pos, row, body, vm, caller_vars, rc, ri)
    top = (1 << caller_vars) - 1
    sim = rs.PathSim(g, t, (1 << g.n_vars) - 1, 0, top)
    for blocks, edges in rs.maximal_walks(g, g.entry, 2):
        sim.run(blocks, edges)
    return True


@pytest.mark.parametrize("seed", range(60))
def test_call_scheme_end_to_end_by_path_simulation(seed):
    _end_to_end(4000 + seed)


# --------------------------------------------------------------------------
# context merging
# --------------------------------------------------------------------------

def _contexts(rng, nv, k):
    """k contexts of one callee: per variable a base state (host only,
    device only, both), each context possibly upgrading it to both or, now
    and then, flipping it to the other side; liveness random."""
    base = rng.integers(0, 3, size=nv)
    out = []
    for _ in range(k):
        eh, ed, xl = 0, 0, 0
        for v in range(nv):
            s = int(base[v])
            u = rng.random()
            if u < 0.3:
                s = 2
            elif u < 0.38:
                s = 1 - s if s < 2 else int(rng.integers(0, 2))
            eh |= (s in (0, 2)) << v
            ed |= (s in (1, 2)) << v
            xl |= int(rng.random() < 0.6) << v
        out.append(tuple(np.array([np.uint64(x)], dtype=np.uint64) for x in (eh, ed, xl)))
    return out


def _check_groups(groups, contexts):
    seen = []
    for m, absorbed in groups:
        held = 0
        for c in absorbed:
            assert not (m[0] & ~c[0]).any() and not (m[1] & ~c[1]).any(), "merged validity above an absorbed one"
            assert not (c[2] & ~m[2]).any(), "merged liveness below an absorbed one"
            held |= rs.word(c[0][0] | c[1][0])
            seen.append(P.ctx_key(c))
        assert not held & ~rs.word(m[0][0] | m[1][0]), "merged context leaves a held variable valid nowhere"
    assert sorted(seen) == sorted({P.ctx_key(c) for c in contexts})


def _serve_check(seed, merge_groups=P.merge_groups, max_contexts=1):
    rng = np.random.default_rng(seed)
    nv = int(rng.integers(1, 6))
    g = wl.random_graph(None, int(rng.integers(1, 6)), nv, max_out=2, acc_max=3, rng=rng)
    ctxs = _contexts(rng, nv, int(rng.integers(2, 7)))
    groups = merge_groups(ctxs, max_contexts)
    walks = rs.maximal_walks(g, g.entry, 2)
    for m, absorbed in groups:
        g.entry_host_valid, g.entry_dev_valid, g.exit_host_live = m
        t = rs.transfers_from_oracle(g, oracle.solve(g))
        for c in absorbed:
            sim = rs.PathSim(g, t, rs.word(c[0][0]), rs.word(c[1][0]), rs.word(c[2][0]))
            for blocks, edges in walks:
                sim.run(blocks, edges)
    return groups, ctxs


@pytest.mark.parametrize("max_contexts", [1, 2])
@pytest.mark.parametrize("seed", range(40))
def test_merged_instance_serves_every_absorbed_context(seed, max_contexts):
    groups, ctxs = _serve_check(7000 + seed, max_contexts=max_contexts)
    _check_groups(groups, ctxs)
    assert len(groups) <= max(max_contexts, len({P.ctx_key(c) for c in ctxs}))


def test_merge_keeps_conflicting_copies_apart():
    one = lambda x: np.array([np.uint64(x)], dtype=np.uint64)  # noqa: E731
    host_only = (one(1), one(0), one(1))
    dev_only = (one(0), one(1), one(1))
    both = (one(1), one(1), one(0))
    groups = P.merge_groups([host_only, dev_only, both], 1)
    assert len(groups) == 2  # `both' absorbs one side; the other stays alone
    _check_groups(groups, [host_only, dev_only, both])


# --------------------------------------------------------------------------
# planted mistakes (copies of the oracle's functions with one change each)
# --------------------------------------------------------------------------

def _map_gen_and(summ, callee_vars, var_map, caller_vars):
    Wr = (caller_vars + 63) // 64
    row = np.zeros((7, Wr), dtype=np.uint64)
    first = {}
    for v in range(callee_vars):
        t = int(var_map[v])
        if t < 0 or t >= caller_vars:
            continue
        for k in range(7):
            x = P._bit(summ[k], v)
            if k in (P.GEN_H, P.GEN_D):
                if x and first.get((t, k), 1):
                    P._set(row[k], t)
                elif not x:
                    row[k][t >> 6] &= ~(np.uint64(1) << np.uint64(t & 63))
                first[(t, k)] = x and first.get((t, k), 1)
            elif x:
                P._set(row[k], t)
    row[P.GEN_H] &= ~row[P.KILL_H]
    row[P.GEN_D] &= ~row[P.KILL_D]
    return row


def _map_no_kill_override(summ, callee_vars, var_map, caller_vars):
    row = np.zeros((7, (caller_vars + 63) // 64), dtype=np.uint64)
    for v in range(callee_vars):
        t = int(var_map[v])
        if 0 <= t < caller_vars:
            for k in range(7):
                if P._bit(summ[k], v):
                    P._set(row[k], t)
    return row


def _map_req_and(summ, callee_vars, var_map, caller_vars):
    row = P.map_summary(summ, callee_vars, var_map, caller_vars)
    seen = {}
    for v in range(callee_vars):
        t = int(var_map[v])
        if 0 <= t < caller_vars:
            for k in (P.REQ_H, P.REQ_D):
                seen[(t, k)] = seen.get((t, k), 1) & P._bit(summ[k], v)
    for (t, k), x in seen.items():
        if not x:
            row[k][t >> 6] &= ~(np.uint64(1) << np.uint64(t & 63))
    return row


def _merge_variant(valid_op, live_op, hole_check):
    def merge(contexts, max_contexts):
        d = {P.ctx_key(c): c for c in contexts}
        keys = sorted(d)
        if len(keys) <= max_contexts:
            return [(d[k], [d[k]]) for k in keys]
        out = [(d[k], [d[k]]) for k in keys[: max_contexts - 1]]
        m = list(d[keys[max_contexts - 1]])
        absorbed = [d[keys[max_contexts - 1]]]
        alone = []
        for k in keys[max_contexts:]:
            c = d[k]
            eh, ed, xl = valid_op(m[0], c[0]), valid_op(m[1], c[1]), live_op(m[2], c[2])
            if hole_check and ((m[0] | m[1] | c[0] | c[1]) & ~(eh | ed)).any():
                alone.append((c, [c]))
                continue
            m = [eh, ed, xl]
            absorbed.append(c)
        return out + [(tuple(m), absorbed)] + alone
    return merge


def _fails(fn, seeds):
    for s in seeds:
        try:
            fn(s)
        except (AssertionError, rs.Violation):
            return True
    return False


def test_planted_alias_mistakes_fail():
    tight = _tight()
    for bad in (_map_gen_and, _map_no_kill_override, _map_req_and):
        got = alias_pair_rows(bad)
        assert any(got[k] != tight[k] for k in tight), bad.__name__
    # the ones that are unsound also fail the bound against the renamed callee
    for bad in (_map_no_kill_override, _map_req_and):
        def case(seed, bad=bad):
            rng = np.random.default_rng(seed)
            cv = int(rng.choice([3, 6, 9]))
            cvars = int(rng.integers(1, 3))
            g = random_callee(rng, cv)
            vm = rng.integers(-1, cvars, size=cv).astype(np.int32)
            assert _sound(bad(oracle.summarize(g), cv, vm, cvars), oracle.summarize(renamed(g, vm, cvars)))
        assert _fails(case, range(600, 800)), bad.__name__


def test_planted_merge_mistakes_fail():
    plants = {
        "liveness merged by AND": _merge_variant(lambda a, b: a & b, lambda a, b: a & b, True),
        "validity merged by OR": _merge_variant(lambda a, b: a | b, lambda a, b: a | b, True),
        "no hole check": _merge_variant(lambda a, b: a & b, lambda a, b: a | b, False),
    }
    for name, bad in plants.items():
        assert _fails(lambda s, bad=bad: _serve_check(s, bad), range(7000, 7300)), name
