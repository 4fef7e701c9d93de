"""Pins of the oracle's interprocedural parts (Sec. IV-C: callee side effects
applied at call sites), checked against things other than the oracle itself:

* a callee summary equals brute-force enumeration of every entry-to-exit
  path of small acyclic callees, simulated access by access;
* a call whose row is the summary of a one-block callee ("reads, then at
  most one write" per variable) is indistinguishable from that block's
  accesses written in place: same states, liveness, edge and exit
  transfers, and the call's transfer planes are the inlined reads' flags;
* the call-site rows (state the callee starts from, liveness after the call)
  equal the entry rows of blocks obtained by cutting the caller's block
  around the call (outside loops: the loop rule reads each block's net
  kills, and a cut inside a loop body can change those).
"""
import numpy as np
import pytest

import oracle
from paper_2406_13881_b300 import workload as wl

KR, KW, KRW = 1, 2, 3
H, D = 0, 1


def bits(row, nv):
    return [(int(row[v >> 6]) >> (v & 63)) & 1 for v in range(nv)]


def to_row(vals, nv):
    W = (nv + 63) // 64
    r = np.zeros(W, dtype=np.uint64)
    for v, x in enumerate(vals):
        if x:
            r[v >> 6] |= np.uint64(1) << np.uint64(v & 63)
    return r


def random_dag(rng, n, nv, acc_max=4, call_rows=None, p_call=0.0):
    """Blocks 0..n-1, edges only forward, block 0 the entry (every block is
    given at least one predecessor so most are reachable)."""
    succs = [[] for _ in range(n)]
    for j in range(1, n):
        succs[int(rng.integers(0, j))].append(j)
    for _ in range(int(rng.integers(0, n))):
        i, j = sorted(rng.integers(0, n, size=2))
        if i < j and j != 0:
            succs[i].append(int(j))
    accs = []
    for _ in range(n):
        lst = []
        for _ in range(int(rng.integers(0, acc_max + 1))):
            if call_rows is not None and rng.random() < p_call:
                lst.append(("call", int(rng.integers(0, len(call_rows)))))
            else:
                lst.append((int(rng.integers(0, nv)), int(rng.integers(1, 4)), int(rng.integers(0, 2))))
        accs.append(lst)
    return succs, accs


def to_cfg(succs, accs, nv, call_rows=None):
    """CFG with plain accesses (var, kind, space) and ("call", row)."""
    plain = [[a for a in lst] for lst in accs]
    so = np.zeros(len(succs) + 1, dtype=np.int32)
    so[1:] = np.cumsum([len(s) for s in succs])
    succ = np.array([t for s in succs for t in s], dtype=np.int32)
    ao = np.zeros(len(accs) + 1, dtype=np.int32)
    ao[1:] = np.cumsum([len(a) for a in plain])
    words = []
    for lst in plain:
        for a in lst:
            if a[0] == "call":
                words.append(0x80000000 | a[1])
            else:
                words.append(int(wl.pack_access([a[0]], [a[1]], [a[2]])[0]))
    g = wl.CFG(len(succs), nv, 0, so, succ, ao, np.array(words, dtype=np.uint32))
    if call_rows is not None:
        g.call_planes = np.ascontiguousarray(np.stack(call_rows), dtype=np.uint64)
    return g


def paths(succs, b=0):
    if not succs[b]:
        yield [b]
        return
    for t in succs[b]:
        for p in paths(succs, t):
            yield [b] + p


def events(path, accs, nv, call_rows):
    """Per-variable event list along a path: ('r', S), ('w', S) and for a
    call ('call', rh, rd, gh, kh, gd, kd, md)."""
    ev = [[] for _ in range(nv)]
    for b in path:
        for a in accs[b]:
            if a[0] == "call":
                row = call_rows[a[1]]
                planes = [bits(row[k], nv) for k in range(7)]
                for v in range(nv):
                    f = tuple(planes[k][v] for k in range(7))
                    if any(f):
                        ev[v].append(("call",) + f)
            else:
                v, k, S = a
                if k & KR:
                    ev[v].append(("r", S))
                if k & KW:
                    ev[v].append(("w", S))
    return ev


def simulate(evs, start_valid):
    """Run one variable's events: [valid on host, valid on device]."""
    val = [start_valid, start_valid]
    for e in evs:
        if e[0] == "r":
            val[e[1]] = 1
        elif e[0] == "w":
            val[e[1]] = 1
            val[1 - e[1]] = 0
        else:
            _, rh, rd, gh, kh, gd, kd, _md = e
            if rh:
                val[H] = 1
            if rd:
                val[D] = 1
            val[H] = 1 if gh else 0 if kh else val[H]
            val[D] = 1 if gd else 0 if kd else val[D]
    return val


def upward(evs, S):
    """Is the first event among {S-read, must-write} an S-read?"""
    for e in evs:
        if e[0] == "r" and e[1] == S:
            return 1
        if e[0] == "w":
            return 0
        if e[0] == "call":
            if (e[1] if S == H else e[2]):
                return 1
            if e[7]:
                return 0
    return 0


def written(evs):
    return int(any(e[0] == "w" or (e[0] == "call" and e[7]) for e in evs))


def brute_summary(succs, accs, nv, call_rows):
    ps = list(paths(succs))
    req = [[0] * nv, [0] * nv]
    gen = [[1] * nv, [1] * nv]
    kill = [[0] * nv, [0] * nv]
    md = [1] * nv
    for p in ps:
        ev = events(p, accs, nv, call_rows)
        for v in range(nv):
            for S in (H, D):
                req[S][v] |= upward(ev[v], S)
            from_stale = simulate(ev[v], 0)
            from_valid = simulate(ev[v], 1)
            for S in (H, D):
                gen[S][v] &= from_stale[S]
                kill[S][v] |= 1 - from_valid[S]
            md[v] &= written(ev[v])
    return [req[H], req[D], gen[H], kill[H], gen[D], kill[D], md]


def random_call_row(rng, nv):
    """A consistent callee row: per variable a random mini-callee's effect."""
    planes = [[0] * nv for _ in range(7)]
    for v in range(nv):
        r = rng.random()
        if r < 0.3:
            continue
        evs = []
        for _ in range(int(rng.integers(1, 4))):
            evs.append(("r" if rng.random() < 0.6 else "w", int(rng.integers(0, 2))))
        planes[0][v] = upward(evs, H)
        planes[1][v] = upward(evs, D)
        st, sv = simulate(evs, 0), simulate(evs, 1)
        planes[2][v], planes[3][v] = st[H], 1 - sv[H]
        planes[4][v], planes[5][v] = st[D], 1 - sv[D]
        planes[6][v] = written(evs)
    return np.stack([to_row(p, nv) for p in planes])


@pytest.mark.parametrize("seed", range(40))
def test_summary_equals_path_enumeration(seed):
    rng = np.random.default_rng(7000 + seed)
    nv = int(rng.choice([3, 5, 70]))
    rows = [random_call_row(rng, nv) for _ in range(3)] if seed % 2 else None
    succs, accs = random_dag(rng, int(rng.integers(1, 8)), nv, call_rows=rows, p_call=0.25)
    g = to_cfg(succs, accs, nv, rows)
    got = oracle.summarize(g)
    want = brute_summary(succs, accs, nv, rows)
    for k, name in enumerate(["ReqH", "ReqD", "GenH", "KillH", "GenD", "KillD", "MustDef"]):
        np.testing.assert_array_equal(got[k], to_row(want[k], nv), err_msg=name)


def test_summary_closed_forms():
    # identity callee: no effect at all
    g = to_cfg([[]], [[]], 4)
    np.testing.assert_array_equal(oracle.summarize(g), np.zeros((7, 1), dtype=np.uint64))
    # a device kernel writing v0 and a host read of v1
    g = to_cfg([[]], [[(0, KW, D), (1, KR, H)]], 2)
    s = oracle.summarize(g)
    assert [int(x[0]) for x in s] == [0b10, 0, 0b10, 0b01, 0b01, 0, 0b01]
    # no reachable exit (the callee loops forever): no net effect
    g = to_cfg([[1], [1]], [[(0, KW, D)], []], 1)
    s = oracle.summarize(g)
    assert [int(x[0]) for x in s[2:]] == [0, 0, 0, 0, 0]


def reads_then_one_write(rng, nv):
    """Accesses of a one-block callee: per touched variable some reads, then
    at most one write (possibly a read-write) as its last event."""
    out = []
    for v in rng.permutation(nv)[: int(rng.integers(1, nv + 1))]:
        for _ in range(int(rng.integers(0, 3))):
            out.append((int(v), KR, int(rng.integers(0, 2))))
        if rng.random() < 0.6:
            out.append((int(v), int(rng.choice([KW, KRW])), int(rng.integers(0, 2))))
    order = rng.permutation(len(out))
    # keep each variable's own order, interleave variables
    per_var = {}
    for a in out:
        per_var.setdefault(a[0], []).append(a)
    seq, idx = [], {v: 0 for v in per_var}
    for i in order:
        v = out[i][0]
        seq.append(per_var[v][idx[v]])
        idx[v] += 1
    return seq


@pytest.mark.parametrize("seed", range(30))
def test_call_equals_inlined_block(seed):
    rng = np.random.default_rng(8000 + seed)
    nv = int(rng.choice([4, 9, 66]))
    base = wl.random_graph(None, int(rng.integers(2, 12)), nv, max_out=2, acc_max=4, rng=rng)
    body = reads_then_one_write(rng, nv)
    row = oracle.summarize(to_cfg([[]], [body], nv))
    b = int(rng.integers(0, base.n_blocks))
    ao, acc = base.acc_off, base.acc
    pos = int(rng.integers(ao[b], ao[b + 1] + 1))
    inl_words = np.array([int(wl.pack_access([v], [k], [S])[0]) for v, k, S in body], dtype=np.uint32)
    # caller with the call in place / with the block inlined
    call_acc = np.concatenate([acc[:pos], [np.uint32(0x80000000)], acc[pos:]]).astype(np.uint32)
    inl_acc = np.concatenate([acc[:pos], inl_words, acc[pos:]]).astype(np.uint32)
    call_ao, inl_ao = ao.copy(), ao.copy()
    call_ao[b + 1:] += 1
    inl_ao[b + 1:] += len(body)
    gc = wl.CFG(base.n_blocks, nv, base.entry, base.succ_off, base.succ, call_ao, call_acc)
    gc.call_planes = row.reshape(1, 7, -1)
    gi = wl.CFG(base.n_blocks, nv, base.entry, base.succ_off, base.succ, inl_ao, inl_acc)
    for k in ("entry_host_valid", "entry_dev_valid", "exit_host_live"):
        setattr(gc, k, getattr(base, k, None))
        setattr(gi, k, getattr(base, k, None))
    rc, ri = oracle.solve(gc), oracle.solve(gi)
    for k in ("h_in", "d_in", "h_out", "d_out", "live_in", "to_edge", "from_edge", "from_exit", "mask_h", "mask_d"):
        np.testing.assert_array_equal(rc[k], ri[k], err_msg=k)
    # flags of the other accesses agree; the call's planes are the inlined reads' flags
    n_before = pos
    np.testing.assert_array_equal(rc["acc_flag"][:n_before], ri["acc_flag"][:n_before])
    np.testing.assert_array_equal(rc["acc_flag"][n_before + 1:], ri["acc_flag"][n_before + len(body):])
    if rc["reachable"][b]:
        to, fr = np.zeros(nv, dtype=int), np.zeros(nv, dtype=int)
        for j, (v, k, S) in enumerate(body):
            f = int(ri["acc_flag"][n_before + j])
            if f == 1:
                to[v] = 1
            if f == 2:
                fr[v] = 1
        np.testing.assert_array_equal(rc["call_to"][0], to_row(to, nv))
        np.testing.assert_array_equal(rc["call_from"][0], to_row(fr, nv))
        assert int(rc["acc_flag"][n_before]) == (1 if to.any() else 0) | (2 if fr.any() else 0)


@pytest.mark.parametrize("seed", range(20))
def test_two_calls_in_one_block_equal_cut_blocks(seed):
    """Two calls in one block: cutting it into [a][call 0][b][call 1][c]
    gives the same call-site rows (the second call's must-writes end the
    first call's liveness).  Only outside loops: inside one, the loop rule
    looks at each block's net kills, which a cut can change."""
    rng = np.random.default_rng(9500 + seed)
    nv = int(rng.choice([3, 8, 65]))
    base = to_cfg(*random_dag(rng, int(rng.integers(2, 8)), nv), nv)
    rows = [random_call_row(rng, nv) for _ in range(2)]
    b = int(rng.integers(0, base.n_blocks))
    ao, acc = base.acc_off, base.acc
    mine = list(acc[ao[b]:ao[b + 1]])
    i, j = sorted(int(x) for x in rng.integers(0, len(mine) + 1, size=2))
    pieces = [mine[:i], [np.uint32(0x80000000)], mine[i:j], [np.uint32(0x80000001)], mine[j:]]
    new_block = sum(pieces, [])
    blocks = [list(acc[ao[k]:ao[k + 1]]) for k in range(base.n_blocks)]
    n = base.n_blocks
    succs = [list(base.succ[base.succ_off[k]:base.succ_off[k + 1]]) for k in range(n)]

    def make(succ_lists, block_lists):
        so = np.zeros(len(succ_lists) + 1, dtype=np.int32)
        so[1:] = np.cumsum([len(x) for x in succ_lists])
        a2 = np.zeros(len(block_lists) + 1, dtype=np.int32)
        a2[1:] = np.cumsum([len(x) for x in block_lists])
        g = wl.CFG(len(succ_lists), nv, base.entry, so, np.array([t for x in succ_lists for t in x], dtype=np.int32),
                   a2, np.array([w for x in block_lists for w in x], dtype=np.uint32))
        g.call_planes = np.stack(rows)
        return g, so

    g, _ = make(succs, blocks[:b] + [new_block] + blocks[b + 1:])
    ids = list(range(n, n + 4))  # call 0, middle, call 1, rest
    cut_succs = [x[:] for x in succs] + [[ids[1]], [ids[2]], [ids[3]], succs[b][:]]
    cut_succs[b] = [ids[0]]
    cut_blocks = [x[:] for x in blocks] + [pieces[1], pieces[2], pieces[3], pieces[4]]
    cut_blocks[b] = pieces[0]
    gcut, _ = make(cut_succs, cut_blocks)
    r, rc = oracle.solve(g), oracle.solve(gcut)
    if not r["reachable"][b]:
        return
    for k, (blk, after) in enumerate([(ids[0], ids[1]), (ids[2], ids[3])]):
        np.testing.assert_array_equal(r["call_entry_h"][k], rc["h_in"][blk] | rows[k][0])
        np.testing.assert_array_equal(r["call_entry_d"][k], rc["d_in"][blk] | rows[k][1])
        np.testing.assert_array_equal(r["call_exit_live"][k], rc["live_in"][after])
        np.testing.assert_array_equal(r["call_to"][k], rc["call_to"][k])
        np.testing.assert_array_equal(r["call_from"][k], rc["call_from"][k])


@pytest.mark.parametrize("seed", range(25))
def test_call_rows_equal_cut_blocks(seed):
    """Cut the block holding a call into [before][call][after] blocks: the
    callee's starting state is the call block's entry state plus what the
    call requires, and the host anticipation after the call is the entry
    anticipation of the block after it."""
    rng = np.random.default_rng(9000 + seed)
    nv = int(rng.choice([3, 8, 65]))
    base = to_cfg(*random_dag(rng, int(rng.integers(2, 10)), nv), nv)
    row = random_call_row(rng, nv)
    b = int(rng.integers(0, base.n_blocks))
    ao, acc = base.acc_off, base.acc
    pos = int(rng.integers(ao[b], ao[b + 1] + 1))
    call_acc = np.concatenate([acc[:pos], [np.uint32(0x80000000)], acc[pos:]]).astype(np.uint32)
    call_ao = ao.copy()
    call_ao[b + 1:] += 1
    g = wl.CFG(base.n_blocks, nv, base.entry, base.succ_off, base.succ, call_ao, call_acc)
    g.call_planes = row.reshape(1, 7, -1)
    # the cut version: b keeps the accesses before the call and jumps to a
    # new block c (the call), which jumps to a new block d (the rest), which
    # takes b's successors
    n = base.n_blocks
    succs = [list(base.succ[base.succ_off[i]:base.succ_off[i + 1]]) for i in range(n)]
    c, d = n, n + 1
    succs_cut = [s[:] for s in succs] + [[d], succs[b][:]]
    succs_cut[b] = [c]
    blocks = [list(acc[ao[i]:ao[i + 1]]) for i in range(n)]
    blocks_cut = [x[:] for x in blocks] + [[np.uint32(0x80000000)], blocks[b][pos - ao[b]:]]
    blocks_cut[b] = blocks[b][: pos - ao[b]]
    so = np.zeros(n + 3, dtype=np.int32)
    so[1:] = np.cumsum([len(s) for s in succs_cut])
    ao2 = np.zeros(n + 3, dtype=np.int32)
    ao2[1:] = np.cumsum([len(x) for x in blocks_cut])
    gcut = wl.CFG(n + 2, nv, base.entry, so, np.array([t for s in succs_cut for t in s], dtype=np.int32), ao2,
                  np.array([w for x in blocks_cut for w in x], dtype=np.uint32))
    gcut.call_planes = g.call_planes
    r, rcut = oracle.solve(g), oracle.solve(gcut)
    if not r["reachable"][b]:
        return
    np.testing.assert_array_equal(r["call_entry_h"][0], rcut["h_in"][c] | row[0])
    np.testing.assert_array_equal(r["call_entry_d"][0], rcut["d_in"][c] | row[1])
    np.testing.assert_array_equal(r["call_exit_live"][0], rcut["live_in"][d])
    np.testing.assert_array_equal(r["call_to"][0], row[1] & ~rcut["d_in"][c])
    np.testing.assert_array_equal(r["call_from"][0], row[0] & ~rcut["h_in"][c])
    # the cut CFG has the same states at the original blocks
    for k in ("h_in", "d_in", "live_in"):
        np.testing.assert_array_equal(r[k], rcut[k][:n], err_msg=k)
    # and no transfer on the two edges the cut added
    e_bc, e_cd = so[b], so[c]
    assert not rcut["to_edge"][[e_bc, e_cd]].any() and not rcut["from_edge"][[e_bc, e_cd]].any()
