"""Pins of the CPU oracle against things other than itself (CPU only).

* the local rule against step-by-step simulation of every short access
  sequence (Sec. IV-D validity semantics);
* every phase against brute-force meet-over-paths (acyclic and bounded
  cyclic CFGs; all block and edge functions are distributive, so the
  fixed point must equal the meet over paths exactly);
* natural loops against the definition of dominance by removal;
* the loop closed form h = x & (g_B | p_B) on single-loop CFGs;
* the paper's listings, hand-translated to access form (tests/golden/);
* path simulation with version counters: no stale read (I1), every
  transfer copies the latest value (I2), transfers within the default
  mapping's count (I3), and no emitted transfer can be dropped.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2406_13881_b300 import workload as wl
import refsim as rs
import listings

pytestmark = pytest.mark.filterwarnings("ignore")

ALL1 = (1 << 64) - 1


def top(n):
    return (1 << n) - 1


# --------------------------------------------------------------------------
# local rule
# --------------------------------------------------------------------------

def _seq_cfg(seqs, n_vars):
    n = len(seqs)
    succs = [[b + 1] for b in range(n - 1)] + [[]]
    return wl.from_lists(succs, seqs, n_vars)


def test_local_rule_matches_step_simulation_exhaustive():
    syms3 = [(v, k, s) for v in (0, 1) for k in (1, 2, 3) for s in (0, 1)]
    syms2 = [(v, k, s) for v in (0, 1) for k in (1, 2) for s in (0, 1)]
    seqs = [[]]
    for L in range(1, 5):
        seqs += [list(p) for p in itertools.product(syms3, repeat=L)]
    seqs += [list(p) for p in itertools.product(syms2, repeat=5)]
    g = _seq_cfg(seqs, 2)
    res = oracle.solve(g, want=["gen_h", "kill_h", "gen_d", "kill_d", "ue_h", "ue_d", "def"])
    names = [("gen_h", ("gen", 0)), ("kill_h", ("kill", 0)), ("gen_d", ("gen", 1)),
             ("kill_d", ("kill", 1)), ("ue_h", ("ue", 0)), ("ue_d", ("ue", 1)), ("def", "def")]
    for b, sq in enumerate(seqs):
        ref = rs.local_sim(sq, 2)
        for on, rn in names:
            assert int(res[on][b, 0]) == ref[rn], (sq, on)


# --------------------------------------------------------------------------
# meet over paths
# --------------------------------------------------------------------------

def _walk_prefixes(g, max_edge_visits=2, limit=400000):
    """Every walk from the entry (each edge at most max_edge_visits times);
    for each block the distinct prefixes (blocks, edges) that end at it."""
    succ, eid = rs.graph_lists(g)
    pre = [dict() for _ in range(g.n_blocks)]
    visits = {}
    count = [0]

    def rec(b, blocks, edges):
        count[0] += 1
        if count[0] > limit:
            raise RuntimeError("walk explosion")
        key = tuple(edges)
        pre[b].setdefault(key, list(blocks))
        for t, e in zip(succ[b], eid[b]):
            if visits.get(e, 0) >= max_edge_visits:
                continue
            visits[e] = visits.get(e, 0) + 1
            rec(t, blocks + [t], edges + [e])
            visits[e] -= 1

    rec(g.entry, [g.entry], [])
    return [[(blocks, list(k)) for k, blocks in d.items()] for d in pre]


def _reachable(g, removed=None):
    succ, _ = rs.graph_lists(g)
    seen = set()
    if removed == g.entry:
        return seen
    st = [g.entry]
    seen.add(g.entry)
    while st:
        b = st.pop()
        for t in succ[b]:
            if t != removed and t not in seen:
                seen.add(t)
                st.append(t)
    return seen


def _brute_loops(g):
    """Natural loops by the definitions: a dominates b iff b is unreachable
    once a is removed; back edge t->h iff h dominates t."""
    succ, eid = rs.graph_lists(g)
    reach = _reachable(g)
    dom = {a: reach - _reachable(g, a) for a in reach}     # nodes dominated by a
    for a in reach:
        dom[a].add(a)
    preds = [[] for _ in range(g.n_blocks)]
    for b in range(g.n_blocks):
        for t, e in zip(succ[b], eid[b]):
            preds[t].append((b, e))
    headers, body = set(), {}
    for t in reach:
        for h, e in zip(succ[t], eid[t]):
            if t in dom[h]:
                headers.add(h)
    for h in headers:
        latches = [p for p, _ in preds[h] if p in reach and p in dom[h]]
        bd = {h}
        st = [x for x in latches if x != h]
        bd.update(st)
        while st:
            b = st.pop()
            for p, _ in preds[b]:
                if p in reach and p not in bd:
                    bd.add(p)
                    st.append(p)
        body[h] = bd
    entry_edges = set()
    for h in headers:
        for p, e in preds[h]:
            if p not in body[h]:
                entry_edges.add(e)
    return reach, headers, body, entry_edges


def _mop_all(g, max_edge_visits=2):
    """Every phase of the method by meet over paths, from the test's own
    local simulation and loop computation."""
    n, V = g.n_blocks, g.n_vars
    T = top(V)
    loc = [rs.local_sim(rs.block_accesses(g, b), V) for b in range(n)]
    reach, headers, body, entry_edges = _brute_loops(g)
    eh = T if g.entry_host_valid is None else rs.word(g.entry_host_valid[0]) & T
    ed = 0 if g.entry_dev_valid is None else rs.word(g.entry_dev_valid[0]) & T
    xl = T if g.exit_host_live is None else rs.word(g.exit_host_live[0]) & T

    def bwd(S):
        return lambda b, x: loc[b]["ue", S] | (x & ~loc[b]["def"])

    ant = {S: rs.mop_backward_may(g, bwd(S), xl if S == 0 else 0, max_edge_visits) for S in (0, 1)}
    live = [ant[0][b] | ant[1][b] for b in range(n)]
    pre = _walk_prefixes(g, max_edge_visits)
    edge_dst = {}
    for b in range(n):
        for e in range(int(g.succ_off[b]), int(g.succ_off[b + 1])):
            edge_dst[e] = (b, int(g.succ[e]))

    def fwd(S, cvec=None):
        def f(b, x):
            if cvec is not None:
                x = x | cvec[b]
            return loc[b]["gen", S] | (x & ~loc[b]["kill", S])
        return f

    hp_in = rs.mop_forward(n, pre, eh, T, fwd(0))
    hp_out = [fwd(0)(b, hp_in[b]) for b in range(n)]
    kill_or = {S: {h: 0 for h in headers} for S in (0, 1)}
    for h in headers:
        for b in body[h]:
            for S in (0, 1):
                kill_or[S][h] |= loc[b]["kill", S]
    # in-loop need: an S-read, before any write, on a walk from h that stays
    # in body(h) and does not come back to h
    lant = {S: {} for S in (0, 1)}
    succ, eid = rs.graph_lists(g)
    for h in headers:
        for S in (0, 1):
            acc = 0
            st = [([h], 0)]
            seen = set()
            while st:
                blocks, _ = st.pop()
                x = 0
                for blk in reversed(blocks):
                    x = loc[blk]["ue", S] | (x & ~loc[blk]["def"])
                acc |= x
                last = blocks[-1]
                for t in succ[last]:
                    if t in body[h] and t != h and blocks.count(t) < 2:
                        st.append((blocks + [t], 0))
            lant[S][h] = acc
    mask = {S: {h: lant[S][h] & ~kill_or[S][h] for h in headers} for S in (0, 1)}

    def edge_d(e, x):
        p, h = edge_dst[e]
        return x | (mask[1][h] & hp_out[p]) if e in entry_edges else x

    d_in = rs.mop_forward(n, pre, ed, T, fwd(1), edge_d)
    d_out = [fwd(1)(b, d_in[b]) for b in range(n)]
    C = [live[b] & ~d_in[b] & T for b in range(n)]

    def edge_h(e, x):
        p, h = edge_dst[e]
        return x | (mask[0][h] & d_out[p]) if e in entry_edges else x

    hm = rs.mop_forward(n, pre, eh, T, fwd(0, C), edge_h)
    h_in = [hm[b] | C[b] if b in reach else T for b in range(n)]
    return dict(reach=reach, headers=headers, entry_edges=entry_edges, ant_h=ant[0], ant_d=ant[1],
                live=live, hp_in=hp_in, d_in=d_in, hm=hm, h_in=h_in, mask_h=mask[0], mask_d=mask[1])


def _check_against_mop(g, max_edge_visits):
    res = oracle.solve(g)
    m = _mop_all(g, max_edge_visits)
    for b in range(g.n_blocks):
        assert bool(res["reachable"][b]) == (b in m["reach"])
        if b not in m["reach"]:
            continue
        assert int(res["ant_h_in"][b, 0]) == m["ant_h"][b], ("AntH", b)
        assert int(res["ant_d_in"][b, 0]) == m["ant_d"][b], ("AntD", b)
        assert int(res["hp_in"][b, 0]) == m["hp_in"][b], ("Hp", b)
        assert int(res["d_in"][b, 0]) == m["d_in"][b], ("D", b)
        assert int(res["hm"][b, 0]) == m["hm"][b], ("Hm", b)
        assert int(res["h_in"][b, 0]) == m["h_in"][b], ("H", b)
        assert bool(res["is_header"][b]) == (b in m["headers"])
        if b in m["headers"]:
            assert int(res["mask_h"][b, 0]) == m["mask_h"][b]
            assert int(res["mask_d"][b, 0]) == m["mask_d"][b]
    for e in range(g.n_edges):
        assert bool(res["is_loop_entry"][e]) == (e in m["entry_edges"])


@pytest.mark.parametrize("seed", range(60))
def test_fixed_point_equals_mop_acyclic(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 10))
    g = wl.random_graph(None, n, int(rng.integers(1, 7)), acyclic=True, max_out=2, rng=rng)
    if seed % 3 == 1:
        g.entry_dev_valid = np.array([rng.integers(0, 1 << 6)], dtype=np.uint64)
    if seed % 4 == 2:
        g.exit_host_live = np.array([rng.integers(0, 1 << 6)], dtype=np.uint64)
    _check_against_mop(g, 1)


@pytest.mark.parametrize("seed", range(40))
def test_fixed_point_equals_mop_cyclic(seed):
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(2, 7))
    g = wl.random_graph(None, n, int(rng.integers(1, 6)), acyclic=False, max_out=2, acc_max=3, rng=rng)
    if seed % 3 == 1:
        g.entry_dev_valid = np.array([rng.integers(0, 1 << 5)], dtype=np.uint64)
    _check_against_mop(g, 2)


@pytest.mark.parametrize("seed", range(8))
def test_fixed_point_equals_mop_structured(seed):
    g = wl.structured(3000 + seed, 12, 4, p_if_then=0.2, p_if_else=0.2, p_while=0.25, body_mean=1.6,
                      max_depth=3, max_loop_depth=2, region_mode="count", n_regions=2,
                      target_frac=0.3, acc_min=0, acc_max=3, var_dist="uniform")
    _check_against_mop(g, 2)


# --------------------------------------------------------------------------
# loops
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(80))
def test_natural_loops_match_dominance_by_removal(seed):
    rng = np.random.default_rng(4000 + seed)
    g = wl.random_graph(None, int(rng.integers(2, 14)), 1, max_out=3, acc_max=0, rng=rng)
    res = oracle.solve(g, want=["is_header", "is_loop_entry", "reachable"])
    reach, headers, body, entry_edges = _brute_loops(g)
    assert {b for b in range(g.n_blocks) if res["is_header"][b]} == headers
    assert {e for e in range(g.n_edges) if res["is_loop_entry"][e]} == entry_edges


def _compose(fs):
    """Compose per-bit functions x -> g | (x & p), applied left to right."""
    g, p = 0, ALL1
    for gi, pi in fs:
        g, p = gi | (g & pi), p & pi
    return g, p


@pytest.mark.parametrize("seed", range(30))
def test_loop_header_closed_form(seed):
    """Single while loop 0 -> 1(h) -> 2 -> 3(latch) -> 1, 1 -> 4: the plain
    host validity at the header is x_entry & (g_B | p_B), with (g_B, p_B) the
    header->body->latch function (Kam-Ullman: one pass suffices)."""
    rng = np.random.default_rng(5000 + seed)
    V = 6
    accs = [[(int(rng.integers(V)), int(rng.integers(1, 4)), int(rng.integers(2))) for _ in range(int(rng.integers(0, 4)))]
            for _ in range(5)]
    g = wl.from_lists([[1], [2, 4], [3], [1], []], accs, V)
    res = oracle.solve(g)
    loc = [rs.local_sim(a, V) for a in accs]
    for S, key_in, key_out in ((0, "hp_in", "hp_out"),):
        gB, pB = _compose([(loc[b]["gen", S], ALL1 & ~loc[b]["kill", S]) for b in (1, 2, 3)])
        x = int(res[key_out][0, 0])
        assert int(res[key_in][1, 0]) == x & (gB | pB) & top(V)


# --------------------------------------------------------------------------
# the paper's listings
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(listings.load()))
def test_paper_listing(name):
    case = listings.load()[name]
    g, vid = listings.to_cfg(case)
    res = oracle.solve(g)
    assert listings.oracle_sets(res) == listings.expected_sets(case, g, vid), case["cite"]


# --------------------------------------------------------------------------
# special cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(20))
def test_host_only_program_needs_no_transfer(seed):
    rng = np.random.default_rng(6000 + seed)
    g = wl.random_graph(None, int(rng.integers(2, 20)), 8, p_dev=0.0, rng=rng)
    res = oracle.solve(g)
    assert not listings.oracle_sets(res)


def test_single_block_uses_local_rule_only():
    # device write then host read then device read of the same variable
    g = wl.from_lists([[]], [[(0, 2, 1), (0, 1, 0), (0, 1, 1), (1, 1, 1)]], 2)
    res = oracle.solve(g)
    # the host read after the device write needs a local `from'; the device
    # read of var 1 at the top needs a `to' from the valid host copy; var 0
    # is device-last-written and live at exit -> no exit copy needed because
    # the local `from' already made the host valid
    assert list(res["acc_flag"]) == [0, 2, 0, 1]
    assert not res["from_exit"].any()
    assert not res["to_edge"].size and not res["from_edge"].size


def test_exit_from_only_for_device_written_live_vars():
    # entry = exit: device writes var 0, host writes var 1, var 2 untouched
    g = wl.from_lists([[]], [[(0, 2, 1), (1, 2, 0)]], 3,
                      exit_host_live=wl.var_mask(3, [0, 1, 2]))
    res = oracle.solve(g)
    assert int(res["from_exit"][0, 0]) == 0b001
    g.exit_host_live = wl.var_mask(3, [1, 2])
    res = oracle.solve(g)
    assert int(res["from_exit"][0, 0]) == 0


def test_invalid_inputs_rejected():
    g = wl.from_lists([[1], [0]], [[], []], 1)          # entry has a predecessor
    with pytest.raises(oracle.OracleError):
        oracle.solve(g)
    g = wl.from_lists([[1], []], [[(5, 1, 0)], []], 2)   # variable out of range
    with pytest.raises(oracle.OracleError):
        oracle.solve(g)
    g = wl.from_lists([[7], []], [[], []], 1)            # successor out of range
    with pytest.raises(oracle.OracleError):
        oracle.solve(g)


# --------------------------------------------------------------------------
# path simulation
# --------------------------------------------------------------------------

def _sim_check(g, max_edge_visits, check_i3, check_irredundant):
    res = oracle.solve(g)
    t = rs.transfers_from_oracle(g, res)
    V = g.n_vars
    eh = top(V) if g.entry_host_valid is None else rs.word(g.entry_host_valid[0])
    ed = 0 if g.entry_dev_valid is None else rs.word(g.entry_dev_valid[0])
    xl = top(V) if g.exit_host_live is None else rs.word(g.exit_host_live[0])
    hoist = [e for e in range(g.n_edges) if res["is_loop_entry"][e]]
    paths = rs.maximal_walks(g, g.entry, max_edge_visits)
    sim = rs.PathSim(g, t, eh, ed, xl, hoist)
    for blocks, edges in paths:
        n_all, charged, default = sim.run(blocks, edges)
        if check_i3:
            assert charged <= default, (blocks, charged, default)
    if check_irredundant and paths:
        for desc, u in rs.each_single_removal(t):
            s2 = rs.PathSim(g, u, eh, ed, xl, hoist)
            broke = False
            for blocks, edges in paths:
                try:
                    s2.run(blocks, edges)
                except rs.Violation:
                    broke = True
                    break
            assert broke, "redundant transfer: " + desc
    return res, paths


@pytest.mark.parametrize("seed", range(40))
def test_paths_random_acyclic(seed):
    rng = np.random.default_rng(7000 + seed)
    g = wl.random_graph(None, int(rng.integers(2, 9)), int(rng.integers(1, 5)), acyclic=True,
                        max_out=2, rng=rng)
    _sim_check(g, 1, False, True)


@pytest.mark.parametrize("seed", range(40))
def test_paths_random_cyclic(seed):
    rng = np.random.default_rng(8000 + seed)
    g = wl.random_graph(None, int(rng.integers(2, 7)), int(rng.integers(1, 4)), max_out=2,
                        acc_max=3, rng=rng)
    _sim_check(g, 2, False, True)


@pytest.mark.parametrize("seed", range(25))
def test_paths_structured_with_kernels(seed):
    g = wl.structured(9000 + seed, int(8 + seed % 9), 3, p_if_then=0.2, p_if_else=0.15,
                      p_while=0.25, body_mean=1.7, max_depth=3, max_loop_depth=2,
                      region_mode="count", n_regions=2, target_frac=0.35, acc_min=0,
                      acc_max=3, var_dist="uniform")
    _sim_check(g, 2, True, True)


@pytest.mark.parametrize("name", sorted(listings.load()))
def test_paths_paper_listings(name):
    g, _ = listings.to_cfg(listings.load()[name])
    res, paths = _sim_check(g, 3, True, True)
    # on the paper's own programs even the raw count stays within the default
    V = g.n_vars
    sim = rs.PathSim(g, rs.transfers_from_oracle(g, res),
                     top(V) if g.entry_host_valid is None else rs.word(g.entry_host_valid[0]),
                     0 if g.entry_dev_valid is None else rs.word(g.entry_dev_valid[0]), top(V), [])
    for blocks, edges in paths:
        n_all, _, default = sim.run(blocks, edges)
        if any(g.region[b] >= 0 for b in blocks):
            assert n_all <= default


def test_small_paper_shaped_cfg_random_paths():
    """The 64-block, one-nest program: 3000 random complete paths."""
    g = wl.single_small(1)
    res = oracle.solve(g)
    t = rs.transfers_from_oracle(g, res)
    hoist = [e for e in range(g.n_edges) if res["is_loop_entry"][e]]
    sim = rs.PathSim(g, t, top(g.n_vars), 0, top(g.n_vars), hoist)
    for blocks, edges in rs.random_paths(g, g.entry, 3000, seed=11):
        n_all, charged, default = sim.run(blocks, edges)
        assert charged <= default
