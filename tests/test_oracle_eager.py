"""Eager `to' placement in the oracle (``oracle.solve(..., eager_to=True)``;
Sec. IV-E: a `target update to' follows the host write that produced the
data, and Algorithm 1 moves it past the loops that sweep the array).

Pinned without the oracle's own equations:
* hand-built programs whose placement follows from the paper's prose (a
  write in a host loop gets its `to' after the loop; a branch that reads
  nothing on the device gets none; a kernel inside the loop keeps it
  inside);
* the must-anticipation plane against brute force over the walks of small
  random CFGs (every walk from the point reads on the device before any
  write or exit);
* path simulation: on every walk the eager transfers leave no stale read
  (I1) and never copy a stale host copy (I2), and on every complete path
  they make no more `to's than the lazy placement does (an eager `to' is
  always followed by a device read that the lazy rule would have paid for);
* planted mistakes (a `to' on a branch that does not read, a `to' from a
  stale host copy) fail those checks.
"""
import numpy as np
import pytest

import oracle
import refsim as rs
from paper_2406_13881_b300 import workload as wl

H, D = 0, 1
R, W, RW = 1, 2, 3


def edge(g, src, dst):
    for e in range(int(g.succ_off[src]), int(g.succ_off[src + 1])):
        if int(g.succ[e]) == dst:
            return e
    raise KeyError((src, dst))


def to_edges(res, v=0):
    return sorted(int(e) for e in np.nonzero((res["to_edge"][:, v >> 6] >> np.uint64(v & 63)) & np.uint64(1))[0])


def both(g):
    return oracle.solve(g), oracle.solve(g, eager_to=True)


def test_straight_line_to_follows_the_write():
    # b0: host write; b1: nothing; b2: device read
    g = wl.from_lists([[1], [2], []], [[(0, W, H)], [], [(0, R, D)]], 1)
    lazy, eager = both(g)
    assert list(lazy["acc_flag"]) == [0, 1] and to_edges(lazy) == []
    assert list(eager["acc_flag"]) == [0, 0] and to_edges(eager) == [edge(g, 0, 1)]


def test_host_loop_sinks_to_its_exit():
    # for (...) a[i] = ...;  (host)   then a kernel reads a
    g = wl.from_lists([[1], [2, 3], [1], []], [[], [], [(0, W, H)], [(0, R, D)]], 1)
    lazy, eager = both(g)
    assert to_edges(lazy) == [] and lazy["acc_flag"][1] == 1
    assert to_edges(eager) == [edge(g, 1, 3)] and eager["acc_flag"][1] == 0


def test_nested_host_loops_sink_out_of_both():
    # outer header 1, inner header 2, inner body 3 writes on the host, the
    # outer latch 4; the kernel 5 after the outer loop
    succ = [[1], [2, 5], [3, 4], [2], [1], []]
    accs = [[], [], [], [(0, W, H)], [], [(0, R, D)]]
    g = wl.from_lists(succ, accs, 1)
    _, eager = both(g)
    assert to_edges(eager) == [edge(g, 1, 5)]


def test_branch_without_device_read_gets_none():
    # b0 writes on the host; b1 reads on the device, b2 only on the host
    g = wl.from_lists([[1, 2], [3], [3], []], [[(0, W, H)], [(0, R, D)], [(0, R, H)], []], 1)
    _, eager = both(g)
    assert to_edges(eager) == [edge(g, 0, 1)]
    assert not eager["acc_flag"].any()


def test_device_write_first_needs_no_to():
    g = wl.from_lists([[1], [2], []], [[(0, W, H)], [(0, W, D)], [(0, R, D)]], 1)
    lazy, eager = both(g)
    assert to_edges(eager) == [] and not eager["acc_flag"].any()
    assert not lazy["acc_flag"].any()


def test_kernel_in_loop_keeps_the_to_inside():
    # each iteration: host write (2), kernel read (3)
    g = wl.from_lists([[1], [2, 4], [3], [1], []], [[], [], [(0, W, H)], [(0, R, D)], []], 1)
    _, eager = both(g)
    assert to_edges(eager) == [edge(g, 2, 3)]


def test_data_valid_at_the_entry():
    # valid on the host at the entry (produced before the function): the
    # `to' goes on the first edge from which every path reads it on the
    # device; a read in the entry block itself keeps the lazy `to'
    g = wl.from_lists([[1], []], [[], [(0, R, D)]], 1)
    lazy, eager = both(g)
    assert list(lazy["acc_flag"]) == [1] and list(eager["acc_flag"]) == [0]
    assert to_edges(eager) == [edge(g, 0, 1)]
    g = wl.from_lists([[1], []], [[(0, R, D)], []], 1)
    lazy, eager = both(g)
    assert list(eager["acc_flag"]) == list(lazy["acc_flag"]) == [1]
    assert to_edges(eager) == []


def test_off_by_default():
    g = wl.single_small(2)
    a = oracle.solve(g)
    assert not a["ant_dm_in"].any()
    b = oracle.solve(g, eager_to=False)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


# --------------------------------------------------------------------------
# brute force
# --------------------------------------------------------------------------

def first_event_ok(g, blocks, v, at_exit):
    """Along a walk: does a device read of v come before any write of v
    (and before the end of a complete path)?  None = undecided."""
    for b in blocks:
        for (u, t, s) in rs.events(rs.block_accesses(g, b)):
            if u != v:
                continue
            if t == "W":
                return False
            if s == D:
                return True
    return False if at_exit else None


def brute_antdm(g, walks_from):
    N, V = g.n_blocks, g.n_vars
    out = np.zeros(N, np.uint64)
    for b in range(N):
        walks = walks_from[b]
        for v in range(V):
            ok = True
            for blocks, _ in walks:
                last = blocks[-1]
                at_exit = g.succ_off[last] == g.succ_off[last + 1]
                if first_event_ok(g, blocks, v, at_exit) is False:
                    ok = False
                    break
            if ok:
                out[b] |= np.uint64(1) << np.uint64(v)
    return out


@pytest.mark.parametrize("seed", range(30))
def test_must_anticipation_brute_force(seed):
    rng = np.random.default_rng(12000 + seed)
    acyclic = seed % 2 == 0
    g = wl.random_graph(None, int(rng.integers(2, 8)), int(rng.integers(1, 5)), acyclic=acyclic,
                        max_out=2, acc_max=3, rng=rng)
    res = oracle.solve(g, eager_to=True)
    reach = res["reachable"].astype(bool)
    walks = {b: rs.maximal_walks(g, b, 2) for b in range(g.n_blocks)}
    want = brute_antdm(g, walks)
    got = res["ant_dm_in"][:, 0]
    for b in range(g.n_blocks):
        if reach[b]:
            assert int(got[b]) == int(want[b]), (b, bin(int(got[b])), bin(int(want[b])))


# --------------------------------------------------------------------------
# path simulation
# --------------------------------------------------------------------------

def count_to(t, g, blocks, edges):
    n = 0
    for e in edges:
        n += bin(t["to_edge"].get(e, 0)).count("1")
    for b in blocks:
        for i in range(int(g.acc_off[b]), int(g.acc_off[b + 1])):
            n += t["flag"].get(i, 0) == 1
    return n


def sim_both(g, max_edge_visits, t_eager=None):
    V = g.n_vars
    eh = (1 << V) - 1 if g.entry_host_valid is None else rs.word(g.entry_host_valid[0])
    ed = 0 if g.entry_dev_valid is None else rs.word(g.entry_dev_valid[0])
    xl = (1 << V) - 1 if g.exit_host_live is None else rs.word(g.exit_host_live[0])
    lazy, eager = both(g)
    tl = rs.transfers_from_oracle(g, lazy)
    te = rs.transfers_from_oracle(g, eager) if t_eager is None else t_eager(g, eager)
    sim = rs.PathSim(g, te, eh, ed, xl)
    walks = rs.maximal_walks(g, g.entry, max_edge_visits)
    for blocks, edges in walks:
        sim.run(blocks, edges)  # raises on I1 / I2
        last = blocks[-1]
        if g.succ_off[last] == g.succ_off[last + 1]:  # a complete path
            assert count_to(te, g, blocks, edges) <= count_to(tl, g, blocks, edges), (blocks, edges)
    return lazy, eager


@pytest.mark.parametrize("seed", range(30))
def test_paths_random_acyclic(seed):
    rng = np.random.default_rng(13000 + seed)
    g = wl.random_graph(None, int(rng.integers(2, 9)), int(rng.integers(1, 5)), acyclic=True,
                        max_out=2, rng=rng)
    sim_both(g, 1)


@pytest.mark.parametrize("seed", range(30))
def test_paths_random_cyclic(seed):
    rng = np.random.default_rng(14000 + seed)
    g = wl.random_graph(None, int(rng.integers(2, 7)), int(rng.integers(1, 4)), max_out=2, acc_max=3,
                        rng=rng)
    sim_both(g, 2)


@pytest.mark.parametrize("seed", range(20))
def test_paths_structured_with_kernels(seed):
    g = wl.structured(15000 + seed, int(8 + seed % 9), 3, p_if_then=0.2, p_if_else=0.15,
                      p_while=0.25, body_mean=1.7, max_depth=3, max_loop_depth=2,
                      region_mode="count", n_regions=2, target_frac=0.35, acc_min=0,
                      acc_max=3, var_dist="uniform")
    lazy, eager = sim_both(g, 2)
    # eager only ever adds device validity
    assert not (lazy["d_in"] & ~eager["d_in"]).any()


def test_planted_to_on_a_branch_that_does_not_read_is_caught():
    g = wl.from_lists([[1, 2], [3], [3], []], [[(0, W, H)], [(0, R, D)], [(0, R, H)], []], 1)

    def plant(g, res):
        t = rs.transfers_from_oracle(g, res)
        t["to_edge"][edge(g, 0, 2)] = 1  # may- instead of must-anticipation
        return t

    with pytest.raises(AssertionError):
        sim_both(g, 1, plant)


def test_planted_to_from_a_stale_host_copy_is_caught():
    # the kernel writes, then reads: a `to' in between copies a stale host copy
    g = wl.from_lists([[1], []], [[(0, W, D)], [(0, R, D)]], 1)

    def plant(g, res):
        t = rs.transfers_from_oracle(g, res)
        t["to_edge"][edge(g, 0, 1)] = 1  # no host-validity test
        return t

    with pytest.raises(rs.Violation):
        sim_both(g, 1, plant)


# --------------------------------------------------------------------------
# with the single target data region and its directives
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(30))
def test_paths_region_mode_and_directives(seed):
    """Eager placement in the data-region mode: the raw transfers and the
    classified program (map clauses, kernel-entry transfers, consolidated
    updates) both leave no stale read and copy no stale value on any walk,
    and eager device validity contains the lazy one."""
    from oracle import classify as C
    from test_oracle_classify import classified_transfers, kernel_cfg
    g = kernel_cfg(20000 + seed, int(8 + seed % 16), int(1 + seed % 4))
    top = (1 << g.n_vars) - 1
    res = oracle.solve(g, data_region=True, eager_to=True)
    lazy = oracle.solve(g, data_region=True)
    assert not (lazy["d_in"] & ~res["d_in"]).any()
    walks = rs.maximal_walks(g, g.entry, 2)
    raw = rs.PathSim(g, rs.transfers_from_oracle(g, res), top, 0, top)
    classified = rs.PathSim(g, classified_transfers(g, res, C.classify(g, res)), top, 0, top)
    for blocks, edges in walks:
        raw.run(blocks, edges)
        classified.run(blocks, edges)
