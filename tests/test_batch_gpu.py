"""Batched analysis (ompdart_batch_* / ompdart_analyze_batch) on the GPU:
every CFG's result in a batch equals the oracle and the same CFG analysed
alone, bit for bit; one bad CFG does not fail the rest; the captured graph,
the direct launches and repeated runs agree."""
import numpy as np
import pytest

import oracle
from paper_2406_13881_b300 import _native, workload as wl
from compare import assert_matches_oracle

pytestmark = pytest.mark.gpu

KEYS = ("h_in", "d_in", "h_out", "d_out", "acc_flag", "from_exit", "exit_blocks", "live_in")


def xfer_key(r):
    x = r["edge_xfers"]
    return sorted(zip(x["edge"].tolist(), x["word"].tolist(), x["to_bits"].tolist(), x["from_bits"].tolist()))


def assert_same(a, b):
    for k in KEYS:
        if k in a or k in b:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert xfer_key(a) == xfer_key(b)


def mixed_cfgs(seed, n=48):
    """Structured CFGs of many sizes and word counts (several CFGs per
    word count, so arenas hold many CFGs), irreducible random graphs (plans
    of their own), unreachable blocks, one-block CFGs, non-default entry
    and exit rows."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 8
        if kind == 7:
            g = wl.random_graph(None, int(rng.integers(1, 30)), int(rng.choice([1, 64, 100])), rng=rng)
        elif kind == 6:
            g = wl.from_lists([[]], [[(0, 2, 1), (0, 1, 0)]], int(rng.choice([1, 64, 100])))
        else:
            nv = int(rng.choice([1, 3, 64, 100, 256, 1024]))
            nb = int(rng.choice([16, 40, 200, 700, 2500]))
            g = wl.structured(None, nb, nv, acc_min=0, acc_max=8, var_dist="uniform",
                              max_loop_depth=3, p_while=0.1, rng=rng)
        if i % 5 == 1:
            g.entry_dev_valid = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
        if i % 5 == 2:
            g.exit_host_live = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
        out.append(g)
    # irreducible: the cycle 1 <-> 2 has two entries (a plan of its own)
    out.append(wl.from_lists([[1, 2], [2], [1, 3], []], [[(0, 2, 1)], [(0, 1, 0)], [(1, 2, 1)], [(0, 1, 0)]], 2))
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_oracle_and_alone(graph):
    cfgs = mixed_cfgs(11)
    b = _native.Batch(cfgs, keep_states=True, no_graph=not graph)
    assert (b.status == 0).all()
    info = b.info()
    assert info["solo"] >= 1 and len(info["arenas"]) >= 3
    b.run()
    assert (b.sync() == 0).all()
    for i, g in enumerate(cfgs):
        res = b.fetch(i)
        assert_matches_oracle(g, res, oracle.solve(g))
        assert_same(res, _native.analyze(g, keep_states=True))
    b.close()


def test_batch_runs_repeat_bit_exact():
    cfgs = mixed_cfgs(12, n=24)
    b = _native.Batch(cfgs, keep_states=True)
    first = None
    for _ in range(3):
        b.run()
        b.sync()
        outs = [b.fetch(i) for i in range(len(cfgs))]
        if first is None:
            first = outs
        else:
            for a, c in zip(first, outs):
                assert_same(a, c)
    b.close()


@pytest.mark.parametrize("target", [1, 3, 16])
def test_batch_many_small_chunks(target):
    """Small chunk targets: many chunks per CFG, so carries and crossing
    edges run next to the CFG boundaries of the arena."""
    rng = np.random.default_rng(50 + target)
    cfgs = [wl.structured(None, int(rng.integers(16, 300)), int(rng.choice([64, 130])), acc_min=0, acc_max=6,
                          var_dist="uniform", max_loop_depth=4, p_while=0.12, rng=rng) for _ in range(20)]
    b = _native.Batch(cfgs, chunk_target=target, keep_states=True)
    b.run()
    assert (b.sync() == 0).all()
    for i, g in enumerate(cfgs):
        assert_matches_oracle(g, b.fetch(i), oracle.solve(g))
    b.close()


def test_bad_cfgs_do_not_fail_the_rest():
    good = wl.single_small(3)
    bad_entry = wl.from_lists([[1], [0]], [[], []], 2)          # the entry has a predecessor
    call = wl.from_lists([[1], []], [[], []], 2)
    call.acc = np.array([0x80000000], dtype=np.uint32)           # call pseudo-access without a table
    call.acc_off = np.array([0, 1, 1], dtype=np.int32)
    other = wl.structured(77, 500, 200)
    cfgs = [good, bad_entry, call, other]
    b = _native.Batch(cfgs, keep_states=True)
    assert list(b.status) == [0, _native.E_INVALID, _native.E_INVALID, 0]
    b.run()
    st = b.sync()
    assert list(st) == [0, _native.E_INVALID, _native.E_INVALID, 0]
    for i in (0, 3):
        assert_matches_oracle(cfgs[i], b.fetch(i), oracle.solve(cfgs[i]))
    with pytest.raises(_native.OmpdartError) as ei:
        b.fetch(1)
    assert ei.value.code == _native.E_INVALID
    b.close()


def test_analyze_batch_one_call():
    cfgs = mixed_cfgs(13, n=32)
    cfgs.insert(5, wl.from_lists([[1], [0]], [[], []], 2))       # rejected, the rest proceed
    res, st = _native.analyze_batch(cfgs, keep_states=True)
    assert st[5] == _native.E_INVALID and res[5] is None
    for i, g in enumerate(cfgs):
        if i != 5:
            assert st[i] == 0
            assert_matches_oracle(g, res[i], oracle.solve(g))


def test_empty_batch():
    b = _native.Batch([])
    b.run()
    assert len(b.sync()) == 0
    assert b.info() == {"arenas": [], "solo": 0, "launches": 0}
    b.close()
    res, st = _native.analyze_batch([])
    assert res == [] and len(st) == 0


def fanout_cfg(n_vars=4096):
    """Two diamonds in a row whose joins need a `from' of every variable on
    one in-edge: 2 x 64 transfer records in one chunk, more than a chunk's
    first record buffer holds (the buffers grow and the emission reruns)."""
    allv = list(range(n_vars))
    dev_w = [(v, 2, 1) for v in allv]
    host_r = [(v, 1, 0) for v in allv]
    return wl.from_lists([[1, 2], [3], [3], [4, 5], [6], [6], []],
                         [[], dev_w, [], host_r, dev_w, [], host_r], n_vars)


def test_record_buffers_grow_plan_and_batch():
    g = fanout_cfg()
    res = _native.analyze(g, path=2, chunk_target=1000, keep_states=True)
    assert_matches_oracle(g, res, oracle.solve(g))
    assert len(res["edge_xfers"]) == 128
    cfgs = [g, wl.structured(5, 300, 4096), fanout_cfg()]
    b = _native.Batch(cfgs, chunk_target=1000, keep_states=True)
    for _ in range(2):  # the second run replays a graph captured after the buffers grew
        b.run()
        assert (b.sync() == 0).all()
        for i, c in enumerate(cfgs):
            assert_matches_oracle(c, b.fetch(i), oracle.solve(c))
    b.close()


def test_plan_graph_replay_after_record_growth():
    """A plan replaying its run as a graph: the first run (the capture)
    overflows the record streams, so the sync grows them and drops the
    graph; the next run captures it again with the new buffers.  Every run
    equals the oracle."""
    g = fanout_cfg()
    orc = oracle.solve(g)
    p = _native.Plan(g, path=2, chunk_target=1000, keep_states=True)
    p.graph(True)
    for _ in range(3):
        p.run()
        p.sync()
        res = p.fetch()
        assert_matches_oracle(g, res, orc)
        assert len(res["edge_xfers"]) == 128
    p.close()


def test_autotuned_batch():
    cfgs = mixed_cfgs(14, n=40)
    b = _native.Batch(cfgs, keep_states=True, tune=True)
    info = b.info()
    for a in info["arenas"]:
        assert a["chunk_target"] in (16, 32, 64, 128, 256, 512) and a["warps_per_cta"] in (2, 4)
    b.run()
    assert (b.sync() == 0).all()
    for i, g in enumerate(cfgs):
        assert_matches_oracle(g, b.fetch(i), oracle.solve(g))
    b.close()


@pytest.mark.slow
def test_paper_shaped_batch_sampled():
    """The 10,000-CFG batch in the launch configuration the batch bench
    times (arenas per word count, captured graph): every 97th CFG against
    the oracle, every CFG's status OK."""
    cfgs = wl.batch(3)
    b = _native.Batch(cfgs)
    b.run()
    assert (b.sync() == 0).all()
    for i in range(0, len(cfgs), 97):
        assert_matches_oracle(cfgs[i], b.fetch(i), oracle.solve(cfgs[i]))
    b.close()
