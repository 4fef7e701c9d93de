"""GPU parity: every output of libompdart (through the C ABI) equals the CPU
oracle bit for bit -- states, per-access flags, edge transfers and exit
transfers.  All of it is integer/bitwise work, so the tolerance is zero."""
import numpy as np
import pytest

import oracle
from paper_2406_13881_b300 import _native, workload as wl
from compare import assert_matches_oracle
import listings

pytestmark = pytest.mark.gpu


def run_both(g, **opts):
    res = _native.analyze(g, **opts)
    orc = oracle.solve(g)
    return res, orc


@pytest.mark.parametrize("path", [1, 0])
@pytest.mark.parametrize("name", sorted(listings.load()))
def test_paper_listings(name, path):
    g, _ = listings.to_cfg(listings.load()[name])
    res, orc = run_both(g, path=path, keep_states=True)
    assert_matches_oracle(g, res, orc)


@pytest.mark.parametrize("path", [1, 0])
@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_small_single_cfg(seed, path):
    g = wl.single_small(seed)
    res, orc = run_both(g, path=path, keep_states=True)
    assert_matches_oracle(g, res, orc)


@pytest.mark.parametrize("seed", range(60))
def test_random_graphs_sweep_path(seed):
    """Unstructured, often irreducible CFGs with unreachable blocks,
    duplicate edges and self-loops; 1 to 3 words per plane."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 40))
    nv = int(rng.choice([1, 5, 63, 64, 65, 130]))
    g = wl.random_graph(None, n, nv, max_out=3, acc_max=6, rng=rng)
    if seed % 3 == 1:
        g.entry_dev_valid = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
    if seed % 4 == 2:
        g.exit_host_live = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
    res, orc = run_both(g, path=1, keep_states=True)
    assert_matches_oracle(g, res, orc)


@pytest.mark.parametrize("seed", range(6))
def test_structured_multiword(seed):
    g = wl.structured(500 + seed, 3000, [64, 200, 700, 1024, 4096, 77][seed],
                      acc_min=1, acc_max=12, var_dist="zipf")
    res, orc = run_both(g, keep_states=True)
    assert_matches_oracle(g, res, orc)


def test_edge_cases():
    cases = [
        wl.from_lists([[]], [[]], 1),                                       # one block, no access
        wl.from_lists([[]], [[(0, 2, 1), (0, 1, 0), (1, 3, 1)]], 2),        # one block
        wl.from_lists([[1, 1], [2], []], [[(0, 2, 1)], [(0, 1, 0)], []], 3),  # duplicate edge
        wl.from_lists([[1], [1, 2], [], [2]], [[], [(0, 3, 1)], [(0, 1, 0)], [(0, 2, 0)]], 1),  # self loop, unreachable block 3
        wl.from_lists([[1], []], [[(5, 1, 1)], [(5, 1, 0)]], 6, entry_dev_valid=wl.var_mask(6, [5]),
                      entry_host_valid=wl.var_mask(6, [])),                   # valid only on the device
    ]
    for g in cases:
        for path in (1, 0):
            res, orc = run_both(g, path=path, keep_states=True)
            assert_matches_oracle(g, res, orc)


def test_bounded_loops_report_noconverge():
    """A fixed point that needs two sweeps with max_sweeps = 1 returns
    E_NOCONVERGE (the device loop stops and reports; nothing traps)."""
    g = wl.from_lists([[1], [2, 3], [1], []], [[], [(0, 1, 1)], [(0, 2, 0)], []], 1)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.analyze(g, path=1, max_sweeps=1)
    assert ei.value.code == _native.E_NOCONVERGE
    # and the library stays usable
    res, orc = run_both(g, path=1)
    assert_matches_oracle(g, res, orc)


def test_plan_reuse_is_deterministic():
    g = wl.single_small(7)
    p = _native.Plan(g, keep_states=True)
    outs = []
    for _ in range(3):
        p.run()
        p.sync()
        outs.append(p.fetch())
    for o in outs[1:]:
        for k in ("h_in", "d_in", "h_out", "d_out", "acc_flag", "from_exit"):
            np.testing.assert_array_equal(o[k], outs[0][k])
    assert p.launches > 0
    p.close()


@pytest.mark.parametrize("path", [1, 2])
def test_graph_replay_equals_oracle(path):
    """Runs replayed as one captured CUDA graph (the first run captures,
    the next ones launch it) give the oracle's answer every time, with and
    without the data region, and stay right after graph replay is switched
    off again."""
    for seed, region in ((3, False), (4, True)):
        g = wl.single_small(seed)
        orc = oracle.solve(g, data_region=region)
        p = _native.Plan(g, path=path, keep_states=True, data_region=region)
        p.graph(True)
        for _ in range(3):
            p.run()
            p.sync()
            assert_matches_oracle(g, p.fetch(), orc)
        p.graph(False)
        p.run()
        p.sync()
        assert_matches_oracle(g, p.fetch(), orc)
        p.close()


# --------------------------------------------------------------------------
# chunked scan solver
# --------------------------------------------------------------------------

@pytest.mark.parametrize("target", [1, 3, 8, 40])
@pytest.mark.parametrize("seed", range(8))
def test_scan_path_many_chunks(seed, target):
    """Structured CFGs cut into many small chunks: every carry, crossing
    edge and loop re-run path of the scan solver is exercised."""
    rng = np.random.default_rng(900 + seed)
    nv = int(rng.choice([3, 64, 100, 200]))
    g = wl.structured(900 + seed, int(rng.integers(20, 600)), nv, acc_min=0, acc_max=6,
                      var_dist="uniform", max_loop_depth=4, p_while=0.12)
    if seed % 2:
        g.entry_dev_valid = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
        g.exit_host_live = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
    res = _native.analyze(g, path=2, chunk_target=target, keep_states=True)
    assert res["path"] == 2
    assert_matches_oracle(g, res, oracle.solve(g))


@pytest.mark.parametrize("name", sorted(listings.load()))
def test_scan_path_listings_one_block_chunks(name):
    g, _ = listings.to_cfg(listings.load()[name])
    res = _native.analyze(g, path=2, chunk_target=1, keep_states=True)
    assert_matches_oracle(g, res, oracle.solve(g))


@pytest.mark.parametrize("seed", range(6))
def test_scan_equals_sweep(seed):
    g = wl.structured(1300 + seed, 5000, 300, acc_min=1, acc_max=10)
    a = _native.analyze(g, path=1, keep_states=True)
    b = _native.analyze(g, path=2, keep_states=True)
    for k in ("h_in", "d_in", "h_out", "d_out", "acc_flag", "from_exit"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    key = lambda r: sorted(zip(r["edge_xfers"]["edge"], r["edge_xfers"]["word"],
                               r["edge_xfers"]["to_bits"], r["edge_xfers"]["from_bits"]))
    assert key(a) == key(b)


def test_back_edge_transfer_without_loop_rerun():
    """A loop header whose entries disagree (host-valid on one, device-valid
    on the other) and whose latch leaves the host copy stale: the latch
    does not grow the header's meet, so no body re-walk happens, yet the
    back edge needs its own `from' (emitted from the latch's final value)."""
    g = wl.from_lists([[1, 2], [3], [3], [4, 5], [3], []],
                      [[], [(0, 2, 0)], [(0, 2, 1)], [(0, 1, 0)], [(0, 2, 1)], []], 1)
    for target in (0, 1, 2):
        res = _native.analyze(g, path=2, chunk_target=target, keep_states=True)
        orc = oracle.solve(g)
        assert orc["from_edge"][6].any()  # edge 6 = the back edge 4 -> 3 carries a `from'
        assert_matches_oracle(g, res, orc)


def test_continue_to_enclosing_loop():
    """Back edges from inside an inner loop to the enclosing loop's header
    (a `continue' of the outer loop) and an inner latch, under random
    accesses to a few variables: the value along the outer back edge leaves
    the inner loop before the outer loop closes."""
    succ = [[1], [2, 7], [3], [4, 6], [5, 1], [3], [1], []]
    rng = np.random.default_rng(11)
    for _ in range(40):
        accs = [[] for _ in succ]
        for b in range(1, 8):
            for v in range(3):
                if rng.random() < 0.45:
                    accs[b].append((v, int(rng.integers(1, 4)), int(rng.integers(0, 2))))
        g = wl.from_lists(succ, accs, 3)
        orc = oracle.solve(g)
        for target in (0, 1, 2):
            res = _native.analyze(g, path=2, chunk_target=target, keep_states=True)
            assert res["path"] == 2
            assert_matches_oracle(g, res, orc)


def test_unreachable_blocks_scan_path():
    g = wl.from_lists([[1], [2], [], [1], [3]], [[(0, 2, 0)], [(0, 1, 1)], [], [(1, 2, 1)], [(0, 3, 1)]], 3)
    res = _native.analyze(g, path=2, keep_states=True)
    assert_matches_oracle(g, res, oracle.solve(g))


@pytest.fixture(scope="module")
def large_cfg():
    return wl.single_large(2)


@pytest.mark.slow
def test_large_cfg_every_word_column(large_cfg):
    """The 2^20-block, 4096-variable CFG in the launch configuration the
    bench times (plan, run, view): every one of its 64 word columns against
    the oracle run on exactly those 64 variables (variables are independent
    bit problems, so a column is exact).  The oracle runs on host threads,
    a few columns at a time."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    g = large_cfg
    p = _native.Plan(g)
    p.run()
    p.sync()
    res = p.fetch()
    p.close()
    assert res["path"] == 2
    want = ["h_in", "d_in", "acc_flag", "to_edge", "from_edge", "from_exit"]

    def column(w):
        sub, keep = wl.restrict_word(g, w)
        return w, sub, keep, oracle.solve(sub, want=want)

    workers = max(1, min(8, os.cpu_count() or 1))
    done = 0
    with ThreadPoolExecutor(max_workers=workers) as ex:
        for lo in range(0, 64, workers):
            for w, sub, keep, orc in ex.map(column, range(lo, min(64, lo + workers))):
                assert_matches_oracle(sub, res, orc, words=slice(w, w + 1), acc_keep=keep)
                done += 1
    assert done == 64


@pytest.mark.parametrize("nv", [64, 300])
def test_large_cfg_parallel_host_build(nv):
    """A CFG large enough that ingestion and plan building run their passes
    on several host threads (and the accesses beside build_meta), with one
    or five words per row, so the chunk-carry scan takes column blocks of 1
    and 8 words: full parity with the oracle."""
    g = wl.structured(4242 + nv, 300_000, nv, acc_min=0, acc_max=4)
    res = _native.analyze(g, keep_states=True)
    assert res["path"] == 2
    assert_matches_oracle(g, res, oracle.solve(g))
