"""Eager `to' placement on the GPU (opts.eager_to; Sec. IV-E, Algorithm 1):
every output through the C ABI equals ``oracle.solve(..., eager_to=True)``
bit for bit -- states, access flags, edge transfers (the eager `to's among
them) and exit transfers -- on both solvers (the chunked scan solver for
reducible CFGs, with edge constants on every edge and the back edges'
constants taken at the loop closure; the sweep solver for any CFG), on
the hand-built programs of the oracle's pins, the paper's listings, random
reducible and irreducible CFGs, wide variable sets, small chunks, batches,
and together with the data region and its directives."""
import numpy as np
import pytest

import listings
import oracle
from compare import assert_matches_oracle
from oracle import classify as C
from paper_2406_13881_b300 import _native, workload as wl
from test_directives_gpu import assert_directives
from test_oracle_classify import kernel_cfg

pytestmark = pytest.mark.gpu

H, D = 0, 1
R, W = 1, 2


def check(g, **opts):
    """Both solvers (the scan solver where the CFG allows it) against the oracle."""
    orc = oracle.solve(g, eager_to=True)
    res = None
    for path in (1, 0):
        res = _native.analyze(g, eager_to=True, keep_states=True, path=path, **opts)
        assert res["path"] == 1 or path == 0
        assert_matches_oracle(g, res, orc)
    return res, orc


HAND = {
    "straight_line": ([[1], [2], []], [[(0, W, H)], [], [(0, R, D)]]),
    "host_loop": ([[1], [2, 3], [1], []], [[], [], [(0, W, H)], [(0, R, D)]]),
    "nested_host_loops": ([[1], [2, 5], [3, 4], [2], [1], []], [[], [], [], [(0, W, H)], [], [(0, R, D)]]),
    "branch": ([[1, 2], [3], [3], []], [[(0, W, H)], [(0, R, D)], [(0, R, H)], []]),
    "device_write_first": ([[1], [2], []], [[(0, W, H)], [(0, W, D)], [(0, R, D)]]),
    "kernel_in_loop": ([[1], [2, 4], [3], [1], []], [[], [], [(0, W, H)], [(0, R, D)], []]),
    "entry_valid": ([[1], []], [[], [(0, R, D)]]),
}


@pytest.mark.parametrize("name", sorted(HAND))
def test_hand_programs(name):
    succ, accs = HAND[name]
    g = wl.from_lists(succ, accs, 1)
    res, orc = check(g)
    if name == "host_loop":  # sunk out of the loop onto its exit edge
        assert orc["to_edge"][2, 0] == 1 and not orc["acc_flag"].any()


@pytest.mark.parametrize("name", sorted(listings.load()))
def test_paper_listings(name):
    g, _ = listings.to_cfg(listings.load()[name])
    check(g)


@pytest.mark.parametrize("seed", range(16))
def test_random_graphs(seed):
    rng = np.random.default_rng(16000 + seed)
    g = wl.random_graph(None, int(rng.integers(3, 60)), int(rng.integers(1, 130)), max_out=3, rng=rng)
    check(g)


@pytest.mark.parametrize("seed", range(8))
def test_structured_wide(seed):
    g = wl.structured(17000 + seed, 1500, [64, 200, 700, 1024][seed % 4], acc_min=1, acc_max=10,
                      var_dist="zipf")
    check(g)


def test_paper_shaped_small_cfgs():
    for seed in range(1, 4):
        check(wl.single_small(seed))


def test_default_is_lazy_and_differs():
    """Off by default; on a program with a host loop the two placements
    differ and each equals its own oracle."""
    g = wl.from_lists(*HAND["host_loop"], 1)
    lazy = _native.analyze(g, keep_states=True)
    assert_matches_oracle(g, lazy, oracle.solve(g))
    eager, _ = check(g)
    assert lazy["acc_flag"].any() and not eager["acc_flag"].any()


def test_with_data_region_and_directives():
    for seed in range(6):
        g = kernel_cfg(18000 + seed, int(10 + seed * 5), int(1 + seed * 20))
        orc = oracle.solve(g, eager_to=True, data_region=True)
        res = _native.analyze(g, eager_to=True, data_region=True, keep_states=True)
        assert_matches_oracle(g, res, orc)
        assert_directives(g, res, g, orc, C.classify(g, orc))


def test_batch():
    cfgs = wl.batch(3, n_cfgs=12)
    b = _native.Batch(cfgs, eager_to=True, keep_states=True)
    b.run()
    assert (b.sync() == 0).all()
    for i, g in enumerate(cfgs):
        assert_matches_oracle(g, b.fetch(i), oracle.solve(g, eager_to=True))
    b.close()


@pytest.mark.parametrize("target", [1, 3, 8])
def test_scan_path_small_chunks(target):
    """Edge constants across chunk boundaries (carry edges) and on back
    edges at every loop closure: structured CFGs cut into tiny chunks."""
    for seed in range(6):
        g = wl.structured(19000 + seed, 400, 130)
        orc = oracle.solve(g, eager_to=True)
        res = _native.analyze(g, eager_to=True, keep_states=True, path=2, chunk_target=target)
        assert res["path"] == 2
        assert_matches_oracle(g, res, orc)


def test_scan_path_is_chosen_for_reducible_cfgs():
    g = wl.single_small(1)
    res = _native.analyze(g, eager_to=True)
    assert res["path"] == 2
    assert_matches_oracle(g, res, oracle.solve(g, eager_to=True))


def test_calls_refused_library_stays_usable():
    """CFGs with call pseudo-accesses take no eager placement (E_INVALID);
    the library answers the next request."""
    from test_calls_gpu import structured_with_calls
    g = structured_with_calls(3, 200, 40)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.analyze(g, eager_to=True)
    assert ei.value.code == _native.E_INVALID
    check(wl.single_small(2))


def test_batch_with_a_calls_cfg_fails_it_alone():
    from test_calls_gpu import structured_with_calls
    good = [wl.single_small(3), wl.structured(19100, 500, 200)]
    cfgs = [good[0], structured_with_calls(5, 200, 40), good[1]]
    b = _native.Batch(cfgs, eager_to=True, keep_states=True)
    b.run()
    st = b.sync()
    assert st[1] == _native.E_INVALID and st[0] == 0 and st[2] == 0
    for i in (0, 2):
        assert_matches_oracle(cfgs[i], b.fetch(i), oracle.solve(cfgs[i], eager_to=True))
    b.close()
