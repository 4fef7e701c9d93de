"""Call pseudo-accesses on the GPU (Sec. IV-C side effects at call sites):
plans and batches of CFGs holding calls equal the oracle bit for bit,
including the call-site rows (transfers before each call, the state the
callee starts from, liveness after it)."""
import numpy as np
import pytest

import oracle
from paper_2406_13881_b300 import _native, workload as wl
from compare import assert_matches_oracle
from test_oracle_calls import random_call_row

pytestmark = pytest.mark.gpu


def with_calls(g, rng, n_rows=4, p_call=0.15):
    """Insert call accesses (random consistent callee rows) at random
    places of g's access lists; some blocks get several calls."""
    rows = [random_call_row(rng, g.n_vars) for _ in range(n_rows)]
    accs = []
    for b in range(g.n_blocks):
        lst = list(g.acc[g.acc_off[b]:g.acc_off[b + 1]])
        k = 0
        while rng.random() < p_call and k < 3:
            lst.insert(int(rng.integers(0, len(lst) + 1)), np.uint32(0x80000000 | int(rng.integers(0, n_rows))))
            k += 1
        accs.append(lst)
    ao = np.zeros(g.n_blocks + 1, dtype=np.int32)
    ao[1:] = np.cumsum([len(x) for x in accs])
    out = wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off, g.succ, ao,
                 np.array([a for x in accs for a in x], dtype=np.uint32))
    out.call_planes = np.ascontiguousarray(np.stack(rows), dtype=np.uint64)
    out.entry_host_valid, out.entry_dev_valid, out.exit_host_live = g.entry_host_valid, g.entry_dev_valid, \
        g.exit_host_live
    return out


def structured_with_calls(seed, n, nv, **kw):
    rng = np.random.default_rng(seed)
    g = wl.structured(None, n, nv, acc_min=0, acc_max=6, var_dist="uniform", max_loop_depth=3, p_while=0.1,
                      rng=rng, **kw)
    if seed % 2:
        g.entry_dev_valid = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
        g.exit_host_live = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
    return with_calls(g, rng)


@pytest.mark.parametrize("target", [0, 1, 5])
@pytest.mark.parametrize("seed", range(10))
def test_plan_with_calls(seed, target):
    nv = [3, 64, 100, 200, 700][seed % 5]
    g = structured_with_calls(300 + seed, int(np.random.default_rng(seed).integers(10, 400)), nv)
    res = _native.analyze(g, keep_states=True, chunk_target=target)
    assert res["path"] == 2 and len(res["call_site_acc"]) > 0
    assert_matches_oracle(g, res, oracle.solve(g))


def test_batch_with_calls():
    cfgs = [structured_with_calls(400 + i, 50 + 37 * i, [64, 100, 130][i % 3]) for i in range(18)]
    cfgs += [wl.structured(500 + i, 200, 64) for i in range(4)]  # and CFGs without calls
    b = _native.Batch(cfgs, keep_states=True)
    b.run()
    assert (b.sync() == 0).all()
    for i, g in enumerate(cfgs):
        assert_matches_oracle(g, b.fetch(i), oracle.solve(g))
    b.close()
    res, st = _native.analyze_batch(cfgs, keep_states=True)
    assert (st == 0).all()
    for g, r in zip(cfgs, res):
        assert_matches_oracle(g, r, oracle.solve(g))


def test_calls_need_the_scan_solver():
    g = wl.from_lists([[1, 2], [2], [1, 3], []], [[(0, 2, 1)], [(0, 1, 0)], [], []], 2)  # irreducible
    g = with_calls(g, np.random.default_rng(1), p_call=1.0)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.analyze(g)
    assert ei.value.code == _native.E_INVALID
    b = _native.Batch([g, wl.single_small(2)])
    assert list(b.status) == [_native.E_INVALID, 0]
    b.close()


def test_batch_one_function_in_several_contexts():
    """The same CFG arrays (calls included) given several times with other
    boundary rows, as the program driver does for a function's calling
    contexts: ingested and folded once, every context still exact."""
    import copy
    rng = np.random.default_rng(77)
    bases = [structured_with_calls(600 + i, 120 + 50 * i, 100) for i in range(3)]
    cfgs = []
    for k in range(12):
        g = copy.copy(bases[k % 3])
        W = g.W
        g.entry_host_valid = rng.integers(0, 2**63, size=W, dtype=np.uint64)
        g.entry_dev_valid = rng.integers(0, 2**63, size=W, dtype=np.uint64)
        g.exit_host_live = rng.integers(0, 2**63, size=W, dtype=np.uint64)
        cfgs.append(g)
    res, st = _native.analyze_batch(cfgs, keep_states=True)
    assert (st == 0).all()
    for g, r in zip(cfgs, res):
        assert_matches_oracle(g, r, oracle.solve(g))
