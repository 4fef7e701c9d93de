"""The serving loop (ompdart_server_*) on the GPU: every request's result is
the same alone and in the mix (bit for bit, and equal to the oracle), the
device-memory budget rejects what can never fit, malformed requests fail on
their own, and Poisson-timed replays complete with recorded latencies."""
import numpy as np
import pytest

import oracle
from paper_2406_13881_b300 import _native, workload as wl
from compare import assert_matches_oracle
from test_batch_gpu import assert_same, mixed_cfgs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("max_batch,max_inflight", [(4096, 2), (8, 3), (1, 1)])
def test_results_same_alone_and_in_the_mix(max_batch, max_inflight):
    cfgs = mixed_cfgs(21, n=40)
    srv = _native.Server(max_batch=max_batch, max_inflight=max_inflight, keep_states=True)
    tickets = [srv.submit(g) for g in cfgs]
    for g, t in zip(cfgs, tickets):
        st, lat, res = srv.wait(t)
        assert st == 0 and lat >= 0.0, (st, _native.load().ompdart_last_error())
        assert_matches_oracle(g, res, oracle.solve(g))
        assert_same(res, _native.analyze(g, keep_states=True))
    s = srv.stats()
    assert s["completed"] == len(cfgs) and s["failed"] == 0
    assert s["batches"] >= (len(cfgs) + max_batch - 1) // max_batch
    assert s["bytes_in_use"] == 0 and s["peak_bytes"] > 0
    srv.close()


def test_budget_and_bad_requests_fail_alone():
    huge = wl.from_lists([[i + 1] for i in range(39)] + [[]], [[(0, 1, 0)]] * 40, 1 << 24)  # 3 planes of 80 MiB
    bad = wl.from_lists([[1], [0]], [[], []], 2)                                            # entry with a predecessor
    good = [wl.single_small(s) for s in (1, 2, 3)]
    srv = _native.Server(hbm_budget_bytes=64 << 20, keep_states=True)
    t_good0 = srv.submit(good[0])
    t_huge = srv.submit(huge)
    t_bad = srv.submit(bad)
    t_rest = [srv.submit(g) for g in good[1:]]
    assert srv.wait(t_huge)[0] == _native.E_BUDGET
    assert srv.wait(t_bad)[0] == _native.E_INVALID
    for g, t in zip(good, [t_good0] + t_rest):
        st, _, res = srv.wait(t)
        assert st == 0
        assert_matches_oracle(g, res, oracle.solve(g))
    with pytest.raises(_native.OmpdartError) as ei:
        srv.wait(t_bad)  # already collected
    assert ei.value.code == _native.E_INVALID
    srv.close()


def test_poisson_replay_completes():
    rng = np.random.default_rng(5)
    pool = wl.batch(8, n_cfgs=60)
    n = 400
    idx = rng.integers(0, len(pool), size=n)
    cfgs = [pool[i] for i in idx]
    arrival = np.cumsum(rng.exponential(1e6 / 20000.0, size=n))  # 20k requests/s
    srv = _native.Server(max_inflight=2)
    tickets = srv.replay(cfgs, arrival)
    srv.drain()
    alone = {}
    for k, (i, t) in enumerate(zip(idx, tickets)):
        st, lat, res = srv.wait(t)
        assert st == 0 and lat > 0.0
        if k % 37 == 0:
            if i not in alone:
                alone[i] = _native.analyze(pool[i])
            assert_same(res, alone[i])
    s = srv.stats()
    assert s["completed"] == n and s["p99_ms"] >= s["p50_ms"] > 0.0
    assert s["mean_batch"] >= 1.0
    srv.close()


def test_wait_timeout_keeps_the_ticket():
    srv = _native.Server()
    g = wl.structured(3, 4000, 2048)
    t = srv.submit(g)
    try:
        st, _, _ = srv.wait(t, timeout_ms=0)
        assert st == 0  # already done: fine too
    except _native.OmpdartError as e:
        assert e.code == _native.E_TIMEOUT
        st, _, res = srv.wait(t)
        assert st == 0 and res is not None
    srv.close()


def _copy_cfg(g, **rows):
    """The same CFG in fresh buffers (what a serving caller sends again),
    with optional other entry / exit rows."""
    h = wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off.copy(), g.succ.copy(), g.acc_off.copy(), g.acc.copy(),
               None if g.region is None else g.region.copy(), g.entry_host_valid, g.entry_dev_valid,
               g.exit_host_live, g.call_planes)
    for k, v in rows.items():
        setattr(h, k, v)
    return h


@pytest.mark.parametrize("workers,group", [(4, 0), (1, 2), (3, 64)])
def test_resident_mode_reuses_plans_with_per_request_rows(workers, group):
    """Resident mode: the same CFGs sent again in fresh buffers hit the plan
    cache, requests for one CFG with different entry / exit rows get their
    own results, and every result equals the oracle -- with groups that
    hold several requests for one plan (successive rounds) and workers
    that find a plan busy in another worker."""
    rng = np.random.default_rng(12)
    base = mixed_cfgs(23, n=12)
    reqs = []
    for rep in range(3):
        for g in base:
            W = g.W
            top = wl.var_mask(g.n_vars, range(g.n_vars))
            rows = {} if rep == 0 else {
                "entry_host_valid": rng.integers(0, 2**63, size=W, dtype=np.uint64) & top | top * np.uint64(rep == 1),
                "entry_dev_valid": rng.integers(0, 2**63, size=W, dtype=np.uint64) & top,
                "exit_host_live": rng.integers(0, 2**63, size=W, dtype=np.uint64) & top}
            reqs.append(_copy_cfg(g, **rows))
    srv = _native.Server(resident=True, workers=workers, max_batch=group, keep_states=True)
    tickets = [srv.submit(g) for g in reqs]
    srv.drain()
    for g, t in zip(reqs, tickets):
        st, lat, res = srv.wait(t)
        assert st == 0 and lat >= 0.0, (st, _native.load().ompdart_last_error())
        assert_matches_oracle(g, res, oracle.solve(g))
    s = srv.stats()
    assert s["completed"] == len(reqs) and s["failed"] == 0
    assert s["cache_misses"] >= len(base) and s["cache_hits"] >= len(reqs) - 2 * len(base)
    assert s["cached_plans"] == len(base)
    srv.close()


def test_resident_mode_budget_and_bad_requests():
    """A budget that holds only some plans: least recently used idle plans
    are dropped and a request that still does not fit runs on a plan of its
    own; requests beyond the whole budget and malformed ones fail alone."""
    huge = wl.from_lists([[i + 1] for i in range(39)] + [[]], [[(0, 1, 0)]] * 40, 1 << 24)
    bad = wl.from_lists([[1], [0]], [[], []], 2)
    good = [wl.structured(40 + k, 8000, 2048) for k in range(4)]
    probe = _native.Server(resident=True, workers=1)
    probe.wait(probe.submit(good[0]))
    one = probe.stats()["bytes_in_use"]  # the device bytes of one cached plan
    probe.close()
    assert one > 0
    budget = int(2.5 * one)  # room for two of the four plans
    srv = _native.Server(hbm_budget_bytes=budget, resident=True, workers=2, keep_states=True)
    ts = [srv.submit(g) for g in good + good[::-1]]
    t_huge, t_bad = srv.submit(huge), srv.submit(bad)
    srv.drain()
    assert srv.wait(t_huge)[0] == _native.E_BUDGET
    assert srv.wait(t_bad)[0] == _native.E_INVALID
    for g, t in zip(good + good[::-1], ts):
        st, _, res = srv.wait(t)
        assert st == 0
        assert_matches_oracle(g, res, oracle.solve(g))
    s = srv.stats()
    assert s["peak_bytes"] <= budget and s["cached_plans"] <= 2
    assert s["cache_misses"] > len(good)  # plans were dropped and rebuilt
    srv.close()


def test_resident_poisson_replay_completes():
    rng = np.random.default_rng(6)
    pool = wl.batch(9, n_cfgs=40)
    n = 300
    idx = rng.integers(0, len(pool), size=n)
    cfgs = [_copy_cfg(pool[i]) for i in idx]
    arrival = np.cumsum(rng.exponential(1e6 / 5000.0, size=n))
    srv = _native.Server(resident=True, workers=8)
    tickets = srv.replay(cfgs, arrival)
    srv.drain()
    for k, (i, t) in enumerate(zip(idx, tickets)):
        st, lat, res = srv.wait(t)
        assert st == 0 and lat > 0.0
        if k % 29 == 0:
            assert_same(res, _native.analyze(pool[i]))
    s = srv.stats()
    assert s["completed"] == n and s["cache_hits"] + s["cache_misses"] == n
    srv.close()
