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
