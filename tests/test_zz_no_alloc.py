"""ompdart_liveness_noalloc: the liveness pass for callers that cannot
allocate device memory (their memory is owned by another runtime or an
application pool, or they must avoid the implicit synchronisation of
cudaMalloc/cudaFree).  The entry point keeps its scratch in a static
device array; this test allocates the inputs and the output itself and
checks the result against the CPU oracle's liveness and against the
ordinary entry point (ompdart_analyze with keep_states, which reports the
same plane), on two calls in a row.  It also runs a chain whose block ids
count down from the entry, the device-side rejections of malformed inputs
(each followed by a good call, which must not see the failed call's
status), and checks that calls allocate no device memory.

The file sorts last on purpose: a failure here leaves every other GPU test
already run."""
import time

import numpy as np
import pytest

import oracle
from paper_2406_13881_b300 import _native, workload as wl

pytestmark = pytest.mark.gpu


def _on_device(a):
    import torch
    a = np.ascontiguousarray(a)
    view = a.view(np.int64) if a.dtype.itemsize == 8 else a.view(np.int32)
    return torch.from_numpy(view.copy()).cuda()


def _device_inputs(g):
    keep = [_on_device(g.succ_off), _on_device(g.succ if len(g.succ) else np.zeros(1, np.int32)),
            _on_device(g.acc_off), _on_device(g.acc if len(g.acc) else np.zeros(1, np.uint32))]
    xl = None if g.exit_host_live is None else _on_device(np.asarray(g.exit_host_live, np.uint64))
    return keep, xl


def _call(g, keep, xl, out):
    import torch
    _native.liveness_noalloc(g.n_blocks, g.n_vars, g.entry, *(t.data_ptr() for t in keep),
                             None if xl is None else xl.data_ptr(), out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)


def _noalloc_live(g):
    import torch
    keep, xl = _device_inputs(g)
    out = torch.full((g.n_blocks * g.W,), -1, dtype=torch.int64, device="cuda")  # garbage in
    _call(g, keep, xl, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64).reshape(g.n_blocks, g.W)


def _oracle_live(g):
    oracle.build()
    return oracle.solve(g, want=["live_in"])["live_in"].reshape(g.n_blocks, g.W)


def _cases():
    rng = np.random.default_rng(77)
    yield wl.single_small(1)
    yield wl.structured(31, 3000, 300, acc_min=1, acc_max=12)
    g = wl.random_graph(None, 40, 130, max_out=3, acc_max=6, rng=rng)  # irreducible, unreachable blocks
    g.exit_host_live = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
    yield g
    yield wl.structured(32, 20000, 4096, acc_min=1, acc_max=16)


def _countdown_chain(n, n_vars, seed):
    """Blocks n-1 -> n-2 -> ... -> 0, entry n-1: block ids run against the
    flow, the worst numbering for sweeps in block order."""
    rng = np.random.default_rng(seed)
    succs = [[b - 1] if b else [] for b in range(n)]
    accs = []
    for _ in range(n):
        k = int(rng.integers(0, 4))
        accs.append(list(zip(rng.integers(0, n_vars, k).tolist(), rng.integers(1, 4, k).tolist(),
                             rng.integers(0, 2, k).tolist())))
    return wl.from_lists(succs, accs, n_vars, entry=n - 1)


def test_noalloc_liveness_matches_oracle_and_analyze_on_two_calls_in_a_row():
    for g in _cases():
        orc = _oracle_live(g)
        ref = _native.analyze(g, keep_states=True)["live_in"].reshape(g.n_blocks, g.W)
        np.testing.assert_array_equal(ref, orc)
        first = _noalloc_live(g)
        second = _noalloc_live(g)
        np.testing.assert_array_equal(first, orc)
        np.testing.assert_array_equal(second, orc)


def test_noalloc_countdown_chain_of_the_maximum_size():
    g = _countdown_chain(65536, 200, 5)
    orc = _oracle_live(g)
    t0 = time.perf_counter()
    got = _noalloc_live(g)
    assert time.perf_counter() - t0 < 15.0
    np.testing.assert_array_equal(got, orc)


def _bad_variants(g):
    su = np.array(g.succ, dtype=np.int32, copy=True)
    su[0] = g.n_blocks + 5  # successor id out of range
    yield "successor id", wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off, su, g.acc_off, g.acc)
    su = np.array(g.succ, dtype=np.int32, copy=True)
    su[len(su) // 2] = g.entry  # an edge into the entry
    yield "edge into the entry", wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off, su, g.acc_off, g.acc)
    acc = np.array(g.acc, dtype=np.uint32, copy=True)
    acc[len(acc) // 3] |= np.uint32(1 << 31)  # a call pseudo-access
    yield "call pseudo-access", wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off, g.succ, g.acc_off, acc)


def test_noalloc_device_side_rejections_then_a_good_call():
    g = wl.structured(33, 500, 200, acc_min=1, acc_max=6)
    orc = _oracle_live(g)
    for what, bad in _bad_variants(g):
        with pytest.raises(_native.OmpdartError) as ei:
            _noalloc_live(bad)
        assert ei.value.code == _native.E_INVALID, what
        np.testing.assert_array_equal(_noalloc_live(g), orc)


def test_noalloc_calls_allocate_no_device_memory():
    import torch
    g = wl.structured(34, 4000, 1000, acc_min=1, acc_max=8)
    keep, xl = _device_inputs(g)
    out = torch.empty((g.n_blocks * g.W,), dtype=torch.int64, device="cuda")
    _call(g, keep, xl, out)  # the first call on the device looks up the scratch array
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _call(g, keep, xl, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint64).reshape(g.n_blocks, g.W), _oracle_live(g))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    with pytest.raises(_native.OmpdartError) as ei:
        _native.liveness_noalloc(70000, 64, 0, 1, 1, 1, 1, None, 1)
    assert ei.value.code == _native.E_BUDGET and "65536" in str(ei.value)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.liveness_noalloc(10, 5000, 0, 1, 1, 1, 1, None, 1)
    assert ei.value.code == _native.E_BUDGET and "4096" in str(ei.value)
