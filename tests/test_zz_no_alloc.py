"""ompdart_liveness_noalloc: the liveness pass for callers that cannot
allocate device memory (their memory is owned by another runtime or an
application pool, or they must avoid the implicit synchronisation of
cudaMalloc/cudaFree).  The entry point keeps its scratch in a static
device array; this test allocates the inputs and the output itself and
checks the result against the ordinary entry point (ompdart_analyze with
keep_states, which reports the same liveness plane), on two calls in a row.

The file sorts last on purpose: a failure here leaves every other GPU test
already run."""
import numpy as np
import pytest

from paper_2406_13881_b300 import _native, workload as wl

pytestmark = pytest.mark.gpu


def _on_device(a):
    import torch
    a = np.ascontiguousarray(a)
    view = a.view(np.int64) if a.dtype.itemsize == 8 else a.view(np.int32)
    return torch.from_numpy(view.copy()).cuda()


def _noalloc_live(g):
    import torch
    keep = [_on_device(g.succ_off), _on_device(g.succ if len(g.succ) else np.zeros(1, np.int32)),
            _on_device(g.acc_off), _on_device(g.acc if len(g.acc) else np.zeros(1, np.uint32))]
    xl = None if g.exit_host_live is None else _on_device(np.asarray(g.exit_host_live, np.uint64))
    out = torch.full((g.n_blocks * g.W,), -1, dtype=torch.int64, device="cuda")  # garbage in
    _native.liveness_noalloc(g.n_blocks, g.n_vars, g.entry, *(t.data_ptr() for t in keep),
                             None if xl is None else xl.data_ptr(), out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64).reshape(g.n_blocks, g.W)


def _cases():
    rng = np.random.default_rng(77)
    yield wl.single_small(1)
    yield wl.structured(31, 3000, 300, acc_min=1, acc_max=12)
    g = wl.random_graph(None, 40, 130, max_out=3, acc_max=6, rng=rng)  # irreducible, unreachable blocks
    g.exit_host_live = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
    yield g
    yield wl.structured(32, 20000, 4096, acc_min=1, acc_max=16)


def test_noalloc_liveness_matches_analyze_on_two_calls_in_a_row():
    for g in _cases():
        ref = _native.analyze(g, keep_states=True)["live_in"]
        first = _noalloc_live(g)
        second = _noalloc_live(g)
        np.testing.assert_array_equal(first, ref)
        np.testing.assert_array_equal(second, ref)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    with pytest.raises(_native.OmpdartError) as ei:
        _native.liveness_noalloc(70000, 64, 0, 1, 1, 1, 1, None, 1)
    assert ei.value.code == _native.E_BUDGET and "65536" in str(ei.value)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.liveness_noalloc(10, 5000, 0, 1, 1, 1, 1, None, 1)
    assert ei.value.code == _native.E_BUDGET and "4096" in str(ei.value)
