"""CFGs given in device memory (ompdart_cfg.mem = OMPDART_MEM_DEVICE):
torch device tensors passed by address through every entry point that
takes a CFG -- ompdart_analyze, ompdart_plan_create, ompdart_analyze_batch,
ompdart_batch_create, ompdart_server_submit, ompdart_summarize_batch /
ompdart_summarize_callee and ompdart_analyze_program -- give exactly the
oracle's results (and the same results as the host-memory form)."""
import numpy as np
import pytest

import oracle
from compare import assert_matches_oracle
from paper_2406_13881_b300 import _native, workload as wl

pytestmark = pytest.mark.gpu


def _t(a, dt):
    import torch
    a = np.ascontiguousarray(a, dtype=dt)
    view = a.view(np.int64) if a.dtype.itemsize == 8 else a.view(np.int32)
    return torch.from_numpy(view.copy()).cuda()


def to_device(g):
    """The CFG's arrays as device tensors, wrapped as a DeviceCfg."""
    keep = {"so": _t(g.succ_off, np.int32), "s": _t(g.succ if len(g.succ) else np.zeros(1), np.int32),
            "ao": _t(g.acc_off, np.int32), "acc": _t(g.acc if len(g.acc) else np.zeros(1), np.uint32)}
    for k in ("entry_host_valid", "entry_dev_valid", "exit_host_live", "call_planes"):
        v = getattr(g, k)
        keep[k] = None if v is None else _t(np.asarray(v).reshape(-1), np.uint64)
    ptr = lambda k: None if keep[k] is None else keep[k].data_ptr()  # noqa: E731
    n_calls = 0 if g.call_planes is None else int(np.asarray(g.call_planes).size // (7 * g.W))
    return _native.DeviceCfg(g.n_blocks, g.n_vars, g.entry, ptr("so"), ptr("s"), ptr("ao"), ptr("acc"),
                             ptr("entry_host_valid"), ptr("entry_dev_valid"), ptr("exit_host_live"),
                             ptr("call_planes"), n_calls, owner=keep)


def _cases():
    rng = np.random.default_rng(5)
    yield wl.single_small(1)
    yield wl.structured(61, 2000, 200, acc_min=1, acc_max=8)
    g = wl.random_graph(None, 30, 70, max_out=3, acc_max=5, rng=rng)  # irreducible: the sweep solver
    top = wl.var_mask(g.n_vars, range(g.n_vars))
    g.entry_dev_valid = rng.integers(0, 2**63, size=g.W, dtype=np.uint64) & top
    g.exit_host_live = rng.integers(0, 2**63, size=g.W, dtype=np.uint64) & top
    yield g


def test_analyze_and_plan_take_device_inputs():
    for g in _cases():
        orc = oracle.solve(g)
        d = to_device(g)
        assert_matches_oracle(g, _native.analyze(d, keep_states=True), orc)
        p = _native.Plan(d, keep_states=True)
        del d  # the plan copied what it needs
        p.run()
        p.sync()
        assert_matches_oracle(g, p.fetch(), orc)
        p.close()


def test_batch_mixes_host_and_device_cfgs_and_a_bad_one_fails_alone():
    gs = list(_cases()) + [wl.structured(62 + k, 300 + 50 * k, 64 * (k + 1), acc_min=1, acc_max=6)
                           for k in range(4)]
    ins = [to_device(g) if i % 2 == 0 else g for i, g in enumerate(gs)]
    # a "device" CFG whose arrays are host memory: rejected alone
    h = gs[1]
    bad = _native.DeviceCfg(h.n_blocks, h.n_vars, h.entry, h.succ_off.ctypes.data, h.succ.ctypes.data,
                            h.acc_off.ctypes.data, h.acc.ctypes.data)
    res, st = _native.analyze_batch(ins + [bad], keep_states=True)
    assert st[-1] == _native.E_INVALID and res[-1] is None
    for g, r, s in zip(gs, res, st):
        assert s == 0
        assert_matches_oracle(g, r, oracle.solve(g))
    # the same function given twice with the same device arrays and other boundary rows
    g = gs[4]
    d = to_device(g)
    d2 = _native.DeviceCfg(*[getattr(d, k) for k in ("n_blocks", "n_vars", "entry")], *d.ptrs[:4],
                           entry_dev_valid=to_device_row(np.full(g.W, ~np.uint64(0), np.uint64), d),
                           owner=d.owner)
    g2 = wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off, g.succ, g.acc_off, g.acc,
                entry_dev_valid=np.full(g.W, ~np.uint64(0), np.uint64))
    b = _native.Batch([d, d2], keep_states=True)
    b.run()
    assert (b.sync() == 0).all()
    assert_matches_oracle(g, b.fetch(0), oracle.solve(g))
    assert_matches_oracle(g2, b.fetch(1), oracle.solve(g2))
    b.close()


def to_device_row(row, d):
    t = _t(row, np.uint64)
    d.owner["extra_%d" % len(d.owner)] = t
    return t.data_ptr()


def test_server_takes_device_inputs():
    gs = list(_cases())
    srv = _native.Server(max_batch=8, max_inflight=2)
    devs = [to_device(g) for g in gs]
    tickets = [srv.submit(d) for d in devs]
    del devs  # submit copied the arrays
    for g, t in zip(gs, tickets):
        st, _, r = srv.wait(t)
        assert st == 0
        assert_matches_oracle(g, r, oracle.solve(g))
    srv.close()


def test_summaries_and_programs_take_device_inputs():
    gs = [wl.structured(70 + k, 100 + 40 * k, 64 + 32 * k, acc_min=1, acc_max=5) for k in range(3)]
    rows, st = _native.summarize_batch([to_device(g) for g in gs])
    assert (st == 0).all()
    for g, r in zip(gs, rows):
        np.testing.assert_array_equal(r, oracle.summarize(g))
    g = gs[1]
    vm = np.arange(g.n_vars, dtype=np.int32) % 40
    np.testing.assert_array_equal(_native.summarize_callee(to_device(g), vm, 40),
                                  _native.summarize_callee(g, vm, 40))
    p = wl.call_graph(9, n_funcs=12, blocks=(32, 128), median_blocks=48)
    host = _native.analyze_program(p.funcs, p.site_off, p.site_callee, p.var_maps)
    dev = _native.analyze_program([to_device(f) for f in p.funcs], p.site_off, p.site_callee, p.var_maps)
    assert len(host["instances"]) == len(dev["instances"])
    for a, b in zip(host["instances"], dev["instances"]):
        assert a[0] == b[0] and a[2] == b[2] == 0
        for x, y in zip(a[1], b[1]):
            np.testing.assert_array_equal(x, y)
        for k in ("h_in", "d_in", "acc_flag", "from_exit"):
            np.testing.assert_array_equal(a[3][k], b[3][k])
    for x, y in zip(host["summaries"], dev["summaries"]):
        np.testing.assert_array_equal(x, y)


def test_mem_field_is_checked():
    g = wl.single_small(1)
    h = _native.DeviceCfg(g.n_blocks, g.n_vars, g.entry, g.succ_off.ctypes.data, g.succ.ctypes.data,
                          g.acc_off.ctypes.data, g.acc.ctypes.data)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.analyze(h)  # host arrays declared as device memory
    assert ei.value.code == _native.E_INVALID and "not device memory" in str(ei.value)
    inp = _native._Inputs(g)
    inp.c.mem = 7
    res = _native.C.POINTER(_native.Result)()
    rc = _native.load().ompdart_analyze(_native.C.byref(inp.c), _native.C.byref(_native._opts()),
                                        _native.C.byref(res))
    assert rc == _native.E_INVALID
