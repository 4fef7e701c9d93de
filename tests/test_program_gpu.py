"""Interprocedural analysis on the GPU (ompdart_summarize_* and
ompdart_analyze_program, Sec. IV-C): callee summaries, the contexts each
function is analysed in and every (function, context) result equal the
reference driver run on the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import program as refprog
from paper_2406_13881_b300 import _native, workload as wl
from compare import assert_matches_oracle
from test_calls_gpu import structured_with_calls
from test_oracle_calls import random_call_row

pytestmark = pytest.mark.gpu


def small_program(seed, n_funcs=30):
    return wl.call_graph(seed, n_funcs=n_funcs, max_depth=4, blocks=(8, 120), median_blocks=30, n_globals=70,
                         max_formals=3)


@pytest.mark.parametrize("seed", range(6))
def test_summaries_equal_oracle(seed):
    rng = np.random.default_rng(600 + seed)
    cfgs = []
    for i in range(12):
        if i % 3 == 2:
            cfgs.append(wl.random_graph(None, int(rng.integers(1, 30)), int(rng.choice([5, 64, 130])), rng=rng))
        else:
            cfgs.append(structured_with_calls(700 + 13 * seed + i, int(rng.integers(5, 300)),
                                              int(rng.choice([5, 64, 130]))))
    sums, st = _native.summarize_batch(cfgs)
    assert (st == 0).all()
    for g, s in zip(cfgs, sums):
        np.testing.assert_array_equal(s, oracle.summarize(g))


def test_summarize_callee_maps_into_the_caller():
    rng = np.random.default_rng(3)
    g = structured_with_calls(901, 200, 70)
    vm = rng.integers(-1, 40, size=70).astype(np.int32)  # aliases and locals
    row = _native.summarize_callee(g, vm, 40)
    want = refprog.map_summary(oracle.summarize(g), 70, vm, 40)
    np.testing.assert_array_equal(row, want)


@pytest.mark.parametrize("max_contexts", [4, 1])
@pytest.mark.parametrize("seed", range(4))
def test_program_equals_reference(seed, max_contexts):
    p = small_program(40 + seed)
    got = _native.analyze_program(p.funcs, p.site_off, p.site_callee, p.var_maps, max_contexts=max_contexts,
                                  keep_states=True)
    ref_sum, ref_res, H = refprog.reference_program(p, max_contexts)
    np.testing.assert_array_equal(got["height"], H)
    for f in range(len(p.funcs)):
        np.testing.assert_array_equal(got["summaries"][f], ref_sum[f], err_msg="summary of %d" % f)
    keys = {(f, refprog.ctx_key(ctx)) for f, ctx, _, _ in got["instances"]}
    assert keys == set(ref_res), (len(keys), len(ref_res))
    for f, ctx, st, res in got["instances"]:
        assert st == 0
        cfg, orc = ref_res[(f, refprog.ctx_key(ctx))]
        assert_matches_oracle(cfg, res, orc)


def test_recursion_rejected():
    p = small_program(50, n_funcs=6)
    if len(p.site_callee) == 0:
        pytest.skip("no call sites drawn")
    sc = p.site_callee.copy()
    caller = int(np.searchsorted(p.site_off, 0, side="right") - 1)
    sc[0] = caller  # the first site calls its own function
    vm = list(p.var_maps)
    vm[0] = np.arange(p.funcs[caller].n_vars, dtype=np.int32)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.analyze_program(p.funcs, p.site_off, sc, vm)
    assert ei.value.code == _native.E_INVALID


@pytest.mark.slow
def test_paper_shaped_program_sampled():
    """The 2,000-function call graph (512 globals, depth 8): every summary
    and every instance of a sample of functions against the reference."""
    p = wl.call_graph(4)
    got = _native.analyze_program(p.funcs, p.site_off, p.site_callee, p.var_maps)
    ref_sum, ref_res, H = refprog.reference_program(p)
    for f in range(len(p.funcs)):
        np.testing.assert_array_equal(got["summaries"][f], ref_sum[f])
    assert {(f, refprog.ctx_key(c)) for f, c, _, _ in got["instances"]} == set(ref_res)
    for f, ctx, st, res in got["instances"][::37]:
        cfg, orc = ref_res[(f, refprog.ctx_key(ctx))]
        assert_matches_oracle(cfg, res, orc)
