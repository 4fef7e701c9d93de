"""Data-region mode, directive classification and firstprivate on the GPU
(opts.data_region; Table II, Sec. IV-D single target data region and
scalar paragraph, Sec. IV-F consolidation): every output of the C ABI --
the analysis with the region-exit rule and the directives -- equals the
oracle (``oracle.solve(..., data_region=True)`` and ``oracle/classify.py``)
bit for bit, on the paper's listings, one program per Table II construct,
small and paper-shaped CFGs (chunked scan and sweep solvers), batches of
many CFGs, and word columns of the 2^20-block CFG."""
import numpy as np
import pytest

import listings
import oracle
from compare import assert_matches_oracle
from oracle import classify as C
from paper_2406_13881_b300 import _native, workload as wl
from test_oracle_classify import TABLE2, kernel_cfg, mixed_kernel_graph

pytestmark = pytest.mark.gpu


def oracle_side(g, scalars=None):
    """(cfg the analysis sees, oracle result, classification, firstprivate rows)."""
    fp = None
    if scalars is not None:
        g2, fp = C.firstprivate_view(g, scalars)
    else:
        g2 = g
    res = oracle.solve(g2, data_region=True)
    return g2, res, C.classify(g2, res), fp


def assert_directives(g, got, orc_cfg, res, cls, fp=None, words=None, acc_keep=None):
    cols = slice(None) if words is None else words
    np.testing.assert_array_equal(got["in_region"], cls["in_region"], err_msg="in_region")
    for k in ("map_to", "map_from", "map_alloc"):
        np.testing.assert_array_equal(got[k][cols], cls[k], err_msg=k)
    for k in ("kernel_to", "kernel_from"):
        np.testing.assert_array_equal(got[k][:, cols], cls[k], err_msg=k)
    if fp is not None:
        np.testing.assert_array_equal(got["firstprivate"][:, cols], fp, err_msg="firstprivate")
    pts = got["acc_point"] if acc_keep is None else got["acc_point"][acc_keep]
    if acc_keep is not None:
        # a point of the full CFG (an access index) is, in the column's own
        # numbering, the first access of the column at or after it (the
        # accesses it moved past belong to other columns)
        keep = np.asarray(acc_keep)
        pts = np.where(pts >= 0, np.searchsorted(keep, np.maximum(pts, 0)), -1)
    np.testing.assert_array_equal(pts, cls["acc_point"], err_msg="acc_point")
    assert sorted(got["region_entry_edges"].tolist()) == cls["region_entry_edges"]
    assert sorted(got["region_exit_edges"].tolist()) == cls["region_exit_edges"]


def check(g, scalars=None, **opts):
    gs = g if scalars is None else _with_scalars(g, scalars)
    orc_cfg, res, cls, fp = oracle_side(g, scalars)
    got = _native.analyze(gs, data_region=True, keep_states=True, **opts)
    assert_matches_oracle(orc_cfg, got, res)
    assert_directives(g, got, orc_cfg, res, cls, fp)
    return got


def _with_scalars(g, scalars):
    h = wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off, g.succ, g.acc_off, g.acc, g.region,
               g.entry_host_valid, g.entry_dev_valid, g.exit_host_live, g.call_planes)
    h.scalar_vars = np.asarray(scalars, np.uint64)
    return h


@pytest.mark.parametrize("name", ["listing1", "listing2", "listing3", "listing5"])
def test_listings(name):
    g, _ = listings.to_cfg(listings.load()[name])
    for path in (1, 2):
        check(g, path=path)


@pytest.mark.parametrize("name", sorted(TABLE2))
def test_table2_constructs(name):
    g = TABLE2[name][0]
    for path in (1, 2):
        check(g, path=path)


@pytest.mark.parametrize("seed", range(24))
def test_small_structured(seed):
    g = kernel_cfg(1200 + seed, int(10 + seed % 40), int(1 + seed % 130))
    for target in (0, 1, 3):
        check(g, path=2, chunk_target=target)
    check(g, path=1)


@pytest.mark.parametrize("seed", range(24))
def test_mixed_blocks_and_irreducible(seed):
    g = mixed_kernel_graph(1300 + seed)
    check(g)  # the library's choice (sweep for irreducible graphs)


@pytest.mark.parametrize("seed", range(16))
def test_firstprivate(seed):
    g = kernel_cfg(1400 + seed, int(10 + seed % 40), int(2 + seed % 70))
    rng = np.random.default_rng(seed)
    scal = wl.var_mask(g.n_vars, [v for v in range(g.n_vars) if rng.random() < 0.5])
    check(g, scal, path=2)
    check(g, scal, path=1)


def test_paper_shaped_small_cfgs():
    """Config-1 shape: 64 blocks, a 2-deep loop nest around a kernel, 3 kernel ranges."""
    for seed in range(1, 6):
        check(wl.single_small(seed))


def test_batch_with_regions_and_firstprivate():
    """Config-3-shaped CFGs (lognormal sizes, 64-2048 variables) in one
    batch, some with scalars, one without kernel information: each equals
    the oracle and the same CFG alone."""
    cfgs = wl.batch(3, n_cfgs=60)
    rng = np.random.default_rng(9)
    scal = []
    for i, g in enumerate(cfgs):
        if i % 3 == 0:
            s = wl.var_mask(g.n_vars, [v for v in range(g.n_vars) if rng.random() < 0.2])
            cfgs[i] = _with_scalars(g, s)
            scal.append(s)
        else:
            scal.append(None)
    cfgs[5].region = None  # no kernel information: no region, consolidation only
    b = _native.Batch(cfgs, data_region=True, keep_states=True)
    b.run()
    assert (b.sync() == 0).all()
    for i, g in enumerate(cfgs):
        got = b.fetch(i)
        base = wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off, g.succ, g.acc_off, g.acc, g.region)
        if g.region is None:
            assert not got["in_region"].any() and got["kernel_to"].shape[0] == 0
        orc_cfg, res, cls, fp = oracle_side(base, scal[i])
        assert_matches_oracle(orc_cfg, got, res)
        assert_directives(base, got, orc_cfg, res, cls, fp)
    b.close()


@pytest.mark.slow
def test_large_cfg_word_columns():
    """The 2^20-block, 4096-variable CFG: word columns 0, 37 and 63 of
    every output against the oracle run on exactly those 64 variables (the
    region depends on the graph and the kernels only; every variable is
    its own bit problem)."""
    g = wl.single_large(2)
    p = _native.Plan(g, data_region=True)
    p.run()
    p.sync()
    got = p.fetch()
    p.close()
    for w in (0, 37, 63):
        sub, keep = wl.restrict_word(g, w)
        sub.region = g.region
        orc_cfg, res, cls, _ = oracle_side(sub)
        assert_matches_oracle(orc_cfg, got, res, words=slice(w, w + 1), acc_keep=keep)
        assert_directives(sub, got, orc_cfg, res, cls, words=slice(w, w + 1), acc_keep=keep)
