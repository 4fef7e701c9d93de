"""Pins of the data-region mode of the oracle and of the directive
classification (``oracle/classify.py``; Table II, Sec. IV-D's single target
data region, Sec. IV-F's one directive per insertion point):

* the paper's listings give the constructs its prose names (fixtures in
  tests/golden/paper_listings.json, each with its citation);
* one hand-made program per Table II construct (map to / from / tofrom /
  alloc, update to / from) gets that construct;
* the region R holds every kernel block and every loop whose body holds
  one, and on structured programs it is entered through one block and left
  into one block;
* region mode: replaying every walk with the emitted transfers reads no
  stale value and copies none, no transfer of device data lies outside R,
  and each transfer is needed (deleting any one breaks a walk);
* the classified program -- map clauses at R's boundary, lifted kernel
  `to's, consolidated updates -- replayed on every walk reads no stale
  value and copies none;
* planted mistakes in copies of the classifier fail these.
"""
import numpy as np
import pytest

import listings
import oracle
import refsim as rs
from oracle import classify as C
from paper_2406_13881_b300 import workload as wl

R, W_, RW = wl.KIND_R, wl.KIND_W, wl.KIND_RW
HOST, DEV = 0, 1


def solve_r(g):
    return oracle.solve(g, data_region=True)


# --------------------------------------------------------------------------
# the paper's listings
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["listing1", "listing2", "listing3"])
def test_listings_classified(name):
    case = listings.load()[name]
    ex = case["classified"]
    g, vid = listings.to_cfg(case)
    res = solve_r(g)
    c = C.classify(g, res)
    assert sorted(np.flatnonzero(c["in_region"]).tolist()) == ex["region_blocks"]
    for v, want in ex["map"].items():
        assert C.construct_of(c, vid[v]) == want, (v, C.construct_of(c, vid[v]))
    assert not c["kernel_to"].any()
    n_updates = c["n_directives"] - 1  # minus the target data construct
    assert n_updates == ex["updates"]
    for s, t, v in ex.get("update_from_edges", []):
        e = [i for i in range(int(g.succ_off[s]), int(g.succ_off[s + 1])) if int(g.succ[i]) == t][0]
        assert (int(c["edge_from"][e, vid[v] >> 6]) >> (vid[v] & 63)) & 1


def test_listing5_without_kernels_has_no_region():
    case = listings.load()["listing5"]
    g, vid = listings.to_cfg(case)
    c = C.classify(g, solve_r(g))
    assert not c["in_region"].any() and c["n_directives"] == 1  # the update from before the loop
    assert (int(c["edge_from"][0, 0]) >> vid["partial_sum"]) & 1


# --------------------------------------------------------------------------
# Table II, one construct per program
# --------------------------------------------------------------------------

def chain(blocks, nv, region, **kw):
    succs = [[i + 1] for i in range(len(blocks) - 1)] + [[]]
    return wl.from_lists(succs, blocks, nv, region=region, **kw)


TABLE2 = {
    # map(to:): the kernel reads data the host wrote; nothing changes it after
    "to": (chain([[(0, W_, HOST)], [(0, R, DEV)], []], 1, [-1, 0, -1]), {0: "to"}, 0),
    # map(from:): the kernel writes data the host reads afterwards
    "from": (chain([[], [(0, W_, DEV)], [(0, R, HOST)]], 1, [-1, 0, -1]), {0: "from"}, 0),
    # map(tofrom:): read and written on the device, live afterwards
    "tofrom": (chain([[(0, W_, HOST)], [(0, RW, DEV)], []], 1, [-1, 0, -1]), {0: "tofrom"}, 0),
    # map(alloc:): a device temporary, dead after the region
    "alloc": (chain([[], [(0, W_, DEV), (0, R, DEV)], []], 1, [-1, 0, -1],
                    exit_host_live=np.zeros(1, np.uint64)), {0: "alloc"}, 0),
    # update to: the host writes between two kernels that read
    "update_to": (chain([[(0, W_, HOST)], [(0, R, DEV)], [(0, W_, HOST)], [(0, R, DEV)], []], 1,
                        [-1, 0, -1, 1, -1]), {0: "to"}, 1),
    # update from: the host reads between two kernels what the first wrote;
    # w: written by the second kernel, live after
    "update_from": (chain([[], [(0, W_, DEV)], [(0, R, HOST)], [(0, R, DEV), (1, W_, DEV)], []], 2,
                          [-1, 0, -1, 1, -1]), {0: "alloc", 1: "from"}, 1),
}


@pytest.mark.parametrize("name", sorted(TABLE2))
def test_table2_construct(name):
    g, want, n_upd = TABLE2[name]
    c = C.classify(g, solve_r(g))
    for v, k in want.items():
        assert C.construct_of(c, v) == k, (v, C.construct_of(c, v))
    assert c["n_directives"] - 1 == n_upd
    if name == "update_to":
        assert c["kernel_to"][1, 0] == 1 and not c["kernel_to"][0].any()
    if name == "update_from":
        pts = np.flatnonzero(c["acc_point"] >= 0)
        assert len(pts) == 1 and int(g.acc_off[2]) == int(pts[0])


# --------------------------------------------------------------------------
# the region
# --------------------------------------------------------------------------

def kernel_cfg(seed, n, nv, **kw):
    return wl.structured(seed, n, nv, p_if_then=0.2, p_if_else=0.15, p_while=0.12, max_loop_depth=2,
                         region_mode="count", n_regions=int(np.random.default_rng(seed).integers(1, 4)),
                         target_frac=0.3, acc_min=0, acc_max=3, var_dist="uniform", **kw)


def loops_of(g, res):
    """(header, body set) of every natural loop, found by dominance by
    removal (a dominates b iff b is unreachable once a is removed)."""
    n = g.n_blocks
    succ = [list(map(int, g.succ[g.succ_off[b]:g.succ_off[b + 1]])) for b in range(n)]

    def reach_without(x):
        seen = {g.entry} if g.entry != x else set()
        st = list(seen)
        while st:
            b = st.pop()
            for t in succ[b]:
                if t != x and t not in seen:
                    seen.add(t)
                    st.append(t)
        return seen

    rs_ = {x: reach_without(x) for x in range(n)}
    reach = res["reachable"].astype(bool)
    out = []
    for h in range(n):
        latches = [t for t in range(n) if reach[t] and h in succ[t] and (t == h or t not in rs_[h])]
        if not latches or not reach[h]:
            continue
        body = {h}
        st = [t for t in latches if t != h]
        body |= set(st)
        pred = [[p for p in range(n) if b in succ[p] and reach[p]] for b in range(n)]
        while st:
            b = st.pop()
            for p in pred[b]:
                if p not in body:
                    body.add(p)
                    st.append(p)
        out.append((h, body))
    return out


@pytest.mark.parametrize("seed", range(40))
def test_region_holds_kernels_and_capturing_loops_and_is_sese(seed):
    g = kernel_cfg(300 + seed, int(12 + seed % 30), 3)
    res = solve_r(g)
    inr = res["in_region"].astype(bool)
    ker = (np.asarray(g.region) >= 0) & res["reachable"].astype(bool)
    if not ker.any():
        assert not inr.any()
        return
    assert inr[ker].all()
    for h, body in loops_of(g, res):
        if any(ker[b] for b in body):
            assert all(inr[b] for b in body), (h, sorted(body))
    c = C.classify(g, res)
    tgt_in = {int(g.succ[e]) for e in c["region_entry_edges"]}
    tgt_out = {int(g.succ[e]) for e in c["region_exit_edges"]}
    assert len(tgt_in) <= 1 and len(tgt_out) <= 1


# --------------------------------------------------------------------------
# region mode by path simulation
# --------------------------------------------------------------------------

def _top(n):
    return (1 << n) - 1


def _region_sim(g, check_irredundant):
    res = solve_r(g)
    t = rs.transfers_from_oracle(g, res)
    hoist = [e for e in range(g.n_edges) if res["is_loop_entry"][e]]
    walks = rs.maximal_walks(g, g.entry, 2)
    sim = rs.PathSim(g, t, _top(g.n_vars), 0, _top(g.n_vars), hoist)
    for blocks, edges in walks:
        sim.run(blocks, edges)
    # no transfer of device data outside the region: edges with both ends
    # outside, flags and exit sets of blocks outside
    inr = res["in_region"].astype(bool)
    for e, x in list(t["to_edge"].items()) + list(t["from_edge"].items()):
        src = int(np.searchsorted(g.succ_off, e, side="right") - 1)
        assert inr[src] or inr[int(g.succ[e])], ("edge", e)
    blk = np.repeat(np.arange(g.n_blocks), np.diff(g.acc_off))
    for i in t["flag"]:
        assert inr[blk[i]], ("flag", i)
    for b in t["from_exit"]:
        assert inr[b], ("exit", b)
    if check_irredundant and walks:
        for desc, u in rs.each_single_removal(t):
            s2 = rs.PathSim(g, u, _top(g.n_vars), 0, _top(g.n_vars), hoist)
            broke = False
            for blocks, edges in walks:
                try:
                    s2.run(blocks, edges)
                except rs.Violation:
                    broke = True
                    break
            assert broke, "redundant transfer: " + desc
    return res


@pytest.mark.parametrize("seed", range(40))
def test_region_mode_paths(seed):
    g = kernel_cfg(400 + seed, int(8 + seed % 14), 3)
    _region_sim(g, check_irredundant=seed % 2 == 0)


@pytest.mark.parametrize("seed", range(30))
def test_region_mode_random_graphs(seed):
    rng = np.random.default_rng(500 + seed)
    g = wl.random_graph(None, int(rng.integers(2, 7)), int(rng.integers(1, 4)), max_out=2, acc_max=3, rng=rng)
    # kernels: every block with a device access (device code runs only in kernels)
    var, kind, space = wl.unpack_access(g.acc)
    reg = np.full(g.n_blocks, -1, np.int32)
    k = 0
    for b in range(g.n_blocks):
        if (space[g.acc_off[b]:g.acc_off[b + 1]] == 1).any():
            reg[b] = k
            k += 1
    g.region = reg
    _region_sim(g, check_irredundant=False)


# --------------------------------------------------------------------------
# the classified program by path simulation
# --------------------------------------------------------------------------

def _bits(x):
    x = int(np.uint64(x))
    v = 0
    while x:
        if x & 1:
            yield v
        x >>= 1
        v += 1


def classified_transfers(g, res, c):
    """The directives of a classification as transfers for PathSim."""
    t = {"to_edge": {}, "from_edge": {}, "flag": {}, "from_exit": {}, "pre": {}, "start": []}
    mt, mf = rs.word(c["map_to"][0]), rs.word(c["map_from"][0])
    for e in c["region_entry_edges"]:
        t["to_edge"][e] = t["to_edge"].get(e, 0) | mt
    if c["in_region"][g.entry]:
        t["start"] += [("to", v) for v in _bits(mt)]
    for e in c["region_exit_edges"]:
        t["from_edge"][e] = t["from_edge"].get(e, 0) | mf
    reach = res["reachable"].astype(bool)
    for b in range(g.n_blocks):
        if reach[b] and c["in_region"][b] and g.succ_off[b] == g.succ_off[b + 1]:
            t["from_exit"][b] = t["from_exit"].get(b, 0) | mf
    region = np.asarray(g.region)
    # right before kernel k: after whatever the edge entering it carries
    t["edge_post"] = {}
    for key, kind in (("kernel_from", "from"), ("kernel_to", "to")):
        for k in range(c[key].shape[0]):
            x = rs.word(c[key][k, 0])
            if not x:
                continue
            for b in range(g.n_blocks):
                for e in range(int(g.succ_off[b]), int(g.succ_off[b + 1])):
                    if region[int(g.succ[e])] == k and region[b] != k and reach[b]:
                        t["edge_post"].setdefault(e, []).extend((kind, v) for v in _bits(x))
            if region[g.entry] == k:
                t["start"] += [(kind, v) for v in _bits(x)]
    for e in range(g.n_edges):
        if c["edge_to"][e, 0]:
            t["to_edge"][e] = t["to_edge"].get(e, 0) | rs.word(c["edge_to"][e, 0])
        if c["edge_from"][e, 0]:
            t["from_edge"][e] = t["from_edge"].get(e, 0) | rs.word(c["edge_from"][e, 0])
    for b in range(g.n_blocks):
        if c["exit_from"][b, 0]:
            t["from_exit"][b] = t["from_exit"].get(b, 0) | rs.word(c["exit_from"][b, 0])
    var, _, _ = wl.unpack_access(g.acc)
    for i in np.flatnonzero(c["acc_point"] >= 0):
        f = int(res["acc_flag"][i])
        kind = "to" if f == 1 else "from"
        t["pre"].setdefault(int(c["acc_point"][i]), []).append((kind, int(var[i])))
    return t


def _classified_sim(g, classify=C.classify):
    res = solve_r(g)
    c = classify(g, res)
    t = classified_transfers(g, res, c)
    sim = rs.PathSim(g, t, _top(g.n_vars), 0, _top(g.n_vars))
    for blocks, edges in rs.maximal_walks(g, g.entry, 2):
        sim.run(blocks, edges)
    return c


@pytest.mark.parametrize("seed", range(60))
def test_classified_program_paths(seed):
    g = kernel_cfg(600 + seed, int(8 + seed % 20), int(1 + seed % 4))
    _classified_sim(g)


def mixed_kernel_graph(seed):
    """A random graph whose blocks with a device access are kernels (so
    kernel blocks may also hold host accesses)."""
    rng = np.random.default_rng(seed)
    g = wl.random_graph(None, int(rng.integers(2, 7)), int(rng.integers(1, 4)), max_out=2, acc_max=4, rng=rng)
    var, kind, space = wl.unpack_access(g.acc)
    reg = np.full(g.n_blocks, -1, np.int32)
    k = 0
    for b in range(g.n_blocks):
        if (space[g.acc_off[b]:g.acc_off[b + 1]] == 1).any():
            reg[b] = k
            k += 1
    g.region = reg
    return g


@pytest.mark.parametrize("seed", range(60))
def test_classified_program_paths_mixed_blocks(seed):
    _classified_sim(mixed_kernel_graph(1000 + seed))


def test_consolidation_merges_host_reads_of_one_block():
    # kernel writes a, b; the host then reads a, c, b in one block: both
    # `from's move to the block's start -- one directive
    g = chain([[], [(0, W_, DEV), (1, W_, DEV)], [(0, R, HOST), (2, R, HOST), (1, R, HOST)], [(0, R, DEV)], []],
              3, [-1, 0, -1, 1, -1])
    c = _classified_sim(g)
    pts = c["acc_point"][c["acc_point"] >= 0]
    assert len(pts) == 2 and len(set(pts.tolist())) == 1 and int(pts[0]) == int(g.acc_off[2])


# --------------------------------------------------------------------------
# planted mistakes
# --------------------------------------------------------------------------

def _plant(mutate):
    def bad(g, res):
        c = C.classify(g, res)
        mutate(g, res, c)
        return c
    return bad


def _no_uniform_from(g, res, c):
    # map(from:) from the first exit edge alone, not every way out
    if c["region_exit_edges"]:
        c["map_from"] |= res["from_edge"][c["region_exit_edges"][0]]


def _consolidate_past_same_var(g, res, c):
    # move every access transfer to its block's start, even past accesses
    # of the same variable
    blk = np.repeat(np.arange(g.n_blocks), np.diff(g.acc_off))
    for i in np.flatnonzero(c["acc_point"] >= 0):
        c["acc_point"][i] = int(g.acc_off[blk[i]])


def _lift_past_writes(g, res, c):
    # move every `to' inside a kernel before it, even past a host write of
    # the same variable in that kernel
    blk = np.repeat(np.arange(g.n_blocks), np.diff(g.acc_off))
    region = np.asarray(g.region)
    var, _, _ = wl.unpack_access(g.acc)
    for i in np.flatnonzero(c["acc_point"] >= 0):
        k = int(region[blk[i]])
        if k >= 0 and int(res["acc_flag"][i]) == 1:
            v = int(var[i])
            c["kernel_to"][k, v >> 6] |= np.uint64(1) << np.uint64(v & 63)
            c["acc_point"][i] = -1


def test_planted_classifier_mistakes_fail():
    for mut in (_no_uniform_from, _consolidate_past_same_var, _lift_past_writes):
        caught = False
        for seed in range(600, 900):
            g = kernel_cfg(seed, int(8 + seed % 20), int(1 + seed % 4)) if seed % 2 else mixed_kernel_graph(seed)
            try:
                _classified_sim(g, _plant(mut))
            except rs.Violation:
                caught = True
                break
        assert caught, mut.__name__


# --------------------------------------------------------------------------
# firstprivate (Sec. IV-D, scalar paragraph)
# --------------------------------------------------------------------------

def test_read_only_scalar_gets_firstprivate_and_no_to():
    # kernel 0 reads scalar s (0) and array a (1); the host wrote both
    g = chain([[(0, W_, HOST), (1, W_, HOST)], [(0, R, DEV), (1, R, DEV)], []], 2, [-1, 0, -1])
    c = C.classify(g, solve_r(g))
    assert C.construct_of(c, 0) == "to" and C.construct_of(c, 1) == "to"
    g2, fp = C.firstprivate_view(g, wl.var_mask(2, [0]))
    assert fp[0, 0] == 1
    c2 = C.classify(g2, solve_r(g2))
    assert C.construct_of(c2, 0) is None and C.construct_of(c2, 1) == "to"
    assert not c2["kernel_to"].any() and not c2["kernel_from"].any()


def test_scalar_written_by_a_kernel_is_not_firstprivate_there():
    # kernel 0 writes s; kernel 1 reads it: firstprivate on kernel 1 only,
    # after an update from before it (the host copy is the private copy's source)
    g = chain([[], [(0, W_, DEV)], [(0, R, DEV)], []], 1, [-1, 0, 1, -1], exit_host_live=np.zeros(1, np.uint64))
    g2, fp = C.firstprivate_view(g, wl.var_mask(1, [0]))
    assert fp[0, 0] == 0 and fp[1, 0] == 1
    c2 = _classified_sim(g2)
    assert c2["kernel_from"][1, 0] == 1


@pytest.mark.parametrize("seed", range(40))
def test_firstprivate_programs_paths(seed):
    g = kernel_cfg(900 + seed, int(8 + seed % 20), int(1 + seed % 4))
    rng = np.random.default_rng(seed)
    scal = wl.var_mask(g.n_vars, [v for v in range(g.n_vars) if rng.random() < 0.5])
    g2, fp = C.firstprivate_view(g, scal)
    c = _classified_sim(g2)
    # a firstprivate scalar of kernel k has no `to' of its own before k
    for k in range(fp.shape[0]):
        assert not (fp[k] & c["kernel_to"][k]).any()
