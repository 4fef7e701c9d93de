"""Loader for tests/golden/paper_listings.json (paper programs in access form)."""
import json
import os

import numpy as np

from paper_2406_13881_b300.workload import KIND_R, KIND_RW, KIND_W, from_lists, var_mask

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_listings.json")
KIND = {"R": KIND_R, "W": KIND_W, "RW": KIND_RW}
SPACE = {"host": 0, "target": 1}


def load():
    with open(PATH) as f:
        d = json.load(f)
    return {k: v for k, v in d.items() if not k.startswith("_")}


def to_cfg(case):
    vars_ = case["vars"]
    vid = {n: i for i, n in enumerate(vars_)}
    succs = [b["succ"] for b in case["blocks"]]
    accs = [[(vid[a[0]], KIND[a[1]], SPACE[a[2]]) for a in b["acc"]] for b in case["blocks"]]
    region = [b.get("region", -1) for b in case["blocks"]]
    kw = {}
    if "entry_host_valid" in case:
        kw["entry_host_valid"] = var_mask(len(vars_), [vid[n] for n in case["entry_host_valid"]])
    if "entry_dev_valid" in case:
        kw["entry_dev_valid"] = var_mask(len(vars_), [vid[n] for n in case["entry_dev_valid"]])
    g = from_lists(succs, accs, len(vars_), region=region, **kw)
    return g, vid


def expected_sets(case, g, vid):
    """Expected transfers as sets: ('to_edge'|'from_edge', edge_id, var),
    ('flag', access_index, 1|2), ('from_exit', block, var)."""
    ex = case["expected"]
    out = set()
    for key in ("to_edge", "from_edge"):
        for s, t, v in ex[key]:
            e = [i for i in range(int(g.succ_off[s]), int(g.succ_off[s + 1])) if int(g.succ[i]) == t]
            assert len(e) == 1
            out.add((key, e[0], vid[v]))
    for b, j, kind in ex["flags"]:
        out.add(("flag", int(g.acc_off[b]) + j, 1 if kind == "to" else 2))
    for b, v in ex["from_exit"]:
        out.add(("from_exit", b, vid[v]))
    return out


def bits(x):
    x = int(np.uint64(x))
    v = 0
    while x:
        if x & 1:
            yield v
        x >>= 1
        v += 1


def oracle_sets(res):
    out = set()
    for key in ("to_edge", "from_edge"):
        a = res[key]
        for e in range(a.shape[0]):
            for w in range(a.shape[1]):
                for v in bits(a[e, w]):
                    out.add((key, e, 64 * w + v))
    for i, f in enumerate(res["acc_flag"]):
        if f:
            out.add(("flag", i, int(f)))
    a = res["from_exit"]
    for b in range(a.shape[0]):
        for w in range(a.shape[1]):
            for v in bits(a[b, w]):
                out.add(("from_exit", b, 64 * w + v))
    return out
