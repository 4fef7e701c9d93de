"""Independent, deliberately naive references used to pin the oracle.

Nothing here is shared with the oracle (C) or the CUDA library: it restates
the paper's semantics directly and checks results by brute force.

* ``local_sim``      per-block effect by *simulating* validity (Sec. IV-D:
                     a write makes the other space stale, a read needs and
                     then has a valid copy), not by the last-event rule.
* ``mop_*``          meet over all paths on acyclic (or path-bounded) CFGs.
* ``PathSim``        replays concrete paths with per-variable version
                     counters and the emitted transfers; checks no stale read
                     (I1), every transfer copies the latest value (I2), and
                     counts transfers against OpenMP's default mapping (I3).

Variables are limited to one word (n_vars <= 64) and sets are python ints.
"""
from __future__ import annotations

import itertools

import numpy as np

from paper_2406_13881_b300.workload import unpack_access

R, W_, RW = 1, 2, 3
HOST, DEV = 0, 1


def block_accesses(cfg, b):
    var, kind, space = unpack_access(cfg.acc[cfg.acc_off[b]:cfg.acc_off[b + 1]])
    return [(int(v), int(k), int(s)) for v, k, s in zip(var, kind, space)]


def events(accs):
    """Expand accesses into (var, 'R'|'W', space) events; RW = read, write."""
    out = []
    for v, k, s in accs:
        if k & R:
            out.append((v, "R", s))
        if k & W_:
            out.append((v, "W", s))
    return out


def local_sim(accs, n_vars):
    """Effect of one block, by simulation.  Returns a dict of int bitsets:
    gen/kill per space (out_S = gen | (in_S & ~kill)), ue per space (an
    S-read that can see the value from before the block), def (written)."""
    ev = events(accs)
    res = {}
    for S in (HOST, DEV):
        gen = kill = 0
        for v in range(n_vars):
            outs = []
            for x in (0, 1):
                val = x
                for (u, t, sp) in ev:
                    if u != v:
                        continue
                    if sp == S:          # S-read (after its transfer) or S-write
                        val = 1
                    elif t == "W":       # write in the other space
                        val = 0
                outs.append(val)
            if outs[0]:
                gen |= 1 << v
            if not outs[1]:
                kill |= 1 << v
        res["gen", S] = gen
        res["kill", S] = kill
    for S in (HOST, DEV):
        ue = 0
        for v in range(n_vars):
            written = False
            for (u, t, sp) in ev:
                if u != v:
                    continue
                if t == "R" and sp == S and not written:
                    ue |= 1 << v
                    break
                if t == "W":
                    written = True
        res["ue", S] = ue
    d = 0
    for (u, t, sp) in ev:
        if t == "W":
            d |= 1 << u
    res["def"] = d
    return res


def word(x):
    return int(np.uint64(x))


def graph_lists(cfg):
    succ = [[int(t) for t in cfg.succ[cfg.succ_off[b]:cfg.succ_off[b + 1]]] for b in range(cfg.n_blocks)]
    eid = [list(range(int(cfg.succ_off[b]), int(cfg.succ_off[b + 1]))) for b in range(cfg.n_blocks)]
    return succ, eid


def paths_from(cfg, start, max_edge_visits=1, limit=200000):
    """All paths start -> (block with no successor), each edge used at most
    max_edge_visits times.  A path is (blocks, edges)."""
    succ, eid = graph_lists(cfg)
    out = []
    visits = {}

    def rec(b, blocks, edges):
        if len(out) >= limit:
            raise RuntimeError("too many paths")
        if not succ[b]:
            out.append((list(blocks), list(edges)))
            return
        for t, e in zip(succ[b], eid[b]):
            if visits.get(e, 0) >= max_edge_visits:
                continue
            visits[e] = visits.get(e, 0) + 1
            blocks.append(t)
            edges.append(e)
            rec(t, blocks, edges)
            blocks.pop()
            edges.pop()
            visits[e] -= 1

    rec(start, [start], [])
    return out


def maximal_walks(cfg, start, max_edge_visits=1, limit=200000):
    """Walks from ``start`` that cannot be extended: they end at a block with
    no successor, or where every out-edge has been used max_edge_visits
    times (this covers loops that never exit).  A walk is (blocks, edges)."""
    succ, eid = graph_lists(cfg)
    out = []
    visits = {}

    def rec(b, blocks, edges):
        if len(out) >= limit:
            raise RuntimeError("too many walks")
        ext = False
        for t, e in zip(succ[b], eid[b]):
            if visits.get(e, 0) >= max_edge_visits:
                continue
            ext = True
            visits[e] = visits.get(e, 0) + 1
            blocks.append(t)
            edges.append(e)
            rec(t, blocks, edges)
            blocks.pop()
            edges.pop()
            visits[e] -= 1
        if not ext:
            out.append((list(blocks), list(edges)))

    rec(start, [start], [])
    return out


def random_paths(cfg, start, n_paths, seed=0, max_len=10000):
    """n_paths random walks from ``start`` to a block with no successor
    (successor chosen uniformly); walks longer than max_len are dropped."""
    succ, eid = graph_lists(cfg)
    rng = np.random.default_rng(seed)
    out = []
    tries = 0
    while len(out) < n_paths and tries < 20 * n_paths:
        tries += 1
        b, blocks, edges = start, [start], []
        while succ[b] and len(blocks) < max_len:
            k = int(rng.integers(len(succ[b])))
            edges.append(eid[b][k])
            b = succ[b][k]
            blocks.append(b)
        if not succ[b]:
            out.append((blocks, edges))
    return out


def prefixes_to(paths, n_blocks):
    """For each block, the list of (blocks, edges) prefixes ending at it."""
    pre = [[] for _ in range(n_blocks)]
    seen = [set() for _ in range(n_blocks)]
    for blocks, edges in paths:
        for i, b in enumerate(blocks):
            key = tuple(edges[:i])
            if key not in seen[b]:
                seen[b].add(key)
                pre[b].append((blocks[:i + 1], edges[:i]))
    return pre


# --------------------------------------------------------------------------
# meet over paths
# --------------------------------------------------------------------------

def mop_forward(n_blocks, prefixes, init, top, block_fn, edge_fn=None):
    """x_in[b] = AND over prefixes entry..b of the composed path function
    applied to init (block functions of all blocks before b, edge functions
    of all edges on the prefix).  Blocks without a prefix get ``top``."""
    xin = [top] * n_blocks
    for b in range(n_blocks):
        acc = None
        for blocks, edges in prefixes[b]:
            x = init
            for i in range(len(blocks) - 1):
                x = block_fn(blocks[i], x)
                if edge_fn is not None:
                    x = edge_fn(edges[i], x)
            acc = x if acc is None else acc & x
        if acc is not None:
            xin[b] = acc
    return xin


def walks_from(cfg, start, max_edge_visits=1, limit=400000):
    """Every finite walk from ``start`` (each edge at most max_edge_visits
    times), ending anywhere.  A walk is a list of blocks."""
    succ, eid = graph_lists(cfg)
    out = []
    visits = {}

    def rec(b, blocks):
        if len(out) >= limit:
            raise RuntimeError("too many walks")
        out.append(list(blocks))
        for t, e in zip(succ[b], eid[b]):
            if visits.get(e, 0) >= max_edge_visits:
                continue
            visits[e] = visits.get(e, 0) + 1
            blocks.append(t)
            rec(t, blocks)
            blocks.pop()
            visits[e] -= 1

    rec(start, [start])
    return out


def mop_backward_may(cfg, block_bwd, exit_val, max_edge_visits=1):
    """x_in[b] = OR over every finite walk b..bk of the backward walk
    function applied to what lies beyond bk: the region-exit value if bk has
    no successor, nothing otherwise (the least solution is the union of all
    finite derivations, including walks inside loops that never exit)."""
    res = [0] * cfg.n_blocks
    for b in range(cfg.n_blocks):
        acc = 0
        for blocks in walks_from(cfg, b, max_edge_visits):
            last = blocks[-1]
            x = exit_val if cfg.succ_off[last] == cfg.succ_off[last + 1] else 0
            for blk in reversed(blocks):
                x = block_bwd(blk, x)
            acc |= x
        res[b] = acc
    return res


# --------------------------------------------------------------------------
# path simulation with version counters
# --------------------------------------------------------------------------

class Violation(Exception):
    pass


class PathSim:
    """Replays paths with the emitted transfers.

    transfers: dict with
      'to_edge'  {edge: bitset}, 'from_edge' {edge: bitset},
      'flag'     {access index: 1 (to) | 2 (from)},
      'from_exit' {block: bitset}
    and optionally
      'pre'      {access index: [('to'|'from', var), ...]} made right
                 before that access (before its own flag),
      'start'    [('to'|'from', var), ...] made before the first block,
      'edge_post' {edge: [('to'|'from', var), ...]} made on the edge after
                 its 'to_edge' / 'from_edge' transfers (right before the
                 block it enters)
    """

    def __init__(self, cfg, transfers, entry_h, entry_d, exit_live, hoist_edges=()):
        self.cfg = cfg
        self.t = transfers
        self.entry_h, self.entry_d, self.exit_live = entry_h, entry_d, exit_live
        self.hoist_edges = set(hoist_edges)
        self.accs = [block_accesses(cfg, b) for b in range(cfg.n_blocks)]
        self.region = None if cfg.region is None else [int(x) for x in cfg.region]
        self.rvars = {}
        if self.region is not None:
            for b in range(cfg.n_blocks):
                if self.region[b] >= 0:
                    s = self.rvars.setdefault(self.region[b], set())
                    s.update(v for v, _, _ in self.accs[b])

    def run(self, blocks, edges):
        """Returns (count_all, count_charged, default) for one path; raises
        Violation on a stale read (I1) or a transfer from a stale copy (I2)."""
        n = self.cfg.n_vars
        latest = [0] * n
        hv = [0 if (self.entry_h >> v) & 1 else -1 for v in range(n)]
        dv = [0 if (self.entry_d >> v) & 1 else -1 for v in range(n)]
        # pending hoisted transfers waiting to be served: (var, space) -> True
        log = []            # (kind 'to'|'from', var, effective, hoisted, position)
        evlog = []          # (position, var, 'R'|'W', space)
        pos = [0]

        def xfer(kind, v, hoisted):
            src, dst = (hv, dv) if kind == "to" else (dv, hv)
            if src[v] != latest[v]:
                raise Violation("I2: %s of var %d copies a stale value" % (kind, v))
            eff = dst[v] != latest[v]
            dst[v] = src[v]
            log.append((kind, v, eff, hoisted, pos[0]))
            pos[0] += 1

        def access(v, t, s):
            own = dv if s == DEV else hv
            oth = hv if s == DEV else dv
            if t == "R":
                if own[v] != latest[v]:
                    raise Violation("I1: stale %s read of var %d" % ("device" if s else "host", v))
            else:
                latest[v] += 1
                own[v] = latest[v]
            evlog.append((pos[0], v, t, s))
            pos[0] += 1

        for kind, v in self.t.get("start", ()):
            xfer(kind, v, False)
        for i, b in enumerate(blocks):
            if i > 0:
                e = edges[i - 1]
                hoist = e in self.hoist_edges
                for v in range(n):
                    if (self.t["to_edge"].get(e, 0) >> v) & 1:
                        xfer("to", v, hoist)
                    if (self.t["from_edge"].get(e, 0) >> v) & 1:
                        xfer("from", v, hoist)
                for kind, v in self.t.get("edge_post", {}).get(e, ()):
                    xfer(kind, v, False)
            base = int(self.cfg.acc_off[b])
            for j, (v, k, s) in enumerate(self.accs[b]):
                for kind, u in self.t.get("pre", {}).get(base + j, ()):
                    xfer(kind, u, False)
                f = self.t["flag"].get(base + j, 0)
                if f == 1:
                    xfer("to", v, False)
                elif f == 2:
                    xfer("from", v, False)
                if k & R:
                    access(v, "R", s)
                if k & W_:
                    access(v, "W", s)
        last = blocks[-1]
        at_exit = self.cfg.succ_off[last] == self.cfg.succ_off[last + 1]
        if at_exit:
            for v in range(n):
                if (self.t["from_exit"].get(last, 0) >> v) & 1:
                    xfer("from", v, False)
            for v in range(n):
                if (self.exit_live >> v) & 1 and hv[v] != latest[v]:
                    raise Violation("I1: host copy of live var %d stale at exit" % v)
        # I3 bookkeeping: effective transfers; a hoisted one counts only if a
        # read in its destination space uses it before any write to the var
        charged = 0
        for kind, v, eff, hoisted, p in log:
            if not eff:
                continue
            if hoisted:
                dst = DEV if kind == "to" else HOST
                served = False
                for (q, u, t, s) in evlog:
                    if q < p or u != v:
                        continue
                    if t == "W":
                        break
                    if s == dst:
                        served = True
                        break
                if not served and at_exit and kind == "from" and (self.exit_live >> v) & 1:
                    served = not any(q > p and u == v and t == "W" for (q, u, t, s) in evlog)
                if not served:
                    continue
            charged += 1
        # a value that is valid only on the device at entry was produced by a
        # kernel before this code; the default mapping copies it back once
        default = sum(1 for v in range(n) if (self.entry_d >> v) & 1 and not (self.entry_h >> v) & 1)
        if self.region is not None:
            prev = -1
            for b in blocks:
                r = self.region[b]
                if r >= 0 and r != prev:
                    default += 2 * len(self.rvars.get(r, ()))
                prev = r
        return len(log), charged, default


def transfers_from_oracle(cfg, res):
    """Dict form of the oracle's emitted transfers (single word)."""
    t = {"to_edge": {}, "from_edge": {}, "flag": {}, "from_exit": {}}
    for e in range(cfg.n_edges):
        if res["to_edge"][e, 0]:
            t["to_edge"][e] = word(res["to_edge"][e, 0])
        if res["from_edge"][e, 0]:
            t["from_edge"][e] = word(res["from_edge"][e, 0])
    for i in range(cfg.n_acc):
        if res["acc_flag"][i]:
            t["flag"][i] = int(res["acc_flag"][i])
    for b in range(cfg.n_blocks):
        if res["from_exit"][b, 0]:
            t["from_exit"][b] = word(res["from_exit"][b, 0])
    return t


def each_single_removal(t):
    """Yield (description, transfers) with exactly one transfer removed."""
    for key in ("to_edge", "from_edge", "from_exit"):
        for loc, bits in t[key].items():
            v = 0
            while bits >> v:
                if (bits >> v) & 1:
                    u = {k: dict(x) for k, x in t.items()}
                    u[key][loc] = bits & ~(1 << v)
                    yield ("%s[%d] var %d" % (key, loc, v), u)
                v += 1
    for i in t["flag"]:
        u = {k: dict(x) for k, x in t.items()}
        del u["flag"][i]
        yield ("flag[%d]" % i, u)
