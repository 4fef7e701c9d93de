"""Seeded synthetic inputs: structured control-flow graphs with per-block
access lists, shaped like the OpenMP offload programs the paper analyses
(Sec. V, Table III: a handful of kernels and mapped variables; Sec. IV-B:
if/switch conditionals, for/while/do loops, offloaded nodes).

This module holds no part of the analysis itself: it only draws graphs and
access lists from seeded distributions, so that the CUDA library and the CPU
oracle can be fed identical inputs.  All randomness comes from
``numpy.random.Generator(PCG64(seed))``.

Input format (shared by the C ABI and the oracle, documented in
``include/ompdart.h``):
  succ_off[N+1], succ[E]      CSR successor lists (int32); edge id = CSR slot
  acc_off[N+1], acc[A]        per-block ordered accesses, packed uint32:
                              bits 0-23 variable, 24-25 kind (1 R, 2 W,
                              3 RW/unknown), bit 26 space (0 host, 1 target)
  region[N]                   kernel id of the block or -1 (tests only)
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import sys

import numpy as np

KIND_R, KIND_W, KIND_RW = 1, 2, 3
SPACE_HOST, SPACE_DEV = 0, 1


def pack_access(var, kind, space):
    var = np.asarray(var, dtype=np.uint32)
    return (var | (np.asarray(kind, dtype=np.uint32) << np.uint32(24))
            | (np.asarray(space, dtype=np.uint32) << np.uint32(26))).astype(np.uint32)


def unpack_access(acc):
    acc = np.asarray(acc, dtype=np.uint32)
    return (acc & 0xFFFFFF).astype(np.int64), ((acc >> 24) & 3).astype(np.int64), ((acc >> 26) & 1).astype(np.int64)


@dataclasses.dataclass
class CFG:
    n_blocks: int
    n_vars: int
    entry: int
    succ_off: np.ndarray
    succ: np.ndarray
    acc_off: np.ndarray
    acc: np.ndarray
    region: np.ndarray | None = None
    entry_host_valid: np.ndarray | None = None
    entry_dev_valid: np.ndarray | None = None
    exit_host_live: np.ndarray | None = None
    # call table (Sec. IV-C): [n_calls, 7, W] rows ReqH, ReqD, GenH, KillH,
    # GenD, KillD, MustDef for call pseudo-accesses (bit 31 | row)
    call_planes: np.ndarray | None = None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_edges(self):
        return int(self.succ_off[-1])

    @property
    def n_acc(self):
        return int(self.acc_off[-1])

    @property
    def W(self):
        return (self.n_vars + 63) // 64

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.succ_off, self.succ, self.acc_off, self.acc):
            h.update(np.ascontiguousarray(a).tobytes())
        h.update(np.int64([self.n_blocks, self.n_vars, self.entry]).tobytes())
        return h.hexdigest()[:16]


def from_lists(succs, accs, n_vars, entry=0, region=None, **kw) -> CFG:
    """Build a CFG from python lists: succs[b] = [targets], accs[b] =
    [(var, kind, space), ...].  Handy for hand-written cases."""
    n = len(succs)
    so = np.zeros(n + 1, dtype=np.int32)
    so[1:] = np.cumsum([len(s) for s in succs])
    s = np.array([t for ss in succs for t in ss], dtype=np.int32)
    ao = np.zeros(n + 1, dtype=np.int32)
    ao[1:] = np.cumsum([len(a) for a in accs])
    flat = [x for aa in accs for x in aa]
    acc = pack_access([x[0] for x in flat], [x[1] for x in flat], [x[2] for x in flat]) if flat \
        else np.zeros(0, dtype=np.uint32)
    reg = None if region is None else np.asarray(region, dtype=np.int32)
    return CFG(n, n_vars, entry, so, s, ao, acc, reg, **kw)


def var_mask(n_vars, vars_):
    """uint64[W] bit-mask with the given variables set."""
    m = np.zeros((n_vars + 63) // 64, dtype=np.uint64)
    for v in vars_:
        m[v >> 6] |= np.uint64(1) << np.uint64(v & 63)
    return m


# --------------------------------------------------------------------------
# structured CFG shapes
# --------------------------------------------------------------------------

class _Builder:
    """Emits blocks of a structured program: sequences of plain blocks,
    if-then, if-then-else and while loops (test at the header, body, back
    edge from every body exit).  Block ids follow program (pre-)order."""

    def __init__(self, rng, cap, p_if_then, p_if_else, p_while, body_mean,
                 max_depth, max_loop_depth):
        self.rng = rng
        self.succs: list[list[int]] = []
        self.pending: list[int] = []
        self.cap = cap                      # blocks that may still be created
        self.pt, self.pe, self.pw = p_if_then, p_if_else, p_while
        self.body_mean = body_mean
        self.max_depth, self.max_loop_depth = max_depth, max_loop_depth
        self.n_back = 0
        self.n_cond = 0
        self.n_head = 0
        self.max_seen_loop_depth = 0
        self.loops = []                     # (header, first, end, loop_depth)
        self.seqs = []                      # (depth, [(first_block, end_block), ...])
        # pre-drawn uniforms keep the python loop cheap
        self._u = rng.random(1 << 16)
        self._ui = 0

    def u(self):
        if self._ui == len(self._u):
            self._u = self.rng.random(1 << 16)
            self._ui = 0
        x = self._u[self._ui]
        self._ui += 1
        return x

    def new_block(self):
        b = len(self.succs)
        self.succs.append([])
        for p in self.pending:
            self.succs[p].append(b)
        self.pending = []
        self.cap -= 1
        return b

    def body_len(self):
        # 1 + geometric with mean body_mean - 1
        m = self.body_mean - 1.0
        if m <= 0:
            return 1
        p = 1.0 / (1.0 + m)
        return 1 + int(math.floor(math.log(max(self.u(), 1e-300)) / math.log(1.0 - p)))

    def seq(self, n_stmts, depth, loop_depth):
        rec = []
        self.seqs.append((depth, rec))
        k = 0
        while (n_stmts is None or k < n_stmts) and self.cap > 0:
            first = len(self.succs)
            self.stmt(depth, loop_depth)
            rec.append((first, len(self.succs)))
            k += 1

    def stmt(self, depth, loop_depth):
        x = self.u()
        can_nest = depth < self.max_depth
        if x < self.pw and can_nest and loop_depth < self.max_loop_depth and self.cap >= 3:
            # for/while loop: header (test) -> body -> latch (increment) -> header
            h = self.new_block()
            self.n_head += 1
            self.pending = [h]
            first = len(self.succs)
            self.cap -= 1                   # keep room for the latch
            self.seq(self.body_len(), depth + 1, loop_depth + 1)
            self.cap += 1
            latch = self.new_block()
            self.succs[latch].append(h)
            self.n_back += 1
            self.pending = [h]
            self.loops.append((h, first, len(self.succs), loop_depth + 1))
            self.max_seen_loop_depth = max(self.max_seen_loop_depth, loop_depth + 1)
        elif x < self.pw + self.pe and can_nest and self.cap >= 3:
            c = self.new_block()
            self.n_cond += 1
            self.pending = [c]
            self.seq(self.body_len(), depth + 1, loop_depth)
            t_exits = self.pending
            self.pending = [c]
            if self.cap > 0:
                self.seq(self.body_len(), depth + 1, loop_depth)
            else:  # no room left for the else body: degenerate to if-then
                pass
            self.pending = t_exits + self.pending
        elif x < self.pw + self.pe + self.pt and can_nest and self.cap >= 2:
            c = self.new_block()
            self.n_cond += 1
            self.pending = [c]
            self.seq(self.body_len(), depth + 1, loop_depth)
            self.pending = self.pending + [c]
        else:
            b = self.new_block()
            self.pending = [b]


def _assign_regions(rng, b: _Builder, n, mode, target_frac, region_mean, n_regions, region_max_depth):
    region = np.full(n, -1, dtype=np.int32)
    seqs = [(d, rec) for d, rec in b.seqs if d <= region_max_depth and rec]
    rid = 0
    if mode == "runs":
        # expected blocks per started run ~ region_mean; choose the start
        # probability per statement so that ~target_frac of blocks are covered
        n_stmt = sum(len(rec) for _, rec in seqs)
        avg_stmt = max(1.0, n / max(1, n_stmt))
        q = min(0.9, target_frac * avg_stmt / region_mean * 1.75)
        for d, rec in seqs:
            i = 0
            while i < len(rec):
                f, e = rec[i]
                if region[f] >= 0 or rng.random() >= q:
                    i += 1
                    continue
                want = max(1, int(rng.geometric(1.0 / region_mean)))
                j, got = i, 0
                while j < len(rec) and got < want and region[rec[j][0]] < 0:
                    got += rec[j][1] - rec[j][0]
                    j += 1
                region[rec[i][0]:rec[j - 1][1]] = rid
                rid += 1
                i = j
    else:  # "count": exactly n_regions runs, ~target_frac of blocks overall
        want = max(1, int(round(target_frac * n / n_regions)))
        cand = [(si, i) for si, (d, rec) in enumerate(seqs) for i in range(len(rec))]
        tries = 0
        while rid < n_regions and tries < 200 * n_regions and cand:
            tries += 1
            si, i = cand[int(rng.integers(len(cand)))]
            rec = seqs[si][1]
            j, got = i, 0
            ok = True
            while j < len(rec) and got < want:
                if (region[rec[j][0]:rec[j][1]] >= 0).any():
                    ok = False
                    break
                got += rec[j][1] - rec[j][0]
                j += 1
            if not ok or j == i or (region[rec[i][0]:rec[j - 1][1]] >= 0).any():
                continue
            # keep kernels apart: the block before a run must not be target
            region[rec[i][0]:rec[j - 1][1]] = rid
            rid += 1
    region[0] = -1
    return region, rid


def structured(seed, n_blocks, n_vars, *, p_if_then=0.13, p_if_else=0.135, p_while=0.075,
               body_mean=2.0, max_depth=6, max_loop_depth=4, region_mode="runs",
               target_frac=0.2, region_mean=32.0, n_regions=3, region_max_depth=2,
               acc_min=1, acc_max=16, var_dist="zipf", zipf_s=1.1, p_write=0.3,
               p_rw=0.0, rng=None) -> CFG:
    """One structured CFG with exactly ``n_blocks`` blocks: an entry block,
    a top-level statement sequence, and one exit block.  Statement mix per
    statement: while p_while, if-then-else p_if_else, if-then p_if_then,
    plain otherwise (nesting and budget permitting).  Accesses per block are
    uniform in [acc_min, acc_max]; variables uniform or Zipf(zipf_s) through
    a seeded rank permutation; kind W with probability p_write (RW with
    p_rw), else R; the space is target inside kernel regions, host outside."""
    rng = np.random.default_rng(seed) if rng is None else rng
    if n_blocks < 2:
        raise ValueError("need at least an entry and an exit block")
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 20000))
    b = _Builder(rng, n_blocks - 1, p_if_then, p_if_else, p_while, body_mean, max_depth, max_loop_depth)
    b.new_block()                       # entry: no predecessors
    b.pending = [0]
    b.seq(None, 0, 0)
    b.cap += 1
    b.new_block()                       # the single exit block
    sys.setrecursionlimit(old)
    n = len(b.succs)
    assert n == n_blocks, (n, n_blocks)
    region, nreg = _assign_regions(rng, b, n, region_mode, target_frac, region_mean, n_regions,
                                   region_max_depth)
    so = np.zeros(n + 1, dtype=np.int32)
    so[1:] = np.cumsum(np.fromiter((len(s) for s in b.succs), dtype=np.int64, count=n))
    succ = np.fromiter((t for s in b.succs for t in s), dtype=np.int32, count=int(so[-1]))
    acc_off, acc = draw_accesses(rng, n, n_vars, region, acc_min, acc_max, var_dist, zipf_s, p_write, p_rw)
    g = CFG(n, n_vars, 0, so, succ, acc_off, acc, region)
    g.meta = dict(seed=seed, n_blocks=n, n_edges=int(so[-1]), n_vars=n_vars,
                  mean_out_degree=float(so[-1]) / n, back_edges=b.n_back,
                  back_edge_frac=b.n_back / max(1, int(so[-1])), headers=b.n_head, conds=b.n_cond,
                  header_frac=b.n_head / n, cond_frac=b.n_cond / n,
                  max_loop_depth=b.max_seen_loop_depth, regions=nreg,
                  target_block_frac=float((region >= 0).mean()), n_acc=int(acc_off[-1]),
                  loops=[(h, f, e, d) for h, f, e, d in b.loops])
    return g


def draw_accesses(rng, n, n_vars, region, acc_min, acc_max, var_dist="uniform", zipf_s=1.1,
                  p_write=0.3, p_rw=0.0):
    cnt = rng.integers(acc_min, acc_max + 1, size=n)
    acc_off = np.zeros(n + 1, dtype=np.int32)
    acc_off[1:] = np.cumsum(cnt)
    A = int(acc_off[-1])
    if var_dist == "zipf":
        ranks = np.arange(1, n_vars + 1, dtype=np.float64)
        cdf = np.cumsum(ranks ** (-zipf_s))
        cdf /= cdf[-1]
        r = np.searchsorted(cdf, rng.random(A), side="right")
        r = np.minimum(r, n_vars - 1)
        perm = rng.permutation(n_vars)
        var = perm[r]
    else:
        var = rng.integers(0, n_vars, size=A)
    u = rng.random(A)
    kind = np.where(u < p_rw, KIND_RW, np.where(u < p_rw + p_write, KIND_W, KIND_R))
    blk = np.repeat(np.arange(n), cnt)
    space = (np.asarray(region)[blk] >= 0).astype(np.int64) if region is not None else np.zeros(A, np.int64)
    return acc_off, pack_access(var, kind, space)


# --------------------------------------------------------------------------
# the paper-shaped workloads
# --------------------------------------------------------------------------

def single_small(seed=1) -> CFG:
    """64 blocks with exactly one loop nest two deep (back edges from the
    latches), 32 variables (one word), 1-8 accesses per block, uniform
    variables, R:W = 70:30, host accesses except in 3 contiguous kernel
    ranges (at least one inside the loop nest); entry state: every variable
    host-valid."""
    rng = np.random.default_rng(seed)
    for _ in range(100000):
        g = structured(None, 64, 32, p_if_then=0.12, p_if_else=0.12, p_while=0.06, body_mean=2.5,
                       max_depth=4, max_loop_depth=2, region_mode="count", target_frac=0.2,
                       n_regions=3, region_max_depth=2, acc_min=1, acc_max=8, var_dist="uniform",
                       p_write=0.3, rng=rng)
        loops = g.meta["loops"]
        inner_kernel = any(g.region[h] < 0 and (g.region[f:e] >= 0).any() for h, f, e, d in loops if d == 1)
        if len(loops) == 2 and {d for *_, d in loops} == {1, 2} and g.meta["regions"] == 3 \
                and inner_kernel:
            g.meta["seed"] = seed
            return g
    raise RuntimeError("no 64-block single-nest shape found")


def single_large(seed=2, n_blocks=1 << 20, n_vars=4096) -> CFG:
    """The large single CFG: 2^20 blocks, mean out-degree ~1.3, loops nested
    up to 4 deep (~5% back edges), 4096 variables (64 words), ~20% of the
    blocks in kernel regions (runs of geometric length, mean 32 blocks),
    1-16 accesses per block, Zipf(1.1) variables, R:W = 70:30."""
    return structured(seed, n_blocks, n_vars, p_if_then=0.14, p_if_else=0.145, p_while=0.078,
                      body_mean=2.0, max_depth=6, max_loop_depth=4, region_mode="runs",
                      target_frac=0.2, region_mean=32.0, region_max_depth=2, acc_min=1,
                      acc_max=16, var_dist="zipf", zipf_s=1.1, p_write=0.3)


def batch_sizes(rng, n, median=512.0, sigma=1.0, lo=16, hi=65536):
    x = np.round(np.exp(rng.normal(math.log(median), sigma, size=n))).astype(np.int64)
    return np.clip(x, lo, hi)


def batch(seed=3, n_cfgs=10000, var_choices=(64, 256, 1024, 2048)) -> list[CFG]:
    """Independent CFGs: block counts lognormal (median 512, sigma 1.0,
    clipped to [16, 65536]), variable counts uniform over var_choices,
    accesses as in the small case (1-8 per block, uniform variables,
    R:W = 70:30), loops nested up to 2 deep, ~20% target blocks in 3 runs."""
    rng = np.random.default_rng(seed)
    sizes = batch_sizes(rng, n_cfgs)
    nv = rng.choice(np.asarray(var_choices), size=n_cfgs)
    out = []
    for i in range(n_cfgs):
        g = structured(None, int(sizes[i]), int(nv[i]), p_if_then=0.11, p_if_else=0.125,
                       p_while=0.065, body_mean=2.0, max_depth=5, max_loop_depth=2,
                       region_mode="count", target_frac=0.2, n_regions=3, region_max_depth=2,
                       acc_min=1, acc_max=8, var_dist="uniform", p_write=0.3, rng=rng)
        g.meta["seed"] = (seed, i)
        out.append(g)
    return out


def random_graph(seed, n_blocks, n_vars, *, p_edge=0.25, max_out=3, acc_max=4, p_dev=0.4,
                 p_write=0.3, p_rw=0.1, acyclic=False, rng=None) -> CFG:
    """Unstructured random CFG (possibly irreducible) for fuzzing: block 0 is
    the entry with no predecessors; every block gets 0..max_out successors
    chosen among blocks 1..N-1 (forward-only if ``acyclic``)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    succs = []
    for b in range(n_blocks):
        k = int(rng.integers(0, max_out + 1)) if b else max(1, int(rng.integers(0, max_out + 1)))
        if acyclic:
            cand = list(range(b + 1, n_blocks))
        else:
            cand = list(range(1, n_blocks))
        if not cand:
            succs.append([])
            continue
        succs.append([int(x) for x in rng.choice(cand, size=min(k, len(cand)), replace=True)])
    accs = []
    for b in range(n_blocks):
        k = int(rng.integers(0, acc_max + 1))
        lst = []
        for _ in range(k):
            u = rng.random()
            kind = KIND_RW if u < p_rw else (KIND_W if u < p_rw + p_write else KIND_R)
            lst.append((int(rng.integers(0, n_vars)), kind, int(rng.random() < p_dev)))
        accs.append(lst)
    return from_lists(succs, accs, n_vars)


def restrict_words(g: CFG, w0: int, w1: int) -> tuple[CFG, np.ndarray]:
    """The same CFG with only the accesses to variables 64*w0 .. 64*w1 - 1,
    renumbered from 0 (n_vars = how many of them exist).  Returns (cfg,
    kept) where ``kept`` are the original access indices.  Entry/exit masks
    are sliced to words w0..w1-1.  A word range is a shard of the problem:
    variables never interact."""
    var, kind, space = unpack_access(g.acc)
    keep = np.nonzero(((var >> 6) >= w0) & ((var >> 6) < w1))[0]
    blk = np.repeat(np.arange(g.n_blocks), np.diff(g.acc_off))
    cnt = np.bincount(blk[keep], minlength=g.n_blocks)
    ao = np.zeros(g.n_blocks + 1, dtype=np.int32)
    ao[1:] = np.cumsum(cnt)
    nv = min(64 * (w1 - w0), g.n_vars - 64 * w0)
    acc = pack_access(var[keep] - 64 * w0, kind[keep], space[keep])

    def sl(m):
        return None if m is None else np.ascontiguousarray(m[w0:w1])

    h = CFG(g.n_blocks, nv, g.entry, g.succ_off, g.succ, ao, acc, g.region,
            sl(g.entry_host_valid), sl(g.entry_dev_valid), sl(g.exit_host_live))
    return h, keep


def restrict_word(g: CFG, w: int) -> tuple[CFG, np.ndarray]:
    """restrict_words for the single word column w (used to check one word
    column of a wide problem against the oracle)."""
    return restrict_words(g, w, w + 1)


# --------------------------------------------------------------------------
# interprocedural workload: a call graph of functions
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Program:
    """Functions (CFGs over globals + their pointer parameters) and call
    sites: function f's k-th call site is site site_off[f] + k, named by the
    call pseudo-access with row k; site s calls site_callee[s] and
    var_maps[s][v] is the caller variable callee variable v denotes."""
    funcs: list
    site_off: np.ndarray
    site_callee: np.ndarray
    var_maps: list
    n_globals: int
    level: np.ndarray
    meta: dict = dataclasses.field(default_factory=dict)


def call_graph(seed=4, n_funcs=2000, max_depth=8, fanout=(1, 6), blocks=(32, 4096), median_blocks=256,
               n_globals=512, max_formals=4) -> Program:
    """A call DAG of n_funcs functions over n_globals globals: each function
    sits on a level 0..max_depth-1 (level 0 are the roots; the last level
    are leaves) and every non-leaf calls 1..6 functions of deeper levels
    (most often the next one).  A function has 0..max_formals pointer
    parameters (variables n_globals.. of its own numbering); each call
    passes, per parameter, a random global or one of the caller's own
    parameters.  Each function's CFG is structured with lognormal block
    counts (median `median_blocks`, clipped to `blocks`), 1-8 accesses per
    block (uniform variables, R:W = 70:30, ~20% target blocks in 3 runs) and
    its calls inserted at random places of random blocks."""
    rng = np.random.default_rng(seed)
    level = np.sort(rng.integers(0, max_depth, size=n_funcs))
    level[: max(1, n_funcs // 50)] = 0
    by_level = [np.flatnonzero(level == L) for L in range(max_depth)]
    n_formals = rng.integers(0, max_formals + 1, size=n_funcs)
    sizes = batch_sizes(rng, n_funcs, median=median_blocks, lo=blocks[0], hi=blocks[1])
    funcs, site_callee, var_maps, site_off = [], [], [], [0]
    for f in range(n_funcs):
        nv = n_globals + int(n_formals[f])
        g = structured(None, int(sizes[f]), nv, p_if_then=0.11, p_if_else=0.125, p_while=0.065, body_mean=2.0,
                       max_depth=5, max_loop_depth=3, region_mode="count", target_frac=0.2, n_regions=3,
                       region_max_depth=2, acc_min=1, acc_max=8, var_dist="uniform", p_write=0.3, rng=rng)
        L = int(level[f])
        deeper = [x for x in range(L + 1, max_depth) if len(by_level[x])]
        callees = []
        if deeper:
            for _ in range(int(rng.integers(fanout[0], fanout[1] + 1))):
                nxt = deeper[0] if rng.random() < 0.7 else deeper[int(rng.integers(0, len(deeper)))]
                callees.append(int(rng.choice(by_level[nxt])))
        accs = [list(g.acc[g.acc_off[b]:g.acc_off[b + 1]]) for b in range(g.n_blocks)]
        for k, c in enumerate(callees):
            b = int(rng.integers(0, g.n_blocks))
            accs[b].insert(int(rng.integers(0, len(accs[b]) + 1)), np.uint32(0x80000000 | k))
            vm = np.arange(n_globals + int(n_formals[c]), dtype=np.int32)
            for j in range(int(n_formals[c])):  # actual of each pointer parameter
                vm[n_globals + j] = int(rng.integers(0, nv)) if rng.random() < 0.5 or nv == n_globals \
                    else n_globals + int(rng.integers(0, nv - n_globals))
            site_callee.append(c)
            var_maps.append(vm)
        ao = np.zeros(g.n_blocks + 1, dtype=np.int32)
        ao[1:] = np.cumsum([len(x) for x in accs])
        h = CFG(g.n_blocks, nv, 0, g.succ_off, g.succ, ao, np.array([a for x in accs for a in x], dtype=np.uint32),
                g.region)
        h.meta = dict(g.meta, n_acc=int(ao[-1]), calls=len(callees), level=L)
        funcs.append(h)
        site_off.append(len(site_callee))
    return Program(funcs, np.array(site_off, dtype=np.int32), np.array(site_callee, dtype=np.int32), var_maps,
                   n_globals, level, dict(seed=seed, n_funcs=n_funcs, max_depth=max_depth))
