"""Directive classification and consolidation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product library never does.  Plain Python over the
result of ``oracle.solve(cfg, data_region=True)``; it shares no code with
the library.

What the paper's rewriter inserts (Table II; Sec. IV-D data region;
Sec. IV-F consolidation), from the transfers of the data-flow:

* kernels: block b belongs to kernel region[b] (>= 0).  A `to' right before
  a device read inside kernel k is made right before kernel k instead (no
  host code runs inside a kernel, so the host copy it reads is the same
  there), one ``target update to`` per kernel; likewise a `from' right
  before a host read inside kernel k (a firstprivate scalar, below) whose
  variable kernel k does not write on the device.
* firstprivate (Sec. IV-D, scalar paragraph): a scalar variable that
  kernel k reads on the device and never writes is passed to k as
  firstprivate: its device reads in k read a private copy made from the
  host value at the launch, so ``firstprivate_view`` relabels them as host
  reads (they need the host copy valid; the device copy stays as it was --
  "the firstprivate data is no longer valid" after the kernel) and the
  kernel gets a firstprivate clause instead of a `to'.
* the single target data region R (``res["in_region"]``): transfers on its
  boundary become map-type clauses of the ``target data`` construct,
  everything inside stays a ``target update``:
    - map(to:)   a `to' made on every way into R: on every edge entering R
                 (and R does not start at the function's entry), or the
                 lifted `to's of the kernel at which R starts (its entry
                 edges are exactly R's entry edges);
    - map(from:) a `from' made on every way out of R: on every edge leaving
                 R and at every function exit inside R;
    - map(tofrom:) both; map(alloc:) a variable some kernel accesses that
                 has neither;
  a transfer on R's boundary that is not made on every way in (out) stays
  an update right after R opens (before it closes) on that way.
* consolidation (Sec. IV-F: one directive per insertion point): a `from'
  right before a host read moves up to just after the previous access of
  the same variable in the block (or the block's start: nothing in between
  touches it); transfers at one point and in one direction form one
  directive.  Edge transfers are one directive per edge and direction,
  exit transfers one per exit block, call-site transfers stay at the call.
"""
import numpy as np

from paper_2406_13881_b300.workload import unpack_access


def firstprivate_view(cfg, scalar_vars):
    """(cfg with the firstprivate reads relabelled, [n_kernels, W] rows of
    the firstprivate clauses)."""
    N, W = cfg.n_blocks, cfg.W
    region = np.asarray(cfg.region, np.int32)
    K = int(region.max()) + 1 if N and region.max() >= 0 else 0
    acc = np.asarray(cfg.acc, np.uint32).copy()
    var, kind, space = unpack_access(acc)
    is_call = (acc >> np.uint32(31)) != 0
    blk = np.repeat(np.arange(N), np.diff(np.asarray(cfg.acc_off)))
    sc = np.asarray(scalar_vars, np.uint64)
    fp = np.zeros((K, W), np.uint64)
    for k in range(K):
        inside = (region[blk] == k) & ~is_call
        for v in set(var[inside].tolist()):
            if not (int(sc[v >> 6]) >> (v & 63)) & 1:
                continue
            mine = inside & (var == v)
            if (kind[mine] & 2).any():
                continue  # written in the kernel: not read-only
            if (space[mine] == 1).any():
                fp[k, v >> 6] |= np.uint64(1) << np.uint64(v & 63)
                acc[mine & (space == 1)] &= ~np.uint32(1 << 26)
    out = type(cfg)(cfg.n_blocks, cfg.n_vars, cfg.entry, cfg.succ_off, cfg.succ, cfg.acc_off, acc, cfg.region,
                    cfg.entry_host_valid, cfg.entry_dev_valid, cfg.exit_host_live, cfg.call_planes)
    return out, fp


def _reachable_edges(cfg, reach):
    for b in range(cfg.n_blocks):
        for e in range(int(cfg.succ_off[b]), int(cfg.succ_off[b + 1])):
            t = int(cfg.succ[e])
            if reach[b] and reach[t]:
                yield b, e, t


def classify(cfg, res):
    N, A, E = cfg.n_blocks, cfg.n_acc, cfg.n_edges
    W = res["h_in"].shape[1]
    reach = res["reachable"].astype(bool)
    inr = res["in_region"].astype(bool)
    region = np.full(N, -1, np.int32) if cfg.region is None else np.asarray(cfg.region, np.int32)
    K = int(region.max()) + 1 if N and region.max() >= 0 else 0
    acc = np.asarray(cfg.acc, np.uint32)
    var, kind, space = unpack_access(acc)
    is_call = (acc >> np.uint32(31)) != 0
    blk = np.repeat(np.arange(N), np.diff(np.asarray(cfg.acc_off)))
    flag = res["acc_flag"].astype(np.int64)
    to_e = res["to_edge"].copy()
    fr_e = res["from_edge"].copy()
    fx = res["from_exit"].copy()

    def bit(v):
        r = np.zeros(W, np.uint64)
        r[v >> 6] = np.uint64(1) << np.uint64(v & 63)
        return r

    # ---- kernel-entry transfers: a `to' (`from') inside kernel k moves
    # before it unless k writes the variable on the host (device)
    kernel_to = np.zeros((K, W), np.uint64)
    kernel_from = np.zeros((K, W), np.uint64)
    wrote = {}
    for i in range(A):
        b = int(blk[i])
        if region[b] >= 0 and not is_call[i] and kind[i] & 2:
            wrote.setdefault((int(region[b]), int(space[i])), set()).add(int(var[i]))
    lifted = np.zeros(A, bool)
    for i in range(A):
        b = int(blk[i])
        if not reach[b] or region[b] < 0 or is_call[i] or flag[i] not in (1, 2):
            continue
        k, v = int(region[b]), int(var[i])
        if flag[i] == 1 and v not in wrote.get((k, 0), ()):
            kernel_to[k] |= bit(v)
            lifted[i] = True
        elif flag[i] == 2 and v not in wrote.get((k, 1), ()):
            kernel_from[k] |= bit(v)
            lifted[i] = True
    # ---- data region boundary
    r_entry, r_exit, k_entry = [], [], [[] for _ in range(K)]
    for b, e, t in _reachable_edges(cfg, reach):
        if not inr[b] and inr[t]:
            r_entry.append(e)
        if inr[b] and not inr[t]:
            r_exit.append(e)
        if region[t] >= 0 and region[b] != region[t]:
            k_entry[region[t]].append(e)
    exits_in_r = [b for b in range(N) if reach[b] and inr[b] and cfg.succ_off[b] == cfg.succ_off[b + 1]]
    entry_in_r = bool(inr[cfg.entry])
    has_region = bool(inr.any())
    map_to = np.zeros(W, np.uint64)
    map_from = np.zeros(W, np.uint64)
    if has_region:
        # `to's on every edge into R (R does not start at the function entry)
        if r_entry and not entry_in_r:
            u = np.full(W, ~np.uint64(0), np.uint64)
            for e in r_entry:
                u &= to_e[e]
            map_to |= u
            for e in r_entry:
                to_e[e] &= ~u
        # the kernel R starts at: its entry edges are exactly R's
        for k in range(K):
            starts = sorted(k_entry[k]) == sorted(r_entry) and entry_in_r == (region[cfg.entry] == k)
            if starts and kernel_to[k].any() and (r_entry or entry_in_r):
                map_to |= kernel_to[k]
                kernel_to[k] = 0
        # `from's at every way out of R
        outs = [fr_e[e] for e in r_exit] + [fx[b] for b in exits_in_r]
        if outs:
            u = np.full(W, ~np.uint64(0), np.uint64)
            for x in outs:
                u &= x
            map_from |= u
            for e in r_exit:
                fr_e[e] &= ~u
            for b in exits_in_r:
                fx[b] &= ~u
    dev = np.zeros(W, np.uint64)
    for i in range(A):
        if reach[blk[i]] and region[blk[i]] >= 0 and not is_call[i] and space[i] == 1:
            dev |= bit(int(var[i]))
    map_alloc = dev & ~map_to & ~map_from if has_region else np.zeros(W, np.uint64)
    # ---- consolidated points of the access transfers
    acc_point = np.full(A, -1, np.int64)
    for i in range(A):
        if not flag[i] or lifted[i] or not reach[blk[i]]:
            continue
        if is_call[i]:
            acc_point[i] = i
            continue
        b = int(blk[i])
        j = i
        while j > int(cfg.acc_off[b]):
            if is_call[j - 1] or int(var[j - 1]) == int(var[i]):
                break
            j -= 1
        acc_point[i] = j
    points = set()
    for i in range(A):
        if acc_point[i] >= 0:
            if flag[i] & 1:
                points.add((int(acc_point[i]), 1))
            if flag[i] & 2:
                points.add((int(acc_point[i]), 2))
    n_dir = (int((kernel_to != 0).any(axis=1).sum()) + int((kernel_from != 0).any(axis=1).sum())
             + int((to_e != 0).any(axis=1).sum())
             + int((fr_e != 0).any(axis=1).sum()) + int((fx != 0).any(axis=1).sum()) + len(points)
             + (1 if has_region else 0))
    return {"in_region": inr.astype(np.uint8), "region_entry_edges": sorted(r_entry),
            "region_exit_edges": sorted(r_exit), "map_to": map_to, "map_from": map_from,
            "map_alloc": map_alloc, "kernel_to": kernel_to, "kernel_from": kernel_from, "edge_to": to_e,
            "edge_from": fr_e,
            "exit_from": fx, "acc_point": acc_point, "n_directives": n_dir}


def construct_of(c, v):
    """Table II construct of variable v on the data region's map clause:
    'tofrom', 'to', 'from', 'alloc' or None."""
    w, m = v >> 6, np.uint64(1) << np.uint64(v & 63)
    t, f, a = bool(c["map_to"][w] & m), bool(c["map_from"][w] & m), bool(c["map_alloc"][w] & m)
    return "tofrom" if t and f else "to" if t else "from" if f else "alloc" if a else None
