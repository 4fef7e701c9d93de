#!/usr/bin/env python
"""Benchmark of the host/device validity data-flow on one B300.

Workload: the single large CFG -- 2^20 basic blocks, mean out-degree ~1.3,
loops nested up to 4 deep (~5% back edges), 4096 variables (64 uint64 words
per state per block), ~20% of the blocks in kernel regions, 1-16 accesses
per block (Zipf(1.1) variables, R:W = 70:30); seed 2; synthetic.

One step = the whole analysis: local summaries, anticipation/liveness,
plain host validity, loop masks, device validity, host validity and the
emission of every transfer (per-access flags, edge records, exit
transfers).  The metric is block x variable-word updates per second to
the fixed point: n_blocks * n_words / step time.

  value  -- device time of K steps (CUDA events on the launch stream),
            inputs resident in HBM, state planes (512 MiB each) larger than
            L2 so no flush is needed
  e2e    -- the same metric through ompdart_analyze with host buffers
            (ingestion, host->device copies, solve, device->host copies)
  roofline  -- the dominant kernel (by CUDA-event time) against the
               measured HBM copy bandwidth, plus `step': the whole step's
               modelled bytes over its time
  batch, serve -- the batched (10,000 CFGs) and serving (Poisson 1k-100k
               requests/s) workloads, CFGs/s and p50/p99 beside the plain
               form (one plan and launch sequence per CFG)
  cpu_baseline, clocks, gpu_launches

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

  --workload batch: the 10,000-CFG batch (block counts lognormal, median
  512, clipped 16-65,536; 64/256/1024/2048 variables; seed 3) through
  ompdart_batch_* (arenas per word count, one captured CUDA graph per run),
  beside the plain form that runs one plan per CFG (one launch sequence
  and one wait per CFG); CFGs/s and p50/p99 latency for both.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "block·var-word updates/s to fixed point"
UNIT = "updates/s"
WORKLOAD = "single large CFG: 2^20 blocks, 4096 variables (64 words), seed 2"


def workload_name(n_blocks):
    return WORKLOAD if n_blocks == 1 << 20 else WORKLOAD.replace("2^20", str(n_blocks))


# DRAM traffic per launch from ncu captures (see profiles/):
# dram__bytes_read.sum + dram__bytes_write.sum on the 2^18-block version of
# the workload, scaled to the bench's launch by block-words.  These are
# estimates from an earlier capture, not counters of this run: each entry
# names the commit its capture was taken at, and an entry is removed when
# its kernel changes.
MEASURED_TRAFFIC = {
    "h_summary": {"bytes_2e18": 319.27e6 + 268.16e6,
                  "profile": "profiles/h_summary_walk_2e18.md", "captured_at": "a70e1ed"},
    "live_summary": {"bytes_2e18": (39.0e6 + 365.88e6 + 38.95e6 + 364.84e6) / 2.0,
                     "profile": "profiles/live_summary_walk_2e18.md", "captured_at": "a70e1ed"},
    "emit": {"bytes_2e18": (854.18e6 + 853.99e6 + 854.08e6) / 3.0,
             "profile": "profiles/emit_2e18.md", "captured_at": "a70e1ed"},
}
# DRAM bytes of the batch workload's emission (10,000 CFGs, four arenas),
# per launch averaged over one run's launches: an ncu capture
BATCH_TRAFFIC = {"emit": {"bytes_per_launch": 6772.0e6 / 4, "profile": "profiles/batch_emit_config3.md",
                          "captured_at": "2de5cc9"}}
# a per-phase traffic model for a dense-state design (each phase reading and
# writing whole state planes, no pairs or chunk carries): about 140 B
# per block-word for the whole step (Ant 37, Hp 18, D 19, H 34, emission 32)
DENSE_BYTES_PER_BLOCK_WORD = 140.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic bytes per launch (the design's own traffic model)
# ---------------------------------------------------------------------------

def byte_model(st):
    """Algorithmic DRAM bytes per launch of each kernel of the chunked scan
    solver, from the workload statistics (the design's minimal traffic: each
    structure read once per walk, each dense plane read or written once).
    A chain walk reads per position its 64 B position record, 8 B per edge
    entry and 4 B per access record (`walk`); a dense plane is W words of
    8 B per block; loop-entry edge constants are W words per edge.  The
    emission resolves H_out itself: each position's own pair (two planes),
    kept for the next position, and the pair of every other in-edge's
    source, counted as the in-edges beyond one per position plus one per
    8-position emission item (the positions whose previous one is elsewhere)."""
    N, M, E, A, W, K, L = (st[k] for k in ("N", "M", "E", "A", "W", "K", "L"))
    G = (W + 63) // 64
    plane = 8.0 * W * N
    edge_plane = 8.0 * W * K
    in_loop = 8.0 * W * st["in_loop"]                  # a plane's rows of the blocks inside loops
    hdr = 2 * 8.0 * W * L                               # one header pair per loop
    hdr_top = 2 * 8.0 * W * st["L_top"]
    in_loop2 = 8.0 * W * st.get("in_loop2", 0.0)
    hdr_2 = 3 * 8.0 * W * st.get("L_2", 0)              # a header triple per second-level loop
    walk = G * (M * 64.0 + E * 8.0 + A * 4.0)
    # two pair planes in, one plane out; forward pairs also take the loop
    # tree (a loop id per position and loop, each header pair once)
    resolve = 3 * plane + 8.0 * M
    fwd_resolve = resolve + 4.0 * (M + L) + hdr
    return {
        "local_summary": A * 20.0,                      # access, link in; record, emission word out
        # Live pairs, the header planes inside loops (two levels)
        "live_summary": walk + 2 * plane + in_loop + in_loop2 + hdr_top + hdr_2,
        "live_resolve": resolve + in_loop + in_loop2 + 8.0 * (M + L) + hdr_top + hdr_2,
        "loop_masks": G * st["body"] * (64.0 + 4.0 * A / max(1, M) + 8.0 * E / max(1, M)) + 2 * L * 8.0 * W,
        "hp_summary": walk + 2 * edge_plane + hdr,      # pairs at loop-entry sources, header pairs
        "src_resolve": 4.5 * edge_plane,                # pairs and loop masks in; edge constants (and D) out
        "d_summary": walk + 3 * edge_plane + 2 * plane + hdr,  # reads `to' constants; writes D_in pairs
        "d_resolve": fwd_resolve,
        "h_summary": walk + edge_plane + 4 * plane + hdr,  # reads Live, D_in; writes H_out pairs
        # reads Live, D_in and the H pairs; writes H_in; other sources' H pairs
        "emit": 5 * plane + (max(0, E - M) + M / 8.0) * 16.0 * W + M * 64.0 + E * 16.0 + A * 9.0
                + 3 * edge_plane,
    }


# ---------------------------------------------------------------------------
# clocks during the timed region (NVML reads only)
# ---------------------------------------------------------------------------

class ClockSampler:
    """Polls nvidia-smi (read-only queries) every 100 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.error = None

    def start(self):
        import subprocess
        import tempfile
        self.out = tempfile.TemporaryFile(mode="w+")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception as e:  # noqa: BLE001
            self.error = repr(e)

    def stop(self):
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            res["error"] = self.error
            return res
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        self.out.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        res.update({"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                    "reasons": sorted(reasons), "samples": len(sm)})
        return res


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_sample(g, words):
    import oracle
    from paper_2406_13881_b300 import workload as wl
    oracle.build()
    t_total = 0.0
    for w in words:
        sub, _ = wl.restrict_word(g, w)
        t0 = time.perf_counter()
        oracle.solve(sub, want=["h_in", "d_in", "to_edge", "from_edge", "from_exit", "acc_flag"])
        t_total += time.perf_counter() - t0
    value = g.n_blocks * len(words) / t_total
    return value, t_total


def cpu_info():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    return model


# ---------------------------------------------------------------------------

def job_time_ms(ms, world, device):
    """The timed region of the whole job: the slowest rank's (every rank
    runs the same steps between barriers), via a MAX all-reduce."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(units_per_rank, world, steps, ms):
    """Whole-job throughput: every rank's units over the job's time."""
    return units_per_rank * world * steps / (ms / 1e3)


def loop_entry_edges(g):
    """Loop-entry edges of a generated CFG: every loop header's in-edges
    except its one back edge (the generator's loops have a single latch)."""
    import numpy as np
    heads = np.array([h for h, _, _, _ in g.meta.get("loops", [])], dtype=np.int64)
    if not len(heads):
        return 0
    indeg = np.bincount(np.asarray(g.succ, dtype=np.int64), minlength=g.n_blocks)
    return int((indeg[heads] - 1).sum())


def workload_stats(g):
    W = g.W
    loops = g.meta.get("loops", [])
    st = {"N": g.n_blocks, "M": g.n_blocks, "E": g.n_edges, "A": g.n_acc, "W": W,
          "K": loop_entry_edges(g), "L": len(loops)}
    st["body"] = float(sum(e - f + 1 for _, f, e, _ in loops))
    # blocks inside some loop (the bodies of the outermost loops) and those loops
    st["in_loop"] = float(sum(e - h for h, _, e, d in loops if d == 1))
    st["L_top"] = sum(1 for *_, d in loops if d == 1)
    # the same one level down (liveness closes those loops with a fourth plane)
    st["in_loop2"] = float(sum(e - h for h, _, e, d in loops if d == 2))
    st["L_2"] = sum(1 for *_, d in loops if d == 2)
    return st


def batch_byte_model(cfgs):
    """Algorithmic bytes per run of each kernel name of a batch: the CFGs of
    one word count share an arena (one plan over all of them), whose model
    is byte_model of the summed statistics; summed over the arenas."""
    groups = {}
    for g in cfgs:
        st = workload_stats(g)
        acc = groups.setdefault(st["W"], {k: 0.0 for k in st})
        for k, v in st.items():
            if k != "W":
                acc[k] += v
        acc["W"] = st["W"]
    total = {}
    for st in groups.values():
        for k, v in byte_model(st).items():
            total[k] = total.get(k, 0.0) + v
    return total


def bytes_per_run(timings, model, n_runs, n_plans=1):
    """Modelled bytes of one run per kernel name: the per-launch model
    (summed over the plans of a batch, which share the launch sequence)
    times the launches of that name per plan and run."""
    return {k: model[k] * v[0] / float(n_runs * n_plans) for k, v in timings.items() if k in model}


def dominant_roofline(timings, per_run, n_runs, peak, src, traffic=None, traffic_source=None):
    """The kernel with the most CUDA-event time: its modelled bytes over its
    measured time, against the measured copy bandwidth."""
    name, (nl, tot_ms) = max(timings.items(), key=lambda kv: kv[1][1])
    avg_ms = tot_ms / max(1, nl)
    b = per_run.get(name)
    per_launch = b * n_runs / max(1, nl) if b is not None else None
    achieved = per_launch / (avg_ms / 1e3) / 1e9 if per_launch else None
    total = sum(x[1] for x in timings.values())
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic, "traffic_source": traffic_source,
            "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
            "algorithmic_bytes_per_launch": per_launch, "avg_launch_ms": avg_ms,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 4), "share": round(v[1] / total, 4)}
                        for k, v in sorted(timings.items(), key=lambda kv: -kv[1][1])}}


def step_roofline(timings, per_run, ms_step, peak, units):
    """The whole step: the summed byte model of every modelled kernel per
    step over the step's time, and the dense-state ~140 B per block-word model
    over the same time."""
    modelled = sum(per_run.values())
    dense = DENSE_BYTES_PER_BLOCK_WORD * units
    gbs = lambda b: b / (ms_step / 1e3) / 1e9  # noqa: E731
    return {"bytes_per_step": modelled, "ms_per_step": ms_step, "achieved": gbs(modelled), "peak": peak,
            "unit": "GB/s", "frac": gbs(modelled) / peak,
            "dense_model_bytes_per_step": dense, "dense_model_frac": gbs(dense) / peak,
            "unmodelled_kernels": sorted(k for k in timings if k not in per_run),
            "note": "achieved = modelled bytes per step / ms_per_step of the timed region; 60%% of the measured "
                    "peak on the dense-state model is %.2f ms per step" % (dense / (0.6 * peak * 1e9) * 1e3)}


def single_config(g, seed, world):
    """The `config' object of the single-CFG workload (both arms)."""
    return {"workload": workload_name(g.n_blocks), "n_blocks": g.n_blocks, "n_vars": g.n_vars, "n_words": g.W,
            "n_edges": g.n_edges, "n_acc": g.n_acc, "seed": seed,
            "l2": "no flush: every state plane (%d MiB) is larger than the 126 MB L2" % (8 * g.n_blocks * g.W >> 20),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2406_13881_b300 import _native, build, workload as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    g = wl.single_large(args.seed, n_blocks=args.n_blocks)

    plan = _native.Plan(g, device=local, chunk_target=args.chunk_target)
    if not args.no_graph:
        plan.graph(True)  # the first warm-up run captures the step; the others replay it
    stream = torch.cuda.Stream(device=local)
    sh = stream.cuda_stream
    for _ in range(args.warmup):
        plan.run(sh)
        plan.sync()
    launches_per_step = plan.launches
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.run(sh)
    ev1.record(stream)
    torch.cuda.synchronize()
    plan.sync()
    clk = clocks.stop()
    reruns = plan.view().sweeps
    ms = ev0.elapsed_time(ev1)
    # per-kernel device time: a few more steps with an event before every
    # launch (the phases then run one after another on one stream)
    plan.profile(True)
    n_prof = min(args.steps, 5)
    for _ in range(n_prof):
        plan.run(sh)
        plan.sync()
    timings = plan.timings()
    plan.profile(False)
    ms = job_time_ms(ms, world, "cuda")
    ms_step = ms / args.steps
    units = g.n_blocks * g.W
    value = job_value(units, world, args.steps, ms)

    out = None
    if rank == 0:
        # ---- roofline of the dominant kernel (CUDA events over the timed region)
        st = workload_stats(g)
        model = byte_model(st)
        peak, src = peaks()
        name = max(timings.items(), key=lambda kv: kv[1][1])[0]
        meas = MEASURED_TRAFFIC.get(name)
        traffic = meas["bytes_2e18"] * (g.n_blocks * g.W) / float((1 << 18) * 64) if meas else None
        tsrc = ("estimate, not counters of this run: an ncu capture (commit %s) of the 2^18-block case scaled by "
                "block-words, %s" % (meas["captured_at"], meas["profile"])) if meas else None
        per_run = bytes_per_run(timings, model, n_prof)
        roof = dominant_roofline(timings, per_run, n_prof, peak, src, traffic, tsrc)
        roof["step"] = step_roofline(timings, per_run, ms_step, peak, g.n_blocks * g.W)
        # ---- end to end through the public API with host buffers
        # (one untimed warm-up call, like the batch workload, then the median
        # of e2e_steps calls)
        e2e_t, h2d, d2h = [float("nan")], 0, 0
        if args.e2e_steps:
            e2e_t = []
        for k in range(1 + args.e2e_steps if args.e2e_steps else 0):
            t0 = time.perf_counter()
            r = _native.analyze(g, device=local)
            if k:
                e2e_t.append(time.perf_counter() - t0)
            h2d, d2h = r["h2d_bytes"], r["d2h_bytes"]
            del r  # the caller is done with this step's result before the next
        e2e_s = statistics.median(e2e_t) if args.e2e_steps else None
        # ---- CPU oracle on a bounded sample of word columns
        words = list(range(0, 64, 64 // max(1, args.cpu_words)))[: args.cpu_words]
        cpu_val, cpu_s = oracle_sample(g, words) if words else (None, 0.0)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": single_config(g, args.seed, world),
            "solver": "chunked scan" if plan.view().path == 2 else "sweep",
            "launch": "kernel by kernel" if args.no_graph else "one CUDA graph per step (ompdart_plan_graph)",
            "roofline": roof,
            "cpu_baseline": {"value": cpu_val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d of 64 word columns of the same CFG, single-threaded C oracle, %.1f s"
                                       % (len(words), cpu_s), "cpu": cpu_info()},
            "e2e": {"value": units / e2e_s if e2e_s else None, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "seconds_per_step": e2e_s,
                    "path": "ompdart_analyze: host ingestion + copies + solve + copy back"},
            "gpu_launches": launches_per_step * args.steps,
            "loop_reruns_last_step": reruns,
            "clocks": clk,
        }
    plan.close()
    if out is not None and world == 1 and args.sub_workloads:
        # the same step with the data region and the directives (Table II,
        # Sec. IV-D/IV-F): the classification's cost beside the analysis
        rp = _native.Plan(g, device=local, chunk_target=args.chunk_target, data_region=True)
        for _ in range(3):
            rp.run(sh)
            rp.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_dr = max(3, min(args.steps, 10))
        e0.record(stream)
        for _ in range(n_dr):
            rp.run(sh)
        e1.record(stream)
        torch.cuda.synchronize()
        rp.sync()
        rp.profile(True)
        for _ in range(3):
            rp.run(sh)
            rp.sync()
        tdr = rp.timings()
        rv = rp.fetch()
        rp.close()
        out["directives"] = {
            "ms_per_step": e0.elapsed_time(e1) / n_dr, "steps": n_dr,
            "classify_ms_per_step": tdr.get("classify", (0, 0.0))[1] / 3,
            "region_blocks": int(rv["in_region"].sum()), "kernels": int(rv["kernel_to"].shape[0]),
            "map_to_vars": int(sum(bin(int(x)).count("1") for x in rv["map_to"])),
            "map_from_vars": int(sum(bin(int(x)).count("1") for x in rv["map_from"])),
            "map_alloc_vars": int(sum(bin(int(x)).count("1") for x in rv["map_alloc"])),
            "mode": "opts.data_region: the single target data region's exit rule, then the classification pass"}
        del rv
        # the same step with eager `to' placement (Sec. IV-E, Algorithm 1):
        # the second backward walk and an edge constant on every edge
        ep = _native.Plan(g, device=local, chunk_target=args.chunk_target, eager_to=True)
        for _ in range(3):
            ep.run(sh)
            ep.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_dr):
            ep.run(sh)
        e1.record(stream)
        torch.cuda.synchronize()
        ep.sync()
        ev_ms = e0.elapsed_time(e1) / n_dr
        ev = ep.view()
        out["eager_to"] = {
            "ms_per_step": ev_ms, "steps": n_dr, "value": g.n_blocks * g.W / (ev_ms / 1e3), "unit": UNIT,
            "solver": "chunked scan" if ev.path == 2 else "sweep", "edge_transfer_records": int(ev.n_edge_xfers),
            "mode": "opts.eager_to: device-read must-anticipation, then a `to' on the first edge after the "
                    "producing host write from which every path reads on the device"}
        ep.close()
        # the metric's CFGs/s and p50/p99 part: the batch (10,000 CFGs) and
        # the serving streams, each beside its plain one-plan-per-CFG form
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.e2e_steps = 10, 3, 1
        sub.plain_cfgs, sub.cpu_seconds = args.sub_plain_cfgs, args.sub_cpu_seconds
        sub.seconds, sub.max_requests, sub.plain_requests = 1.0, args.sub_max_requests, args.sub_plain_requests
        bt = measure_batch(sub, local, 1)
        out["batch"] = {k: bt[k] for k in ("value", "unit", "ms_per_step", "steps", "cfgs_per_s", "batch_latency_ms",
                                           "plain_per_cfg", "speedup_vs_plain", "roofline", "e2e", "cpu_baseline",
                                           "cpu_baseline_parallel", "gpu_launches", "config")}
        sv = measure_serve(sub, local)
        out["serve"] = {k: sv[k] for k in ("config", "served", "plain_per_cfg", "resident", "note")}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def percentile(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def run_batch(args):
    """Batched analysis of config-3-shaped CFGs vs one plan per CFG."""
    import torch
    from paper_2406_13881_b300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    out = measure_batch(args, local, world)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out if rank == 0 else None


def measure_batch(args, local, world):
    """The 10,000-CFG batch: graph replays (CUDA events), batch latency,
    per-kernel events for the roofline, the plain form, end to end through
    ompdart_analyze_batch, and the oracle on a sample."""
    import torch
    from paper_2406_13881_b300 import _native, workload as wl

    t0 = time.perf_counter()
    cfgs = wl.batch(args.batch_seed, n_cfgs=args.n_cfgs)
    t_gen = time.perf_counter() - t0
    units = sum(g.n_blocks * g.W for g in cfgs)
    t0 = time.perf_counter()
    b = _native.Batch(cfgs, device=local, tune=args.tune, chunk_target=args.chunk_target)
    t_create = time.perf_counter() - t0
    assert (b.status == 0).all()
    info = b.info()
    stream = torch.cuda.Stream(device=local)
    sh = stream.cuda_stream
    for _ in range(args.warmup):
        b.run(sh)
        assert (b.sync() == 0).all()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for k in range(args.steps):
        b.run(sh)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    b.sync()
    clk = clocks.stop()
    info = b.info()  # launches per run are known once it has run
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    ms = job_time_ms(sum(step_ms), world, "cuda")
    # latency of a batch as the caller sees it: run() to sync() returning
    lat_b = []
    for _ in range(max(3, min(args.steps, 10))):
        t0 = time.perf_counter()
        b.run(sh)
        b.sync()
        lat_b.append(1e3 * (time.perf_counter() - t0))
    # per-kernel CUDA events (arenas one after another on the stream) for the
    # roofline of the batch's dominant kernel
    b.profile(True)
    n_prof = 3
    for _ in range(n_prof):
        b.run(sh)
        b.sync()
    timings = b.timings()
    b.profile(False)
    b.close()
    peak, src = peaks()
    # the byte model covers the chunked scan solver's kernels, which every
    # arena launches once per run (a solo CFG runs the sweep solver's)
    n_plans = max(1, len(info["arenas"]))
    per_run = bytes_per_run(timings, batch_byte_model(cfgs), n_prof, n_plans)
    dom = max(timings.items(), key=lambda kv: kv[1][1])[0] if timings else None
    bt = BATCH_TRAFFIC.get(dom) if (args.n_cfgs == 10000 and args.batch_seed == 3) else None
    roof = dominant_roofline(timings, per_run, n_prof, peak, src, bt["bytes_per_launch"] if bt else None,
                             ("estimate, not counters of this run: an ncu capture (commit %s) of the same batch, "
                              "%s" % (bt["captured_at"], bt["profile"])) if bt else
                             "no DRAM counters of this kernel's batch launch")
    roof["run_under_profile_ms"] = sum(v[1] for v in timings.values()) / n_prof
    roof["note"] = ("per-kernel events serialise the arenas (no graph, no overlap); bytes per kernel from "
                    "byte_model of each arena's summed statistics")
    # ---- the plain form: one plan per CFG, one launch sequence and one wait per CFG
    n_plain = len(cfgs) if args.plain_cfgs <= 0 else min(args.plain_cfgs, len(cfgs))
    plans = [_native.Plan(g, device=local) for g in cfgs[:n_plain]]
    for p in plans[: min(50, n_plain)]:
        p.run(sh)
        p.sync()
    lat_p = []
    t_all = time.perf_counter()
    for p in plans:
        t0 = time.perf_counter()
        p.run(sh)
        p.sync()
        lat_p.append(1e3 * (time.perf_counter() - t0))
    t_all = time.perf_counter() - t_all
    # and all plans enqueued back to back, one wait at the end
    torch.cuda.synchronize()
    t_async = time.perf_counter()
    for p in plans:
        p.run(sh)
    torch.cuda.synchronize()
    t_async = time.perf_counter() - t_async
    plain_launches = sum(p.launches for p in plans)
    for p in plans:
        p.close()
    # ---- end to end: ompdart_analyze_batch with host buffers (one untimed
    # warm-up call, then the median of e2e_steps calls)
    e2e_t = []
    for k in range(1 + max(1, args.e2e_steps)):
        t0 = time.perf_counter()
        res, st = _native.analyze_batch(cfgs, device=local)
        if k:
            e2e_t.append(time.perf_counter() - t0)
        h2d = sum(r["h2d_bytes"] for r in res if r is not None)
        d2h = sum(r["d2h_bytes"] for r in res if r is not None)
        del res
    e2e_s = statistics.median(e2e_t)
    # ---- CPU oracle on a bounded sample of the same CFGs
    import oracle
    oracle.build()
    want = ["h_in", "d_in", "to_edge", "from_edge", "from_exit", "acc_flag"]
    t_cpu, n_cpu, u_cpu = 0.0, 0, 0
    sample = []
    for g in cfgs[:: max(1, len(cfgs) // 400)]:
        t0 = time.perf_counter()
        oracle.solve(g, want=want)
        t_cpu += time.perf_counter() - t0
        n_cpu += 1
        u_cpu += g.n_blocks * g.W
        sample.append(g)
        if t_cpu > args.cpu_seconds:
            break
    # the same sample, one CFG per host thread (the C oracle runs outside the GIL)
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda g: oracle.solve(g, want=want), sample))
    t_par = time.perf_counter() - t0
    value = job_value(units, world, args.steps, ms)
    cps = job_value(len(cfgs), world, args.steps, ms)
    return {
        "metric": "block·var-word updates/s to fixed point; CFGs/s and p50/p99 vs per-CFG launch",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batched: %d independent CFGs, blocks lognormal (median 512, clipped 16-65536), "
                               "variables uniform in {64, 256, 1024, 2048}, seed %d" % (len(cfgs), args.batch_seed),
                   "n_cfgs": len(cfgs), "blocks": int(sum(g.n_blocks for g in cfgs)), "block_words": int(units),
                   "accesses": int(sum(g.n_acc for g in cfgs)), "arenas": info["arenas"], "solo_plans": info["solo"],
                   "autotuned": bool(args.tune),
                   "l2": "no flush: the arenas' state planes (%.1f GB) are larger than the 126 MB L2"
                         % (3 * 8 * units / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "cfgs_per_s": cps,
        "batch_latency_ms": {"p50": percentile(lat_b, 50), "p99": percentile(lat_b, 99),
                             "device_p50": percentile(step_ms, 50), "device_p99": percentile(step_ms, 99),
                             "note": "every CFG of a batch completes with the batch"},
        "plain_per_cfg": {"cfgs": n_plain, "cfgs_per_s": n_plain / t_all, "p50_ms": percentile(lat_p, 50),
                          "p99_ms": percentile(lat_p, 99), "max_ms": max(lat_p),
                          "enqueued_back_to_back_cfgs_per_s": n_plain / t_async,
                          "launches_per_pass": plain_launches,
                          "form": "one ompdart_plan per CFG: plan_run + plan_sync per CFG (latency = their wall time)"},
        "speedup_vs_plain": cps / (n_plain / t_all),
        "host_seconds": {"generate": t_gen, "batch_create": t_create},
        "cpu_baseline": {"value": u_cpu / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "cfgs_per_s": n_cpu / t_cpu,
                         "sample": "%d CFGs (every %d-th), single-threaded C oracle, %.1f s"
                                   % (n_cpu, max(1, len(cfgs) // 400), t_cpu), "cpu": cpu_info()},
        "cpu_baseline_parallel": {"value": u_cpu / t_par, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "cfgs_per_s": n_cpu / t_par,
                                  "sample": "the same %d CFGs, one per host thread on %d threads, %.1f s"
                                            % (n_cpu, cores, t_par)},
        "e2e": {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "seconds_per_step": e2e_s, "cfgs_per_s": len(cfgs) / e2e_s,
                "path": "ompdart_analyze_batch: host ingestion + copies + solve + copy back"},
        "roofline": roof,
        "gpu_launches": info["launches"] * args.steps,
        "clocks": clk,
    }


def serve_pool(seed, n_small, n_large, large_blocks):
    """Request pool of the serving workload: batch-shaped CFGs (lognormal
    blocks, 64-2048 variables) and a few single-large-shaped CFGs (same
    generator parameters, `large_blocks` blocks, 4096 variables)."""
    from paper_2406_13881_b300 import workload as wl
    small = wl.batch(seed, n_cfgs=n_small)
    large = [wl.single_large(seed + 100 + k, n_blocks=large_blocks) for k in range(n_large)]
    return small, large


def run_serve(args):
    """Poisson request streams through the serving loop at several arrival
    rates, beside the plain form (one plan and launch sequence per request)."""
    import torch
    from paper_2406_13881_b300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    out = measure_serve(args, local)
    return out if rank == 0 else None


def measure_serve(args, local):
    import numpy as np
    from paper_2406_13881_b300 import _native

    small, large = serve_pool(args.batch_seed, args.pool, 2, args.large_blocks)
    rng = np.random.default_rng(args.batch_seed)

    def draw(n):
        pick_large = rng.random(n) < args.large_frac
        cfgs = [large[rng.integers(len(large))] if pl else small[rng.integers(len(small))] for pl in pick_large]
        return cfgs

    def one(rate, n, max_batch, max_inflight):
        cfgs = draw(n)
        arrival = np.cumsum(rng.exponential(1e6 / rate, size=n))
        srv = _native.Server(hbm_budget_bytes=args.budget_gb << 30, max_batch=max_batch,
                             max_inflight=max_inflight, device=local)
        t0 = time.perf_counter()
        tickets = srv.replay(cfgs, arrival)
        t_sub = time.perf_counter() - t0
        srv.drain()
        wall = time.perf_counter() - t0
        lats, fails = [], 0
        for t in tickets:
            st, lat, _ = srv.wait(t, want_result=False)
            lats.append(lat)
            fails += st != 0
        stats = srv.stats()
        srv.close()
        units = sum(g.n_blocks * g.W for g in cfgs)
        return {"rate_req_s": rate, "requests": n, "offered_req_s": n / (arrival[-1] / 1e6),
                "submitted_req_s": n / t_sub, "cfgs_per_s": n / wall, "updates_per_s": units / wall,
                "p50_ms": percentile(lats, 50), "p99_ms": percentile(lats, 99), "max_ms": max(lats),
                "failed": int(fails), "batches": stats["batches"], "mean_batch": stats["mean_batch"],
                "peak_device_bytes": stats["peak_bytes"], "wall_s": wall}

    # warm the library (first CUDA context, pool) outside the measurements
    one(1000, 50, 4096, 2)
    served, plain = [], []
    for rate in args.rates:
        n = int(min(args.max_requests, max(200, rate * args.seconds)))
        served.append(one(rate, n, 4096, args.inflight))
        plain.append(one(rate, int(min(n, args.plain_requests)), 1, 1))
    # resident mode: CFGs stay on the device between requests (a plan per
    # distinct CFG, cached by content); one server for every rate, its cache
    # filled with the request pool first (untimed)
    rsrv = _native.Server(hbm_budget_bytes=args.budget_gb << 30, resident=True, workers=args.workers,
                          max_batch=args.group, device=local)
    warm = [rsrv.submit(g) for g in small + large]
    rsrv.drain()
    for t in warm:
        rsrv.wait(t, want_result=False)
    resident = []
    for rate in args.rates:
        n = int(min(args.max_requests, max(200, rate * args.seconds)))
        cfgs = draw(n)
        arrival = np.cumsum(rng.exponential(1e6 / rate, size=n))
        s0 = rsrv.stats()
        t0 = time.perf_counter()
        tickets = rsrv.replay(cfgs, arrival)
        t_sub = time.perf_counter() - t0
        rsrv.drain()
        wall = time.perf_counter() - t0
        lats, fails = [], 0
        for t in tickets:
            st, lat, _ = rsrv.wait(t, want_result=False)
            lats.append(lat)
            fails += st != 0
        s1 = rsrv.stats()
        units = sum(g.n_blocks * g.W for g in cfgs)
        resident.append({"rate_req_s": rate, "requests": n, "offered_req_s": n / (arrival[-1] / 1e6),
                         "submitted_req_s": n / t_sub, "cfgs_per_s": n / wall, "updates_per_s": units / wall,
                         "p50_ms": percentile(lats, 50), "p99_ms": percentile(lats, 99), "max_ms": max(lats),
                         "failed": int(fails), "cache_hits": s1["cache_hits"] - s0["cache_hits"],
                         "cache_misses": s1["cache_misses"] - s0["cache_misses"],
                         "cached_plans": s1["cached_plans"], "device_bytes": s1["bytes_in_use"], "wall_s": wall})
    rsrv.close()
    top = served[-1]
    return {
        "metric": "block·var-word updates/s to fixed point; CFGs/s and p50/p99 vs per-CFG launch",
        "value": top["updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": len(args.rates), "warmup": 1,
        "ms_per_step": 1e3 * top["wall_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": "serving: Poisson request streams of batch-shaped CFGs (lognormal blocks, median 512; "
                               "64-2048 variables) with %.1f%% single-large-shaped CFGs (%d blocks, 4096 variables)"
                               % (100 * args.large_frac, args.large_blocks),
                   "pool": {"small": len(small), "large": len(large)}, "rates_req_s": args.rates,
                   "hbm_budget_gb": args.budget_gb, "max_inflight": args.inflight,
                   "parallelism": "single GPU"},
        "served": served,
        "plain_per_cfg": plain,
        "resident": resident,
        "note": "value = updates/s completed at the highest rate (batched serving); latency = submission to result "
                "on the host; `resident': CFGs kept on the device between requests (plan cache warmed with the "
                "request pool first)",
    }


def run_program(args):
    """The interprocedural workload: a 2,000-function call graph (depth <= 8,
    fan-out 1-6, 32-4,096 blocks, 512 globals + pointer parameters) through
    ompdart_analyze_program (summaries bottom-up, contexts top-down)."""
    import numpy as np
    import torch
    from paper_2406_13881_b300 import _native, build, workload as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    t0 = time.perf_counter()
    p = wl.call_graph(args.program_seed, n_funcs=args.n_funcs)
    t_gen = time.perf_counter() - t0
    for _ in range(args.warmup if args.warmup < 3 else 1):
        _native.analyze_program(p.funcs, p.site_off, p.site_callee, p.var_maps, device=local)
    clocks = ClockSampler(local)
    clocks.start()
    times, out = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = _native.analyze_program(p.funcs, p.site_off, p.site_callee, p.var_maps, device=local)
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    inst = out["instances"]
    units = sum(p.funcs[f].n_blocks * p.funcs[f].W for f, _, _, _ in inst)
    sec = statistics.median(times)
    # CPU oracle: the summaries and a bounded sample of the instances
    import oracle
    oracle.build()
    t_cpu, u_cpu, n_cpu = 0.0, 0, 0
    for f in range(0, len(p.funcs), max(1, len(p.funcs) // 300)):
        t0 = time.perf_counter()
        oracle.solve(p.funcs[f] if p.site_off[f + 1] == p.site_off[f] else _strip_calls(p.funcs[f]))
        t_cpu += time.perf_counter() - t0
        u_cpu += p.funcs[f].n_blocks * p.funcs[f].W
        n_cpu += 1
        if t_cpu > args.cpu_seconds:
            break
    if rank != 0:
        return None
    return {
        "metric": "block·var-word updates/s to fixed point; CFGs/s and p50/p99 vs per-CFG launch",
        "value": units / sec, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": 1e3 * sec, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": "interprocedural: call graph of %d functions (depth <= 8, fan-out 1-6), 32-4096 "
                               "blocks each, 512 globals + pointer parameters, seed %d" % (len(p.funcs),
                                                                                          args.program_seed),
                   "functions": len(p.funcs), "call_sites": int(p.site_off[-1]),
                   "blocks": int(sum(g.n_blocks for g in p.funcs)), "levels": int(out["levels"]),
                   "instances": len(inst), "max_contexts_per_site": 4, "parallelism": "single GPU"},
        "instances_per_s": len(inst) / sec,
        "functions_per_s": len(p.funcs) / sec,
        "seconds": {"generate": t_gen, "analyze_median": sec, "all": times},
        "cpu_baseline": {"value": u_cpu / t_cpu if t_cpu else None, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d functions analysed alone (calls as no-ops), single-threaded C oracle, %.1f s"
                                   % (n_cpu, t_cpu), "cpu": cpu_info()},
        "e2e": {"value": units / sec, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "path": "ompdart_analyze_program: host buffers in, every instance's result on the host"},
        "clocks": clk,
    }


def _strip_calls(g):
    """The function with its call accesses removed (oracle timing only)."""
    import numpy as np
    from paper_2406_13881_b300 import workload as wl
    keep = (np.asarray(g.acc, np.uint32) >> np.uint32(31)) == 0
    blk = np.repeat(np.arange(g.n_blocks), np.diff(g.acc_off))
    ao = np.zeros(g.n_blocks + 1, dtype=np.int32)
    ao[1:] = np.cumsum(np.bincount(blk[keep], minlength=g.n_blocks))
    return wl.CFG(g.n_blocks, g.n_vars, g.entry, g.succ_off, g.succ, ao, np.asarray(g.acc)[keep])


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on the host cores, on
    a bounded sample of the same workload (a few word columns per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from paper_2406_13881_b300 import workload as wl
    g = wl.single_large(args.seed)
    words_per_step = 1
    times = []
    for i in range(args.warmup + args.steps):
        w = (7 * i) % 64
        _, t = oracle_sample(g, [w])
        if i >= args.warmup:
            times.append(t)
    tot = sum(times)
    value = g.n_blocks * words_per_step * len(times) / tot
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": single_config(g, args.seed, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one of 64 word columns of the CFG per step", "cpu": cpu_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-words", type=int, default=8)
    ap.add_argument("--no-graph", action="store_true",
                    help="single workload: launch every kernel of a step instead of replaying one CUDA graph")
    ap.add_argument("--chunk-target", type=int, default=0,
                    help="positions per chunk of the scan solver (0 = the library's choice)")
    ap.add_argument("--n-blocks", type=int, default=1 << 20,
                    help="blocks of the workload (smaller only for profiler captures)")
    ap.add_argument("--workload", choices=["single", "batch", "serve", "program"], default="single")
    ap.add_argument("--n-funcs", type=int, default=2000)
    ap.add_argument("--program-seed", type=int, default=4)
    ap.add_argument("--rates", type=lambda x: [int(v) for v in x.split(",")], default=[1000, 10000, 100000])
    ap.add_argument("--seconds", type=float, default=2.0, help="serve: seconds of arrivals per rate")
    ap.add_argument("--max-requests", type=int, default=100000)
    ap.add_argument("--plain-requests", type=int, default=1500)
    ap.add_argument("--pool", type=int, default=2000)
    ap.add_argument("--large-frac", type=float, default=0.002)
    ap.add_argument("--large-blocks", type=int, default=1 << 16)
    ap.add_argument("--budget-gb", type=int, default=40)
    ap.add_argument("--inflight", type=int, default=2)
    ap.add_argument("--group", type=int, default=0, help="serve: requests a resident worker launches at once (0 = 16)")
    ap.add_argument("--workers", type=int, default=4, help="serve: worker threads of the resident mode")
    ap.add_argument("--n-cfgs", type=int, default=10000, help="CFGs of the batch workload")
    ap.add_argument("--batch-seed", type=int, default=3)
    ap.add_argument("--tune", type=int, default=1, help="batch: autotune the arenas' launch shapes")
    ap.add_argument("--plain-cfgs", type=int, default=0,
                    help="batch: CFGs timed in the one-plan-per-CFG form (0 = all)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--sub-workloads", type=int, default=1,
                    help="single: also run the batch and serving workloads (sub-objects `batch' and `serve')")
    ap.add_argument("--sub-plain-cfgs", type=int, default=2000)
    ap.add_argument("--sub-cpu-seconds", type=float, default=4.0)
    ap.add_argument("--sub-max-requests", type=int, default=20000)
    ap.add_argument("--sub-plain-requests", type=int, default=1000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        out = run_reference(args)
    elif args.workload == "batch":
        out = run_batch(args)
    elif args.workload == "serve":
        out = run_serve(args)
    elif args.workload == "program":
        out = run_program(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
