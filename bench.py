#!/usr/bin/env python3
"""Benchmark of the GB300 HyperBall step.

One bench step is one whole HyperBall computation on the resident graph:
re-initialise the counters (Algorithm 2, first loop), iterate to the
fixpoint (every iteration: frontier, gather + union, estimator and
accumulators), and finalise the four centralities into device buffers.
Setup (outside the timed region, like the degree relabelling): the
light-class sizing of the gather kernel, chosen by the library's
autotuner unless --aps fixes it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Metric: arc-updates per second (arcs scanned by all iterations / time to
fixpoint), plus time to fixpoint and the roofline fraction of the gather
kernel.  The default workload is the largest single graph, the web-like
precision form: R-MAT (0.57, 0.19, 0.19, 0.05) at scale 28 (268,435,456
nodes) with edge factor 16 (2^32 arcs drawn, 4.26G after dedup), int64
offsets, scanned as its transpose, log2m = 4, FP32 estimates and FP64
accumulators.  The encyclopedia-like graph (4,206,785 nodes, 101,355,853
arcs drawn, log2m = 6, FP64) is measured the same way under "secondary",
and a reduced run of the batched and served forms against one graph at a
time under "forms".  Under torchrun each rank runs an independent replica
(weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HyperBall arc-updates/s per step and % HBM roofline; time to fixpoint"
UNIT = "arc-updates/s"

WORKLOADS = {
    "enwiki": dict(log2m=6, seed=42, desc="R-MAT(0.57,0.19,0.19,0.05) scale 23, 4,206,785 nodes, "
                                         "101,355,853 arcs drawn, dedup, transpose scanned, log2m=6"),
    "plain": dict(log2m=4, seed=42, desc="Zipf(2.1) out-degree on {1..1000}, 10,000 nodes, uniform "
                                        "targets, transpose scanned, log2m=4"),
    "web": dict(log2m=4, seed=42, desc="R-MAT scale 28 (268,435,456 nodes), edge factor 16, dedup, "
                                      "transpose scanned, log2m=4, FP32 estimates"),
    "web24": dict(log2m=4, seed=42, desc="R-MAT scale 24 (16,777,216 nodes), edge factor 16, dedup, "
                                        "transpose scanned, log2m=4, FP32 estimates (profiling size)"),
    "web25": dict(log2m=4, seed=42, desc="R-MAT scale 25 (33,554,432 nodes), edge factor 16, dedup, "
                                        "transpose scanned, log2m=4, FP32 estimates (profiling size: "
                                        "counters well above L2)"),
}


def make_graph(name, device):
    from paper_1308_2144_gb300 import graphs
    if name == "enwiki":
        return graphs.enwiki_graph(device=device)
    if name == "plain":
        return graphs.plain_graph(device=device)
    if name == "web":
        return graphs.web_graph(device=device)
    if name == "web24":
        return graphs.web_graph(scale=24, device=device, bucket_bits=2)
    if name == "web25":
        return graphs.web_graph(scale=25, device=device, bucket_bits=3)
    raise ValueError(name)


# ----------------------------------------------------------------- helpers --

class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(workload):
    """DRAM traffic per gather-kernel launch from the committed ncu summary,
    valid only while the kernel source is the one that was profiled."""
    path = os.path.join(ROOT, "profiles", f"step_kernel_{workload}_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if "=" in ln and not ln.startswith("#"):
            k, v = ln.split("=", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != kernel_source_digest():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def recorded_traffic_note(workload):
    """Why no DRAM traffic accompanies this workload's line."""
    path = os.path.join(ROOT, "profiles", f"step_kernel_{workload}_traffic.txt")
    if not os.path.exists(path):
        return (f"no committed capture for this workload (profiles/step_kernel_{workload}_traffic.txt): "
                "a full-size capture exceeds the profiling size rule and its traffic does not scale with "
                "size (the L2 hit rate falls as the counters grow); see the profiling-size captures")
    return "the committed capture was taken on other kernel sources (digest mismatch)"


def kernel_source_digest():
    """sha256 over the sources the gather kernel is compiled from."""
    h = hashlib.sha256()
    for f in ("hb_step.cu", "hb_step_dev.cuh", "hb_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1308_2144_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _all_reduce(x, world, op):
    if world <= 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    import torch.distributed as dist
    return _all_reduce(x, world, dist.ReduceOp.MAX if world > 1 else None)


def sum_over_ranks(x, world):
    import torch.distributed as dist
    return _all_reduce(x, world, dist.ReduceOp.SUM if world > 1 else None)


def replica_throughput(units, ms, world):
    """Whole-job throughput of independent replicas: the units all ranks
    processed divided by the slowest rank's time (weak scaling)."""
    return sum_over_ranks(units, world) / (max_over_ranks(ms, world) / 1e3)


# ------------------------------------------------------------- the oracle --

def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo or lscpu)."""
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _oracle_rows(oracle, off, tgt, log2m, c, rows):
    """One Algorithm 2 iteration (t = 0) of the oracle, as it stands, on the
    first `rows` nodes of the graph (their arcs reach every node's counter
    in c); returns (arc-updates, seconds)."""
    n = off.size - 1
    sumd = np.zeros(n)
    harm = np.zeros(n)
    t0 = time.perf_counter()
    oracle.step(off[:rows + 1], tgt, log2m, 0, c, sumd, harm)
    return int(off[rows] - off[0]), time.perf_counter() - t0


def _sized_rows(oracle, off, tgt, log2m, c, budget_s):
    """A prefix of the rows whose oracle iteration takes about budget_s
    (labels are permuted, so a prefix is a uniform node sample)."""
    n = off.size - 1
    rows = min(n, max(1024, n // 4096))
    arcs, secs = _oracle_rows(oracle, off, tgt, log2m, c, rows)
    while rows < n and secs < 0.25 * budget_s:
        rows = min(n, rows * 4)
        arcs, secs = _oracle_rows(oracle, off, tgt, log2m, c, rows)
    if rows < n and secs > 0:
        rows = int(min(n, max(rows, rows * budget_s / secs)))
    return rows


def cpu_oracle_sample(g_cpu, log2m, seed, budget_s=12.0, budget_one_s=6.0):
    """The oracle, as it stands, on the host cores: one Algorithm 2
    iteration (every sampled node recomputed from all its successors) over a
    prefix of the nodes sized to about budget_s with every thread, and over
    a smaller prefix with one thread."""
    import oracle
    off, tgt = g_cpu
    n = off.size - 1
    c = oracle.init(n, log2m, seed)
    threads = oracle.get_threads()
    rows = _sized_rows(oracle, off, tgt, log2m, c, budget_s)
    arcs, secs = _oracle_rows(oracle, off, tgt, log2m, c, rows)
    oracle.set_threads(1)
    try:
        rows1 = _sized_rows(oracle, off, tgt, log2m, c, budget_one_s)
        arcs1, secs1 = _oracle_rows(oracle, off, tgt, log2m, c, rows1)
    finally:
        oracle.set_threads(0)
    return {"value": arcs / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": f"one Algorithm 2 iteration (t = 0, every sampled node recomputed from all its "
                      f"successors) over the first {rows} of {n} nodes (a uniform sample: labels are "
                      f"permuted): {arcs} arc-updates in {secs:.2f} s on {threads} threads",
            "single_thread": {"value": arcs1 / secs1, "unit": UNIT, "cores": 1,
                              "sample": f"the same iteration over the first {rows1} nodes: {arcs1} "
                                        f"arc-updates in {secs1:.2f} s"}}


# ------------------------------------------------------------------ arms --

def run_reference(args, world, rank):
    """The oracle on the host cores, as it stands: each step is one
    Algorithm 2 iteration over a fixed prefix of the workload's nodes (a
    uniform sample; sized at setup to about --ref-step-s seconds)."""
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    g = make_graph(args.workload, dev)
    off, tgt = g.numpy()
    del g
    import oracle
    n = off.size - 1
    c = oracle.init(n, wl["log2m"], wl["seed"])
    rows = _sized_rows(oracle, off, tgt, wl["log2m"], c, args.ref_step_s)
    secs_all, arcs_all = [], 0
    for k in range(args.warmup + args.steps):
        arcs, dt = _oracle_rows(oracle, off, tgt, wl["log2m"], c, rows)
        if k >= args.warmup:
            secs_all.append(dt)
            arcs_all += arcs
    total = sum(secs_all)
    value = arcs_all / total
    sample = (f"one Algorithm 2 iteration (t = 0, every sampled node recomputed from all its successors) "
              f"over the first {rows} of {n} nodes per step (a uniform sample: labels are permuted)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(secs_all),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "n": int(n), "m": int(tgt.size), "log2m": wl["log2m"],
                   "step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "nproc": os.cpu_count(), "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure(args, name, world, local, stream, with_e2e):
    """One workload on the GPU: setup (graph, handle, tuning), W untimed
    and K timed whole computations, the gather kernel's roofline; returns
    the fields of the JSON line."""
    from paper_1308_2144_gb300 import hyperball as hbl
    wl = WORKLOADS[name]
    fp32 = args.fp32 or name.startswith("web")
    g = make_graph(name, "cuda")
    n, m, log2m = g.n, g.m, wl["log2m"]
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    opts = dict(log2m=log2m, seed=wl["seed"], n=n, fp32=fp32, frontier=args.frontier,
                stream=stream, profile=True, relabel=not args.no_relabel)
    hb = hbl.HyperBall(g.offsets, g.targets, **opts)
    # class sizing and hot range of the gather: part of setup, like the relabelling
    if args.aps == "tune":
        aps = hb.tune()
    else:
        aps = int(args.aps)
        hb.set_class_sizing(aps)
    if args.hot_mib is not None:
        hb.set_hot_nodes((int(args.hot_mib) << 20) >> log2m, args.hot_passes)
    hot, hot_passes = hb.info()["hot_nodes"], hb.info()["hot_passes"]
    cen = {k: torch.empty(n, dtype=torch.float64, device="cuda")
           for k in ("closeness", "harmonic", "lin", "reachable")}

    def one_run(seed):
        hbl.hb_reset(hb._h, seed)
        steps = hbl.hb_run_to_fixpoint(hb._h)
        hbl.hb_get_centralities(hb._h, cen["closeness"], cen["harmonic"], cen["lin"], cen["reachable"])
        return steps, hb.info()

    for k in range(args.warmup):
        one_run(wl["seed"] + k)
    torch.cuda.synchronize()
    if args.trace:
        trace_run(hb, wl["seed"], log2m)
    launches0 = hb.info()["launches"]
    arcs, kms, kbytes, klaunch, steps_list = 0, 0.0, 0.0, 0, []
    pms, pbytes, plaunch = 0.0, 0.0, 0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for k in range(args.steps):
            steps, info = one_run(wl["seed"] + args.warmup + k)
            arcs += info["total_arcs"]
            kms += info["kernel_ms"]
            kbytes += info["kernel_bytes"]
            klaunch += info["kernel_launches"]
            pms += info["push_ms"]
            pbytes += info["push_bytes"]
            plaunch += info["push_launches"]
            steps_list.append(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    launches = hb.info()["launches"] - launches0
    ms_max = max_over_ranks(ms, world)
    value = replica_throughput(arcs, ms, world)

    # roofline of the gather kernel (events recorded by the library on this stream)
    peak, peak_kind = measured_peaks()
    ms_launch = kms / klaunch if klaunch else 0.0
    bytes_launch = kbytes / klaunch if klaunch else 0.0
    achieved = bytes_launch / (ms_launch / 1e3) / 1e9 if klaunch else 0.0
    traffic = recorded_traffic(name)
    dram = traffic / (ms_launch / 1e3) / 1e9 if traffic and ms_launch else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "dram_frac": dram / peak if dram else None,
                "dram_over_algorithmic": traffic / bytes_launch if traffic and bytes_launch else None,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "kernel": "step_kernel (gather + union + estimator; both launches of the two-phase gather)",
                "bytes_per_launch": bytes_launch, "ms_per_launch": ms_launch,
                "launches_timed": klaunch,
                # frontier iterations done by the pushed union (separate kernels)
                "pushed_iterations": {"per_step": plaunch / args.steps,
                                      "ms_per_iteration": pms / plaunch if plaunch else 0.0,
                                      "GBps": pbytes / pms / 1e6 if pms else 0.0}}
    if traffic is None:
        roofline["traffic_note"] = recorded_traffic_note(name)
    out = {
        "value": value, "ms_per_step": ms_max / args.steps, "gpu_launches": launches,
        "config": {"workload": wl["desc"], "n": n, "m": m, "log2m": log2m,
                   "estimate": "fp32" if fp32 else "fp64", "accumulators": "fp64",
                   "frontier": args.frontier, "arcs_per_slot": aps, "hot_nodes": hot,
                   "hot_passes": hot_passes,
                   "gather_tuning": "autotuner" if args.aps == "tune" else "fixed",
                   "iterations_to_fixpoint": steps_list,
                   "arc_updates_per_step": arcs / args.steps,
                   "time_to_fixpoint_ms": ms_max / args.steps,
                   "l2": "inputs larger than L2 (no flush): counters 2 x %.0f MB, targets %.0f MB"
                         % (n * (1 << log2m) / 1e6, m * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roofline, "clocks": clk.summary(),
    }
    if with_e2e:
        out["e2e"] = run_e2e(args, g, opts, wl, world, cen, aps, hot, hot_passes)
    hb.close()
    out["_graph"] = g
    return out


def run_ours(args, world, rank, local):
    from paper_1308_2144_gb300 import build, hyperball as hbl
    build.build()
    hbl.load()
    stream = torch.cuda.current_stream()
    # L2 fetch granularity: a limit of this process's context, put back at the end
    l2_prev = hbl.hb_set_l2_fetch_bytes(args.l2_fetch)
    try:
        _run_ours(args, world, rank, local, stream, l2_prev)
    finally:
        if args.l2_fetch and l2_prev:
            hbl.hb_set_l2_fetch_bytes(l2_prev)


def _run_ours(args, world, rank, local, stream, l2_prev):
    head = measure(args, args.workload, world, local, stream, not args.no_e2e)
    g = head.pop("_graph")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(g.numpy(), WORKLOADS[args.workload]["log2m"], WORKLOADS[args.workload]["seed"])
    del g
    torch.cuda.empty_cache()
    secondary = None
    if args.secondary and args.secondary != args.workload:
        sec = measure(args, args.secondary, world, local, stream, False)
        sec.pop("_graph")
        torch.cuda.empty_cache()
        secondary = {"workload": sec["config"]["workload"], "value": sec["value"], "unit": UNIT,
                     "ms_per_step": sec["ms_per_step"], "config": sec["config"], "roofline": sec["roofline"],
                     "clocks": sec["clocks"]}
    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        from paper_1308_2144_gb300 import bench_forms
        forms = bench_forms.forms_summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": head["config"], "roofline": head["roofline"], "cpu_baseline": cpu,
            "e2e": head.get("e2e"), "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
            "secondary": secondary, "forms": forms,
        }
        line["config"]["l2_fetch_bytes"] = args.l2_fetch or l2_prev
        print(json.dumps(line), flush=True)


def trace_run(hb, seed, log2m):
    """One run, iteration by iteration, to stderr (diagnostics)."""
    from paper_1308_2144_gb300 import hyperball as hbl
    hbl.hb_reset(hb._h, seed)
    prev_ms = prev_b = 0.0
    while True:
        k = hb.step()
        info = hb.info()
        ms = info["kernel_ms"] + info["push_ms"] - prev_ms
        by = info["kernel_bytes"] + info["push_bytes"] - prev_b
        prev_ms, prev_b = info["kernel_ms"] + info["push_ms"], info["kernel_bytes"] + info["push_bytes"]
        print(json.dumps({"t": info["t"] - 1, "sparse": info["last_sparse"], "nodes": info["last_nodes"],
                          "arcs": info["last_arcs"], "changed": k, "kernel_ms": round(ms, 4),
                          "GBps": round(by / ms / 1e6, 1) if ms > 0 else None}), file=sys.stderr,
              flush=True)
        if k == 0:
            break


def run_e2e(args, g, opts, wl, world, cen, aps, hot, hot_passes):
    """Same metric through the public API from host memory: pinned host CSR
    in, handle created (upload + setup) with the class sizing and hot range
    chosen above given at creation (hb_options.arcs_per_slot, hot_nodes,
    hot_passes),
    run to the fixpoint, centralities back to pinned host memory, handle
    destroyed, every step; one untimed step first."""
    from paper_1308_2144_gb300 import hyperball as hbl
    n = g.n
    off_h = g.offsets.cpu().pin_memory()
    tgt_h = g.targets.cpu().pin_memory()
    outs_h = {k: torch.empty(n, dtype=torch.float64).pin_memory() for k in cen}
    e2e_steps = max(1, min(args.steps, 5))
    e2e_arcs = 0
    opts_h = dict(opts)
    opts_h.pop("profile")

    phases = {"create": [], "run": [], "results": [], "destroy": []}

    def one(seed):
        # every call below returns once its device work is done
        t_a = time.perf_counter()
        h = hbl.HyperBall(off_h, tgt_h, **dict(opts_h, seed=seed, arcs_per_slot=aps, hot_nodes=hot,
                                                   hot_passes=hot_passes))
        t_b = time.perf_counter()
        h.run()
        t_c = time.perf_counter()
        hbl.hb_get_centralities(h._h, outs_h["closeness"], outs_h["harmonic"], outs_h["lin"],
                                outs_h["reachable"])
        t_d = time.perf_counter()
        arcs = h.info()["total_arcs"]
        h.close()
        t_e = time.perf_counter()
        for k_, (x, y) in zip(phases, ((t_a, t_b), (t_b, t_c), (t_c, t_d), (t_d, t_e))):
            phases[k_].append(1e3 * (y - x))
        return arcs

    # one untimed pass first, as for the device-resident steps: the first
    # handle of a process grows the library's memory pool
    one(wl["seed"] + 99)
    for v in phases.values():
        v.clear()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        e2e_arcs += one(wl["seed"] + 100 + k)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_val = sum_over_ranks(e2e_arcs, world) / e2e_s
    h2d = off_h.numel() * off_h.element_size() + tgt_h.numel() * tgt_h.element_size()
    d2h = 4 * n * 8
    return {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s / e2e_steps,
            "phase_ms_median": {k: round(statistics.median(v), 1) for k, v in phases.items() if v}}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="web")
    ap.add_argument("--secondary", choices=sorted(WORKLOADS) + [""], default="enwiki",
                    help="a second workload measured the same way and reported under 'secondary' "
                         "('' for none)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the reduced batched and served measurement ('forms')")
    ap.add_argument("--hot-mib", type=int, default=None,
                    help="fix the gather's hot range (MiB of counters; 0 = none) instead of the "
                         "autotuner's choice")
    ap.add_argument("--hot-passes", type=int, choices=[1, 2], default=1,
                    help="with --hot-mib: one pass with L2 priorities (1) or the two-phase gather (2)")
    ap.add_argument("--l2-fetch", type=int, choices=[0, 32, 64, 128], default=128,
                    help="L2 fetch granularity of this process's context while it runs (0: leave it)")
    ap.add_argument("--ref-step-s", type=float, default=1.5,
                    help="--impl reference: seconds of oracle work per step")
    ap.add_argument("--frontier", choices=["auto", "push", "pull", "off"], default="auto")
    ap.add_argument("--fp32", action="store_true", help="precision form (FP32 estimates)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-relabel", action="store_true", help="keep the generator's node order")
    ap.add_argument("--trace", action="store_true", help="per-iteration diagnostics on stderr")
    ap.add_argument("--aps", choices=["1", "2", "4", "8", "16", "32", "64", "128", "tune"], default="tune",
                    help="light-class sizing (arcs per slot), or 'tune' for the autotuner")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
