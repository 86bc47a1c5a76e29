#!/usr/bin/env python3
"""Measurements of the batched and served forms against one-graph-at-a-time
runs on the same GPU.

    python -m paper_1308_2144_gb300.bench_forms batch [--graphs 512]
    python -m paper_1308_2144_gb300.bench_forms serve [--rate 200 --seconds 60 --warm 10]
    python -m paper_1308_2144_gb300.bench_forms runs [--runs 16]
    python -m paper_1308_2144_gb300.bench_forms packed [--graph enwiki --log2m 6]
    python -m paper_1308_2144_gb300.bench_forms switch [--graph web]

batch: independent R-MAT graphs (0.57, 0.19, 0.19, 0.05) with node counts
log-uniform in [1e3, 2e6], edge factor uniform in 4..32, log2m uniform in
{4, 5, 6, 7}, seeds 1000+i, scanned as transposes.  All advanced together
(hb_batch_run: one CUDA-graph launch to every fixpoint) versus
hb_run_to_fixpoint on each graph in turn.  Prints one JSON line: time to
all-fixpoint for both, aggregate arc-updates/s, speedup.

serve: a pool of R-MAT graphs (node counts log-uniform in [1e4, 2e7], edge
factor 16), requests arriving as a Poisson stream (graph uniform from the
pool, log2m 4 or 6, seed = request id).  The continuous-batching server
(many slots) with at most --large-slots requests on graphs of the pool's top
quarter by arcs running at once, the same server without that limit, and
the server with one slot (a FIFO one at a time), on the same arrival
stream.  Prints one JSON line per server: p50/p99 latency from arrival to
results in host memory, and arc-updates/s.

runs: the paper's multiple runs (Sec. 5) on the encyclopedia-like graph
(log2m 6): R runs with seeds 42..42+R-1, each to its fixpoint, then the
per-node mean and standard deviation of all four centralities, three ways:
one handle whose rows hold every run (hb_create_runs), a batch of R runs
sharing one copy of the graph (hb_batch_create_runs), and the R runs one
after the other on one handle (statistics of the R results with torch).
Prints one JSON line: time of each, and arc-updates/s counted per run (the
arcs each run scans, summed over the runs).

packed: registers held in six bits (HB_PACKED_REGISTERS, Sec. 4.1 register
width) against byte registers on one graph (encyclopedia-like, or web-like
at scale 25 or 28, scanned as transposes): both with every node recomputed
at every iteration (HB_FRONTIER_OFF, the packed form's policy), and byte
registers with the default frontier policy for context.  Each arm runs
--repeat times from t = 0 to its fixpoint (best time kept); every arm must
end with the same accumulators, else the line says so.  Prints one JSON
line: per arm the time to the fixpoint, iterations, arc-updates/s, the
gather kernel's mean duration and algorithmic GB/s (CUDA events,
HB_PROFILE), and the bytes of the counters.

switch: the frontier switch of HB_FRONTIER_AUTO (hb_set_frontier_switch:
push when the arcs to push are at most that fraction of m, else recompute
every node) on one graph with the gather options the autotuner picks for it
(web-like: 16 arcs per slot, one pass with L2 priorities for the hot 64 MiB,
128-byte L2 fetches; encyclopedia-like: 128 arcs per slot).  For each
fraction, the best of --repeat runs from t = 0 to the fixpoint, then one run
iteration by iteration (synchronised after each) for the per-iteration mode,
arcs and time.  Every fraction must end with the same accumulators.  Prints
one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1308_2144_gb300 import build, graphs  # noqa: E402
from paper_1308_2144_gb300 import hyperball as hbl  # noqa: E402


def _rmat(n, ef, seed):
    scale = max(4, int(np.ceil(np.log2(max(n, 2)))))
    return graphs.rmat_graph(scale=scale, edge_factor=ef, seed=seed, n=n, device="cuda")


def batch_main(args):
    print(json.dumps(batch_measure(args)), flush=True)


def batch_measure(args) -> dict:
    rng = np.random.default_rng(args.seed)
    mix = []
    t0 = time.time()
    for i in range(args.graphs):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(args.max_n))))
        ef = int(rng.integers(4, 33))
        b = int(rng.choice([4, 5, 6, 7]))
        mix.append((_rmat(n, ef, 1000 + i), b, 1000 + i))
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    arcs_total = sum(g.m for g, _, _ in mix)
    descs = [(g.offsets, g.targets, g.n, b, s) for g, b, s in mix]
    t0 = time.time()
    batch = hbl.HyperBallBatch(descs, fp32=args.fp32)
    create_s = time.time() - t0
    batch.run()
    times = []
    for _ in range(args.repeat):
        batch.reset()
        torch.cuda.synchronize()
        t = time.perf_counter()
        iters = batch.run()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    _, _, arcs = batch.totals()
    batch.close()
    solos = [hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=s, n=g.n, fp32=args.fp32) for g, b, s in mix]
    solo_times = []
    solo_arcs = 0
    for r in range(args.repeat):
        for (g, b, s), h in zip(mix, solos):
            hbl.hb_reset(h._h, s)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for h in solos:
            h.run()
        torch.cuda.synchronize()
        solo_times.append(time.perf_counter() - t)
        solo_arcs = sum(h.info()["total_arcs"] for h in solos)
    for h in solos:
        h.close()
    bt, st = min(times), min(solo_times)
    return {
        "form": "batched", "graphs": args.graphs, "arcs_in_graphs": arcs_total,
        "batch_ms": round(1e3 * bt, 3), "batch_iterations": iters, "arc_updates": arcs,
        "batch_arc_updates_per_s": arcs / bt, "one_at_a_time_ms": round(1e3 * st, 3),
        "one_at_a_time_arc_updates_per_s": solo_arcs / st, "speedup": st / bt,
        "estimate": "fp32" if args.fp32 else "fp64", "generate_s": round(gen_s, 1),
        "create_s": round(create_s, 1)}


def serve_run(pool, args, slots, label, large_slots=0, large_arcs=None):
    srv = hbl.HyperBallServer(slots=slots, fp32=args.fp32, reserve_bytes=args.reserve_gb << 30,
                              large_slots=large_slots, large_arcs=large_arcs)
    gids = [srv.add_graph(g.offsets, g.targets, g.n, log2ms=(4, 6)) for g in pool]
    rng = np.random.default_rng(args.seed + 7)
    total = args.warm + args.seconds
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=int(args.rate * total * 1.2) + 10))
    arrivals = arrivals[arrivals < total]
    jobs = [(float(a), int(rng.integers(0, len(pool))), int(rng.choice([4, 6]))) for a in arrivals]
    rids = [None] * len(jobs)
    submit_wall = [0.0] * len(jobs)
    lat = [None] * len(jobs)
    done_wall = [0.0] * len(jobs)
    infos = [None] * len(jobs)
    start = time.perf_counter()

    def producer():
        for j, (at, gi, b) in enumerate(jobs):
            now = time.perf_counter() - start
            if at > now:
                time.sleep(at - now)
            submit_wall[j] = time.perf_counter() - start
            rids[j] = srv.submit(gids[gi], b, j + 1)

    nmax = max(g.n for g in pool)
    pinned = torch.empty((4, nmax), dtype=torch.float64).pin_memory()

    def consumer():
        for j in range(len(jobs)):
            while rids[j] is None:
                time.sleep(0.0005)
            info = srv.wait(rids[j], timeout=-1)
            n = pool[jobs[j][1]].n
            srv.take(rids[j], n, out={k: pinned[q, :n] for q, k in
                                      enumerate(("closeness", "harmonic", "lin", "reachable"))})
            done_wall[j] = time.perf_counter() - start
            lat[j] = done_wall[j] - jobs[j][0]
            infos[j] = info

    tp = threading.Thread(target=producer)
    tc = threading.Thread(target=consumer)
    tp.start()
    tc.start()
    tp.join()
    tc.join()
    end = time.perf_counter() - start
    srv.close()
    sel = [j for j in range(len(jobs)) if jobs[j][0] >= args.warm]
    L = np.array([lat[j] for j in sel])
    arcs = sum(infos[j]["arcs"] for j in sel)
    window = max(done_wall[j] for j in sel) - args.warm
    # latency by request size: graphs in the top quarter of the pool by arcs
    big_m = np.quantile([g.m for g in pool], 0.75)
    big = np.array([pool[jobs[j][1]].m >= big_m for j in sel])
    by_size = {}
    for key, mask in (("large_quarter", big), ("rest", ~big)):
        if mask.any():
            by_size[key] = {"requests": int(mask.sum()), "p50_s": float(np.percentile(L[mask], 50)),
                            "p99_s": float(np.percentile(L[mask], 99))}
    return {"form": "served", "server": label, "slots": slots, "large_slots": large_slots,
            "large_arcs": large_arcs, "rate_per_s": args.rate,
            "requests": len(sel), "p50_latency_s": float(np.percentile(L, 50)),
            "p99_latency_s": float(np.percentile(L, 99)), "mean_latency_s": float(L.mean()),
            "latency_by_size": by_size,
            "arc_updates_per_s": arcs / window, "drain_s": round(end - total, 2),
            "estimate": "fp32" if args.fp32 else "fp64", "pool_graphs": len(pool),
            "pool_arcs": int(sum(g.m for g in pool))}


def serve_pool(args):
    rng = np.random.default_rng(args.seed)
    pool = []
    t0 = time.time()
    for i in range(args.pool):
        n = int(np.exp(rng.uniform(np.log(1e4), np.log(args.max_n))))
        pool.append(_rmat(n, 16, 5000 + i))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return pool, time.time() - t0


def serve_measure(args) -> list:
    """On the same arrival stream over the same pool: the continuous-batching
    server with at most one large request running (large: a graph in the
    top quarter of the pool by arcs), the same server without that limit,
    and the FIFO one-at-a-time server."""
    pool, gen_s = serve_pool(args)
    large = int(np.quantile([g.m for g in pool], 0.75))
    out = []
    for slots, label, ls in ((args.slots, "continuous-batching-size-aware", args.large_slots),
                             (args.slots, "continuous-batching", 0), (1, "fifo-one-at-a-time", 0)):
        r = serve_run(pool, args, slots, label, large_slots=ls, large_arcs=large if ls else None)
        r["generate_s"] = round(gen_s, 1)
        out.append(r)
    return out


def serve_main(args):
    for r in serve_measure(args):
        print(json.dumps(r), flush=True)


def forms_summary(graphs=64, rate=200.0, seconds=8.0, warm=2.0, pool=16, fp32=False) -> dict:
    """A reduced run of both forms for the benchmark line: a batch of
    `graphs` graphs of the batched mix against one graph at a time, and
    both servers at `rate` requests/s over a pool of `pool` graphs."""
    ba = argparse.Namespace(graphs=graphs, max_n=2e6, repeat=3, seed=4, fp32=fp32)
    sa = argparse.Namespace(pool=pool, max_n=2e7, rate=rate, seconds=seconds, warm=warm, slots=32,
                            reserve_gb=8, seed=5, fp32=fp32, large_slots=1)
    batched = batch_measure(ba)
    served = serve_measure(sa)
    cb, cb_plain, fifo = served
    keep = ("requests", "p50_latency_s", "p99_latency_s", "arc_updates_per_s", "latency_by_size")
    return {
        "batched": {k: batched[k] for k in ("graphs", "arcs_in_graphs", "batch_ms", "one_at_a_time_ms",
                                            "speedup", "batch_arc_updates_per_s", "estimate")},
        "served": {"rate_per_s": rate, "seconds": seconds, "pool_graphs": pool,
                   "continuous_batching": dict({k: cb[k] for k in keep}, large_slots=cb["large_slots"],
                                               large_arcs=cb["large_arcs"]),
                   "continuous_batching_no_large_limit": {k: cb_plain[k] for k in keep},
                   "fifo_one_at_a_time": {k: fifo[k] for k in keep},
                   "p50_ratio_fifo_over_batching": fifo["p50_latency_s"] / cb["p50_latency_s"],
                   "p99_ratio_fifo_over_batching": fifo["p99_latency_s"] / cb["p99_latency_s"]},
    }


def runs_main(args):
    if args.graph == "web":
        g = graphs.web_graph(device="cuda")
        b, args.fp32 = 4, True
        desc = "web-like (R-MAT scale 28, 268,435,456 nodes, edge factor 16), transpose, log2m 4, FP32 estimates"
    elif args.graph == "web25":
        g = graphs.web_graph(scale=25, device="cuda", bucket_bits=3)
        b, args.fp32 = 4, True
        desc = "web-like at profiling size (R-MAT scale 25, 33,554,432 nodes, edge factor 16), transpose, log2m 4, FP32"
    else:
        g = graphs.enwiki_graph(device="cuda")
        b = 6
        desc = "encyclopedia-like (R-MAT scale 23, 4,206,785 nodes), transpose, log2m 6"
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    n = g.n
    seeds = [42 + r for r in range(args.runs)]
    names = hbl.HyperBallBatch.CENTRALITIES
    lib = hbl.load()
    out = {k: (torch.empty(n, dtype=torch.float64, device="cuda"),
               torch.empty(n, dtype=torch.float64, device="cuda")) for k in names}

    # one handle whose rows hold every run (hb_create_runs)
    wide = hbl.HyperBall.runs(g.offsets, g.targets, b, seeds, n=n, fp32=args.fp32)

    def one_handle():
        hbl.hb_reset(wide._h, 0)
        wide.run()
        for w, k in enumerate(names):
            hbl._check(lib.hb_get_run_stats(wide._h, w, hbl._ptr(out[k][0]), hbl._ptr(out[k][1])))
        return wide.info()["total_arcs"], wide.info()["t"]

    # a batch of R runs sharing one copy of the graph (hb_batch_create_runs);
    # left out on the web-like graph, where it would hold a further copy of
    # every run's state and adds nothing to the comparison
    batch = None
    if not args.graph.startswith("web"):
        batch = hbl.HyperBallBatch.runs(g.offsets, g.targets, n, b, seeds, fp32=args.fp32)

    def batched():
        batch.reset(seeds)
        iters = batch.run()
        for w, k in enumerate(names):
            hbl._check(lib.hb_batch_get_run_stats(batch._h, w, hbl._ptr(out[k][0]), hbl._ptr(out[k][1])))
        return batch.totals()[2], iters

    # the same runs one after the other on one handle, statistics with torch
    solo = hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=seeds[0], n=n, fp32=args.fp32)
    vals = torch.empty((4, args.runs, n), dtype=torch.float64, device="cuda")

    def one_at_a_time():
        arcs = 0
        for r, s in enumerate(seeds):
            hbl.hb_reset(solo._h, s)
            solo.run()
            hbl.hb_get_centralities(solo._h, vals[0, r], vals[1, r], vals[2, r], vals[3, r])
            arcs += solo.info()["total_arcs"]
        torch.std_mean(vals, dim=1)
        return arcs, None

    arms = {"one_handle": one_handle, "batch": batched, "one_at_a_time": one_at_a_time}
    if batch is None:
        del arms["batch"]
    best = {k: float("inf") for k in arms}
    work = {}
    for f in arms.values():
        f()
    for _ in range(args.repeat):
        for k, f in arms.items():
            torch.cuda.synchronize()
            t = time.perf_counter()
            work[k] = f()
            torch.cuda.synchronize()
            best[k] = min(best[k], time.perf_counter() - t)
    wide.close()
    if batch is not None:
        batch.close()
    solo.close()
    # arc-updates: arcs scanned per run summed over the runs (the one-handle
    # form scans each arc once for all runs of a row)
    solo_arcs = work["one_at_a_time"][0]
    line = {"form": "runs", "graph": desc,
            "runs": args.runs, "n": n, "m": g.m, "estimate": "fp32" if args.fp32 else "fp64",
            "includes": "all runs to their fixpoints and the per-node mean and std of the four centralities"}
    for k in arms:
        line[f"{k}_ms"] = round(1e3 * best[k], 3)
        line[f"{k}_run_arc_updates_per_s"] = solo_arcs / best[k]
    line["one_handle_iterations"] = work["one_handle"][1]
    line["one_handle_speedup"] = best["one_at_a_time"] / best["one_handle"]
    if "batch" in arms:
        line["batch_iterations"] = work["batch"][1]
        line["batch_speedup"] = best["one_at_a_time"] / best["batch"]
    print(json.dumps(line), flush=True)


def packed_main(args):
    if args.graph == "web":
        g = graphs.web_graph(device="cuda")
        desc = "web-like (R-MAT scale 28, 268,435,456 nodes, edge factor 16), transpose"
    elif args.graph == "web25":
        g = graphs.web_graph(scale=25, device="cuda", bucket_bits=3)
        desc = "web-like at profiling size (R-MAT scale 25, 33,554,432 nodes, edge factor 16), transpose"
    else:
        g = graphs.enwiki_graph(device="cuda")
        desc = "encyclopedia-like (R-MAT scale 23, 4,206,785 nodes), transpose"
    b = args.log2m
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    arms = {"byte_off": dict(frontier="off"), "packed_off": dict(frontier="off", packed=True),
            "byte_auto": dict(frontier="auto")}
    line = {"form": "packed", "graph": desc, "n": g.n, "m": g.m, "log2m": b,
            "estimate": "fp32" if args.fp32 else "fp64"}
    ref_acc = None
    identical = True
    for name, opts in arms.items():
        h = hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=42, n=g.n, fp32=args.fp32, profile=True, **opts)
        h.run()                                   # warm-up
        best, info = float("inf"), None
        for _ in range(args.repeat):
            h.reset(42)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.run()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if dt < best:
                best, info = dt, h.info()
        acc = h.accumulators()
        if ref_acc is None:
            ref_acc = acc
        else:
            identical &= all(torch.equal(x, y) for x, y in zip(acc, ref_acc))
        del acc
        h.close()
        torch.cuda.empty_cache()
        line[f"{name}_ms"] = round(1e3 * best, 3)
        line[f"{name}_iterations"] = info["t"]
        line[f"{name}_arc_updates_per_s"] = info["total_arcs"] / best
        if info["kernel_launches"]:
            line[f"{name}_gather_ms"] = round(info["kernel_ms"] / info["kernel_launches"], 4)
            line[f"{name}_gather_gbs"] = round(info["kernel_bytes"] / (1e6 * info["kernel_ms"]), 1)
        line[f"{name}_counter_bytes"] = g.n * ((3 << b) // 4 if opts.get("packed") else 1 << b)
    line["identical_accumulators"] = bool(identical)
    line["packed_speedup_vs_byte_off"] = line["byte_off_ms"] / line["packed_off_ms"]
    print(json.dumps(line), flush=True)


def _bench_graph(name):
    if name == "web":
        return graphs.web_graph(device="cuda"), 4, True, 16, 64, \
            "web-like (R-MAT scale 28, 268,435,456 nodes, edge factor 16), transpose, log2m 4, FP32"
    if name == "web25":
        return graphs.web_graph(scale=25, device="cuda", bucket_bits=3), 4, True, 16, 64, \
            "web-like at profiling size (R-MAT scale 25, 33,554,432 nodes), transpose, log2m 4, FP32"
    return graphs.enwiki_graph(device="cuda"), 6, False, 128, 0, \
        "encyclopedia-like (R-MAT scale 23, 4,206,785 nodes), transpose, log2m 6, FP64"


def switch_main(args):
    g, b, fp32, aps, hot_mib, desc = _bench_graph(args.graph)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    prev = hbl.hb_set_l2_fetch_bytes(128)
    h = hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=42, n=g.n, fp32=fp32, arcs_per_slot=aps,
                      hot_nodes=(hot_mib << 20) >> b, hot_passes=1)
    line = {"form": "switch", "graph": desc, "n": g.n, "m": g.m, "arcs_per_slot": aps, "hot_mib": hot_mib}
    ref_acc, identical, rows = None, True, []
    for frac in args.fracs:
        h.set_frontier_switch(frac)
        h.reset(42)
        h.run()                                   # warm-up
        best = float("inf")
        for _ in range(args.repeat):
            h.reset(42)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.run()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        arcs = h.info()["total_arcs"]
        acc = h.accumulators()
        if ref_acc is None:
            ref_acc = acc
        else:
            identical &= all(torch.equal(x, y) for x, y in zip(acc, ref_acc))
        del acc
        h.reset(42)
        its = []
        while True:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            k = h.step()
            torch.cuda.synchronize()
            inf = h.info()
            its.append(["push" if inf["last_sparse"] else "dense", inf["last_arcs"],
                        round(1e3 * (time.perf_counter() - t0), 3)])
            if k == 0:
                break
        rows.append({"frac": frac, "ms": round(1e3 * best, 3), "iterations": len(its),
                     "arc_updates_per_s": arcs / best, "per_iteration": its})
    h.close()
    hbl.hb_set_l2_fetch_bytes(prev)
    line["identical_accumulators"] = bool(identical)
    line["fracs"] = rows
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("batch")
    b.add_argument("--graphs", type=int, default=512)
    b.add_argument("--max-n", type=float, default=2e6)
    b.add_argument("--repeat", type=int, default=3)
    b.add_argument("--seed", type=int, default=4)
    b.add_argument("--fp32", action="store_true")
    s = sub.add_parser("serve")
    s.add_argument("--pool", type=int, default=64)
    s.add_argument("--max-n", type=float, default=2e7)
    s.add_argument("--rate", type=float, default=200.0)
    s.add_argument("--seconds", type=float, default=60.0)
    s.add_argument("--warm", type=float, default=10.0)
    s.add_argument("--slots", type=int, default=32)
    s.add_argument("--large-slots", type=int, default=1,
                   help="large requests running at once in the size-aware server")
    s.add_argument("--reserve-gb", type=int, default=8)
    s.add_argument("--seed", type=int, default=5)
    s.add_argument("--fp32", action="store_true")
    r = sub.add_parser("runs")
    r.add_argument("--runs", type=int, default=16)
    r.add_argument("--graph", choices=["enwiki", "web", "web25"], default="enwiki")
    r.add_argument("--repeat", type=int, default=3)
    r.add_argument("--fp32", action="store_true")
    k = sub.add_parser("packed")
    k.add_argument("--graph", choices=["enwiki", "web", "web25"], default="enwiki")
    k.add_argument("--log2m", type=int, default=6)
    k.add_argument("--repeat", type=int, default=3)
    k.add_argument("--fp32", action="store_true")
    w = sub.add_parser("switch")
    w.add_argument("--graph", choices=["enwiki", "web", "web25"], default="web")
    w.add_argument("--fracs", type=float, nargs="+", default=[0.0625, 0.125, 0.25, 0.5, 1.0, 2.0])
    w.add_argument("--repeat", type=int, default=3)
    args = ap.parse_args()
    build.build()
    hbl.load()
    {"batch": batch_main, "serve": serve_main, "runs": runs_main, "packed": packed_main,
     "switch": switch_main}[args.cmd](args)


if __name__ == "__main__":
    main()
