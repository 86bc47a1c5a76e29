#!/usr/bin/env python3
"""Measurements of the batched and served forms against one-graph-at-a-time
runs on the same GPU.

    python -m paper_1308_2144_gb300.bench_forms batch [--graphs 512]
    python -m paper_1308_2144_gb300.bench_forms serve [--rate 200 --seconds 60 --warm 10]
    python -m paper_1308_2144_gb300.bench_forms runs [--runs 16]

batch: independent R-MAT graphs (0.57, 0.19, 0.19, 0.05) with node counts
log-uniform in [1e3, 2e6], edge factor uniform in 4..32, log2m uniform in
{4, 5, 6, 7}, seeds 1000+i, scanned as transposes.  All advanced together
(hb_batch_run: one CUDA-graph launch to every fixpoint) versus
hb_run_to_fixpoint on each graph in turn.  Prints one JSON line: time to
all-fixpoint for both, aggregate arc-updates/s, speedup.

serve: a pool of R-MAT graphs (node counts log-uniform in [1e4, 2e7], edge
factor 16), requests arriving as a Poisson stream (graph uniform from the
pool, log2m 4 or 6, seed = request id).  The continuous-batching server
(many slots) versus the same server with one slot (a FIFO one at a time),
on the same arrival stream.  Prints one JSON line per server: p50/p99
latency from arrival to results in host memory, and arc-updates/s.

runs: the paper's multiple runs (Sec. 5) on the encyclopedia-like graph
(log2m 6): R runs with seeds 42..42+R-1 in one batch sharing one copy of the
graph (hb_batch_create_runs, hb_batch_run), then the per-node mean and
standard deviation of all four centralities, versus the same R runs one
after the other on one handle (hb_reset, hb_run_to_fixpoint,
hb_get_centralities, statistics of the R results on the GPU).  Prints one
JSON line: time for all R runs and their statistics both ways, and
arc-updates/s.
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
    print(json.dumps({
        "form": "batched", "graphs": args.graphs, "arcs_in_graphs": arcs_total,
        "batch_ms": round(1e3 * bt, 3), "batch_iterations": iters, "arc_updates": arcs,
        "batch_arc_updates_per_s": arcs / bt, "one_at_a_time_ms": round(1e3 * st, 3),
        "one_at_a_time_arc_updates_per_s": solo_arcs / st, "speedup": st / bt,
        "estimate": "fp32" if args.fp32 else "fp64", "generate_s": round(gen_s, 1),
        "create_s": round(create_s, 1)}), flush=True)


def serve_run(pool, args, slots, label):
    srv = hbl.HyperBallServer(slots=slots, fp32=args.fp32, reserve_bytes=args.reserve_gb << 30)
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
    return {"form": "served", "server": label, "slots": slots, "rate_per_s": args.rate,
            "requests": len(sel), "p50_latency_s": float(np.percentile(L, 50)),
            "p99_latency_s": float(np.percentile(L, 99)), "mean_latency_s": float(L.mean()),
            "arc_updates_per_s": arcs / window, "drain_s": round(end - total, 2),
            "estimate": "fp32" if args.fp32 else "fp64", "pool_graphs": len(pool),
            "pool_arcs": int(sum(g.m for g in pool))}


def serve_main(args):
    rng = np.random.default_rng(args.seed)
    pool = []
    t0 = time.time()
    for i in range(args.pool):
        n = int(np.exp(rng.uniform(np.log(1e4), np.log(args.max_n))))
        pool.append(_rmat(n, 16, 5000 + i))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    gen_s = time.time() - t0
    for slots, label in ((args.slots, "continuous-batching"), (1, "fifo-one-at-a-time")):
        r = serve_run(pool, args, slots, label)
        r["generate_s"] = round(gen_s, 1)
        print(json.dumps(r), flush=True)


def runs_main(args):
    g = graphs.enwiki_graph(device="cuda")
    n, b = g.n, 6
    seeds = [42 + r for r in range(args.runs)]
    batch = hbl.HyperBallBatch.runs(g.offsets, g.targets, n, b, seeds, fp32=args.fp32)
    outs = {k: (torch.empty(n, dtype=torch.float64, device="cuda"),
                torch.empty(n, dtype=torch.float64, device="cuda")) for k in hbl.HyperBallBatch.CENTRALITIES}
    lib = hbl.load()

    def batched():
        batch.reset(seeds)
        iters = batch.run()
        for w, k in enumerate(hbl.HyperBallBatch.CENTRALITIES):
            hbl._check(lib.hb_batch_get_run_stats(batch._h, w, hbl._ptr(outs[k][0]), hbl._ptr(outs[k][1])))
        return iters

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
        return arcs

    batched()
    one_at_a_time()
    bt, st = [], []
    for _ in range(args.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        iters = batched()
        torch.cuda.synchronize()
        bt.append(time.perf_counter() - t)
        t = time.perf_counter()
        solo_arcs = one_at_a_time()
        torch.cuda.synchronize()
        st.append(time.perf_counter() - t)
    _, _, arcs = batch.totals()
    batch.close()
    solo.close()
    b_s, s_s = min(bt), min(st)
    print(json.dumps({
        "form": "runs", "graph": "encyclopedia-like (R-MAT scale 23, 4,206,785 nodes), transpose, log2m 6",
        "runs": args.runs, "n": n, "m": g.m, "batch_ms": round(1e3 * b_s, 3), "batch_iterations": iters,
        "batch_arc_updates_per_s": arcs / b_s, "one_at_a_time_ms": round(1e3 * s_s, 3),
        "one_at_a_time_arc_updates_per_s": solo_arcs / s_s, "speedup": s_s / b_s,
        "estimate": "fp32" if args.fp32 else "fp64",
        "includes": "all runs to their fixpoints and the per-node mean and std of the four centralities"}),
        flush=True)


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
    s.add_argument("--reserve-gb", type=int, default=8)
    s.add_argument("--seed", type=int, default=5)
    s.add_argument("--fp32", action="store_true")
    r = sub.add_parser("runs")
    r.add_argument("--runs", type=int, default=16)
    r.add_argument("--repeat", type=int, default=3)
    r.add_argument("--fp32", action="store_true")
    args = ap.parse_args()
    build.build()
    hbl.load()
    {"batch": batch_main, "serve": serve_main, "runs": runs_main}[args.cmd](args)


if __name__ == "__main__":
    main()
