"""bench.py's multi-rank path (independent replicas, weak scaling) on CPU
ranks with the gloo backend: the slowest rank's time and the sum of all
ranks' units make the whole-job number."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000.0 * (rank + 1)          # rank r processed 1000 (r+1) arc-updates
    ms = 10.0 + 5.0 * rank               # the slowest rank took 15 ms
    val = bench.replica_throughput(units, ms, world)
    mx = bench.max_over_ranks(ms, world)
    sm = bench.sum_over_ranks(units, world)
    bench.barrier(world)
    out[rank] = (val, mx, sm)
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        val, mx, sm = out[r]
        assert mx == 15.0
        assert sm == 3000.0
        assert val == pytest.approx(3000.0 / 0.015)


def test_single_rank_is_identity():
    import bench
    assert bench.replica_throughput(500.0, 10.0, 1) == pytest.approx(50000.0)
    assert bench.max_over_ranks(3.0, 1) == 3.0


def test_reference_arm_reports_the_oracle():
    """bench.py --impl reference times the CPU oracle (no GPU) on the same
    metric and prints one JSON line with the reference arm's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "plain", "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600,
                       cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 1
    assert line["unit"] == "arc-updates/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["n"] == 10_000


def test_cpu_baseline_sample_reports_threads_model_and_one_thread():
    """bench.py's cpu_baseline: the oracle on a prefix of the nodes with
    every thread and with one, the core count, nproc and the CPU model."""
    import bench
    from paper_1308_2144_gb300 import graphs
    off, tgt = graphs.plain_graph(n=10_000, seed=1).numpy()
    cpu = bench.cpu_oracle_sample((off, tgt), 4, 42, budget_s=0.5, budget_one_s=0.2)
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1
    assert cpu["nproc"] == os.cpu_count() and isinstance(cpu["cpu_model"], str) and cpu["cpu_model"]
    assert cpu["single_thread"]["cores"] == 1 and cpu["single_thread"]["value"] > 0
    assert "of 10000 nodes" in cpu["sample"]
