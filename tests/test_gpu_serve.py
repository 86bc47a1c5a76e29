"""Serving form: requests admitted while others run (continuous batching)
give the same centralities as the same job run alone, and as the oracle."""
import time

import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


def _pool():
    return [graphs.plain_graph(n=4000, seed=3), graphs.rmat_graph(scale=13, edge_factor=16, seed=4),
            graphs.rmat_graph(scale=11, edge_factor=8, seed=5)]


def _solo(g, b, seed):
    h = hbl.HyperBall(g.offsets.cuda(), g.targets.cuda(), log2m=b, seed=seed, n=g.n)
    steps = h.run()
    cen = {k: v.cpu().numpy() for k, v in h.centralities().items()}
    h.close()
    return steps, cen


@pytest.mark.parametrize("slots", [4, 1])
def test_requests_in_the_mix_equal_solo_runs(orc, slots):
    pool = _pool()
    srv = hbl.HyperBallServer(slots=slots, reserve_bytes=0)
    gids = [srv.add_graph(g.offsets.cuda(), g.targets.cuda(), g.n, log2ms=(4, 6)) for g in pool]
    rng = np.random.default_rng(slots)
    jobs = []
    for r in range(10):
        gi = int(rng.integers(0, len(pool)))
        b = int(rng.choice([4, 6]))
        seed = 1000 + r
        jobs.append((gi, b, seed, srv.submit(gids[gi], b, seed)))
        time.sleep(0.002 * float(rng.random()))     # arrivals while others run
    for gi, b, seed, rid in jobs:
        info = srv.wait(rid, timeout=120)
        assert info["state"] == hbl.HB_REQ_DONE
        res = srv.take(rid, pool[gi].n)
        steps, solo = _solo(pool[gi], b, seed)
        assert info["steps"] == steps
        for key in solo:
            assert np.array_equal(res[key], solo[key]), key
        assert info["admit_s"] >= info["submit_s"] and info["done_s"] >= info["admit_s"]
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["arcs"] > 0
    # one request against the oracle
    gi, b, seed, _ = jobs[0]
    off, tgt = pool[gi].numpy()
    ref = orc.run(off, tgt, b, seed)
    fin = orc.finalize(b, ref.regs, ref.sumd, ref.harm)
    rid = srv.submit(gids[gi], b, seed)
    srv.wait(rid, timeout=120)
    res = srv.take(rid, pool[gi].n)
    for key in fin:
        np.testing.assert_allclose(res[key], fin[key], rtol=1e-9, atol=0)
    srv.close()


def test_server_rejects_unknown_graph_and_log2m():
    srv = hbl.HyperBallServer(slots=2)
    g = graphs.plain_graph(n=100, seed=1)
    gid = srv.add_graph(g.offsets.cuda(), g.targets.cuda(), g.n, log2ms=(4,))
    with pytest.raises(hbl.HBError):
        srv.submit(gid + 5, 4, 1)
    with pytest.raises(hbl.HBError):
        srv.submit(gid, 6, 1)
    srv.close()
