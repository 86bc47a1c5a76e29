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


def _state(srv, rid):
    info = hbl.RequestInfo()
    st = hbl.load().hb_server_wait(srv._h, int(rid), 0.0, hbl.ctypes.byref(info))
    return st, info.state


def test_cancel_queued_and_running_requests():
    pool = _pool()
    big = graphs.rmat_graph(scale=18, edge_factor=16, seed=6)
    srv = hbl.HyperBallServer(slots=1, reserve_bytes=0)
    gids = [srv.add_graph(g.offsets.cuda(), g.targets.cuda(), g.n, log2ms=(4, 6)) for g in pool]
    gbig = srv.add_graph(big.offsets.cuda(), big.targets.cuda(), big.n, log2ms=(6,))
    # one slot: the first request runs, the next two wait in the queue
    r0 = srv.submit(gbig, 6, 1)
    r1 = srv.submit(gids[0], 4, 2)
    r2 = srv.submit(gids[2], 4, 3)
    srv.cancel(r1)                       # queued: leaves the queue at once
    with pytest.raises(hbl.HBError) as e:
        srv.wait(r1, timeout=10)
    assert e.value.status == hbl.HB_ERR_STATE
    assert _state(srv, r1)[1] == hbl.HB_REQ_CANCELLED
    for rid, g, b, seed in ((r0, big, 6, 1), (r2, pool[2], 4, 3)):
        info = srv.wait(rid, timeout=120)
        steps, solo = _solo(g, b, seed)
        assert info["steps"] == steps
        res = srv.take(rid, g.n)
        for key in solo:
            assert np.array_equal(res[key], solo[key]), key
    with pytest.raises(hbl.HBError) as e:
        srv.cancel(r0)                   # taken: unknown now
    with pytest.raises(hbl.HBError) as e:
        srv.take(r1, pool[0].n)          # a cancelled request is forgotten
    assert e.value.status == hbl.HB_ERR_STATE
    # a running request: retired at an iteration boundary, its slot reused
    r3 = srv.submit(gbig, 6, 9)
    for _ in range(2000):
        if _state(srv, r3)[1] != hbl.HB_REQ_QUEUED:
            break
        time.sleep(0.001)
    try:
        srv.cancel(r3)
        cancelled = True
    except hbl.HBError:                  # it finished before the cancel arrived
        cancelled = False
    st, state = _state(srv, r3)
    if cancelled:
        with pytest.raises(hbl.HBError):
            srv.wait(r3, timeout=60)
        assert _state(srv, r3)[1] == hbl.HB_REQ_CANCELLED
    r4 = srv.submit(gids[1], 6, 4)
    info = srv.wait(r4, timeout=120)
    steps, solo = _solo(pool[1], 6, 4)
    assert info["steps"] == steps
    res = srv.take(r4, pool[1].n)
    for key in solo:
        assert np.array_equal(res[key], solo[key]), key
    srv.close()


def test_request_that_cannot_fit_is_refused():
    g = graphs.plain_graph(n=2000, seed=1)
    srv = hbl.HyperBallServer(slots=2, reserve_bytes=1 << 50)   # more than any device has
    gid = srv.add_graph(g.offsets.cuda(), g.targets.cuda(), g.n, log2ms=(4,))
    rid = srv.submit(gid, 4, 1)
    with pytest.raises(hbl.HBError) as e:
        srv.wait(rid, timeout=30)
    assert e.value.status == hbl.HB_ERR_OOM
    assert _state(srv, rid)[1] == hbl.HB_REQ_FAILED
    srv.close()


def test_size_aware_admission_keeps_one_large_request_and_results():
    """With large_slots = 1, at most one request on a large graph runs at a
    time (their admit-to-done intervals never overlap), small requests
    submitted behind a large one are admitted while it waits, and every
    result equals the solo run bit for bit."""
    pool = _pool()
    large = pool[1].m                      # the scale-13 graph is "large"
    srv = hbl.HyperBallServer(slots=6, reserve_bytes=0, large_slots=1, large_arcs=large)
    gids = [srv.add_graph(g.offsets.cuda(), g.targets.cuda(), g.n, log2ms=(4, 6)) for g in pool]
    order = [1, 1, 1, 0, 2, 1, 0, 2, 2, 1, 0]
    jobs = [(gi, 4 + 2 * (r % 2), 500 + r, srv.submit(gids[gi], 4 + 2 * (r % 2), 500 + r))
            for r, gi in enumerate(order)]
    infos = []
    for gi, b, seed, rid in jobs:
        info = srv.wait(rid, timeout=120)
        assert info["state"] == hbl.HB_REQ_DONE
        res = srv.take(rid, pool[gi].n)
        steps, solo = _solo(pool[gi], b, seed)
        assert info["steps"] == steps
        for key in solo:
            assert np.array_equal(res[key], solo[key]), key
        infos.append((gi, info))
    spans = sorted((i["admit_s"], i["done_s"]) for gi, i in infos if gi == 1)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 1e-6, (a0, d0, a1, d1)
    # the small request submitted behind the first three large ones is
    # admitted before the last of them
    small_admit = infos[3][1]["admit_s"]
    assert small_admit <= max(i["admit_s"] for gi, i in infos[:3])
    srv.close()


def test_server_rejects_negative_large_options():
    with pytest.raises(hbl.HBError) as e:
        hbl.HyperBallServer(slots=2, large_slots=-1)
    assert e.value.status == hbl.HB_ERR_INVALID
