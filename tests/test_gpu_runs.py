"""Multiple runs of one graph (Sec. 5) in one batch, through the C ABI:
each run equals its solo run with the same seed (registers and iteration
counts bit-exact, accumulators within 1e-9), and the per-node mean and
empirical standard deviation of every centrality equal the oracle's over
the same seeds within 1e-9 of the mean."""
import math

import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl
from tests.test_gpu_parity import close, to_dev

pytestmark = pytest.mark.gpu

CENTRALITIES = ("closeness", "harmonic", "lin", "reachable")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


def check_stats(orc, batch, off, tgt, b, seeds):
    for which in CENTRALITIES:
        mean, sd = (x.cpu().numpy() for x in batch.run_stats(which))
        m_ref, s_ref = orc.run_stats(off, tgt, b, seeds, which)
        close(mean, m_ref)
        assert np.all(np.abs(sd - s_ref) <= 1e-9 * np.abs(m_ref)), which


@pytest.mark.parametrize("b,frontier", [(4, "auto"), (6, "auto"), (6, "off"), (9, "push")])
def test_runs_match_solo_runs_and_oracle(orc, b, frontier):
    off, tgt = graphs.rmat_graph(scale=12, edge_factor=8, seed=50 + b).numpy()
    n = off.size - 1
    seeds = [100 + 7 * r for r in range(8)]
    d_off, d_tgt = to_dev(off, tgt)
    batch = hbl.HyperBallBatch.runs(d_off, d_tgt, n, b, seeds, frontier=frontier)
    batch.run()
    for r, s in enumerate(seeds):
        ref = orc.run(off, tgt, b, s)
        assert batch.info(r)["t"] == ref.steps
        assert np.array_equal(batch.registers(r).cpu().numpy(), ref.regs)
        gs, gh = batch.accumulators(r)
        close(gs.cpu().numpy(), ref.sumd)
        close(gh.cpu().numpy(), ref.harm)
    check_stats(orc, batch, off, tgt, b, seeds)
    # a reset with new seeds gives the statistics of those
    seeds2 = [900 + r for r in range(8)]
    batch.reset(seeds2)
    batch.run()
    check_stats(orc, batch, off, tgt, b, seeds2)
    batch.close()


def test_runs_from_host_csr_fp32_and_one_run(orc):
    off, tgt = graphs.plain_graph(n=5000, seed=4).numpy()
    n = off.size - 1
    seeds = [11, 12, 13]
    batch = hbl.HyperBallBatch.runs(torch.from_numpy(off), torch.from_numpy(tgt), n, 5, seeds, fp32=True)
    batch.run()
    for r, s in enumerate(seeds):
        assert np.array_equal(batch.registers(r).cpu().numpy(), orc.run(off, tgt, 5, s).regs)
    batch.close()
    one = hbl.HyperBallBatch.runs(torch.from_numpy(off), torch.from_numpy(tgt), n, 5, [11])
    one.run()
    mean, sd = one.run_stats("harmonic", device="cpu")
    ref = orc.run(off, tgt, 5, 11)
    close(mean.numpy(), ref.harm)
    assert not sd.numpy().any()
    one.close()


def test_same_graph_batch_and_mixed_sizes(orc):
    off, tgt = graphs.rmat_graph(scale=11, edge_factor=8, seed=9).numpy()
    n = off.size - 1
    d_off, d_tgt = to_dev(off, tgt)
    seeds = [5, 6, 7, 8]
    batch = hbl.HyperBallBatch([(d_off, d_tgt, n, 6, s) for s in seeds])
    batch.run()
    check_stats(orc, batch, off, tgt, 6, seeds)
    batch.close()
    off2, tgt2 = graphs.rmat_graph(scale=10, edge_factor=8, seed=9).numpy()
    mixed = hbl.HyperBallBatch([(d_off, d_tgt, n, 6, 1), (*to_dev(off2, tgt2), off2.size - 1, 6, 2)])
    with pytest.raises(hbl.HBError) as e:
        mixed.run_stats("lin")
    assert e.value.status == hbl.HB_ERR_INVALID
    mixed.close()


# ------------------------------------------------- runs in one handle --

def check_wide(orc, hb, off, tgt, b, seeds, weights=None, discount=None):
    n = off.size - 1
    p = 1 << b
    regs = hb.registers().cpu().numpy()
    assert regs.shape == (n, len(seeds) * p)
    steps = hb.run_steps()
    for r, s in enumerate(seeds):
        ref = orc.run(off, tgt, b, s, weights=weights, discount=discount)
        assert steps[r] == ref.steps, (r, steps[r], ref.steps)
        assert np.array_equal(regs[:, r * p:(r + 1) * p], ref.regs), r
        gs, gh = hb.run_accumulators(r)
        close(gs.cpu().numpy(), ref.sumd)
        close(gh.cpu().numpy(), ref.harm)
        if discount is not None:
            close(hb.run_discounted(r).cpu().numpy(), ref.disc)
        fin = orc.finalize(b, ref.regs, ref.sumd, ref.harm)
        cen = hb.run_centralities(r)
        for k in CENTRALITIES:
            close(cen[k].cpu().numpy(), fin[k])
    assert hb.info()["t"] == max(steps)
    for which in CENTRALITIES + (("discounted",) if discount is not None else ()):
        mean, sd = (x.cpu().numpy() for x in hb.run_stats(which))
        m_ref, s_ref = orc.run_stats(off, tgt, b, seeds, which, weights=weights, discount=discount)
        close(mean, m_ref)
        assert np.all(np.abs(sd - s_ref) <= 1e-9 * np.abs(m_ref)), which


@pytest.mark.parametrize("b,R,frontier", [(4, 2, "auto"), (4, 16, "auto"), (4, 64, "off"), (5, 64, "push"),
                                          (6, 4, "off"), (6, 16, "push"), (7, 32, "auto"), (9, 8, "pull")])
def test_runs_in_one_handle_equal_solo_runs(orc, b, R, frontier):
    """Each run of a row equals its solo run: counters, iteration count,
    accumulators and centralities; the statistics equal the oracle's."""
    off, tgt = graphs.rmat_graph(scale=11, edge_factor=8, seed=60 + b + R).numpy()
    seeds = [300 + 11 * r for r in range(R)]
    hb = hbl.HyperBall.runs(*to_dev(off, tgt), b, seeds, n=off.size - 1, frontier=frontier)
    hb.run()
    check_wide(orc, hb, off, tgt, b, seeds)
    # a reset keeps the seeds and gives the same runs again
    hb.reset(0)
    hb.run()
    check_wide(orc, hb, off, tgt, b, seeds)
    hb.close()


def test_runs_in_one_handle_every_iteration(orc):
    """At every iteration each run's slice of the rows equals the oracle's
    counters of that run, and a node is flagged changed exactly when one of
    its runs changed.  Hubs above the split threshold of the wide rows."""
    off, tgt = graphs.rmat_graph(scale=13, edge_factor=16, seed=8).numpy()
    n = off.size - 1
    b, seeds = 6, [5, 6, 7, 8]
    p = 1 << b
    hb = hbl.HyperBall.runs(*to_dev(off, tgt), b, seeds, n=n)
    cs = [orc.init(n, b, s) for s in seeds]
    acc = [(np.zeros(n), np.zeros(n)) for _ in seeds]
    t = 0
    while True:
        outs = [orc.step(off, tgt, b, t, cs[r], *acc[r]) for r in range(len(seeds))]
        k = hb.step()
        regs = hb.registers().cpu().numpy()
        changed = np.zeros(n, dtype=bool)
        for r, (nxt, ch, _) in enumerate(outs):
            assert np.array_equal(regs[:, r * p:(r + 1) * p], nxt), (t, r)
            changed |= ch.astype(bool)
            cs[r] = nxt
        assert k == int(changed.sum())
        assert np.array_equal(hb.frontier()[0].cpu().numpy().astype(bool), changed)
        t += 1
        if k == 0:
            break
    hb.close()


def test_runs_in_one_handle_fp32_host_csr_and_limits(orc):
    off, tgt = graphs.plain_graph(n=4000, seed=9).numpy()
    n = off.size - 1
    seeds = [21, 22, 23, 24, 25, 26, 27, 28]
    hb = hbl.HyperBall.runs(torch.from_numpy(off), torch.from_numpy(tgt), 4, seeds, n=n, fp32=True)
    hb.tune()
    hb.run()
    regs = hb.registers().cpu().numpy()
    for r, s in enumerate(seeds):
        assert np.array_equal(regs[:, 16 * r:16 * (r + 1)], orc.run(off, tgt, 4, s).regs)
    for call in (lambda: hb.centralities(), lambda: hb.accumulators(), lambda: hb.run_discounted(0),
                 lambda: hb.run_stats("discounted"), lambda: hb.save("/tmp/never-written.ckpt")):
        with pytest.raises(hbl.HBError) as e:
            call()
        assert e.value.status == hbl.HB_ERR_STATE
    hb.set_discount([1.0])
    with pytest.raises(hbl.HBError) as e:   # one accumulator per run: hb_get_run_discounted
        hb.discounted()
    assert e.value.status == hbl.HB_ERR_STATE
    hb.close()
    d_off, d_tgt = to_dev(off, tgt)
    for b, seeds in ((4, [1, 2, 3]), (10, [1, 2]), (7, list(range(64))), (4, [1])):
        with pytest.raises(hbl.HBError) as e:
            hbl.HyperBall.runs(d_off, d_tgt, b, seeds, n=n)
        assert e.value.status == hbl.HB_ERR_INVALID


@pytest.mark.parametrize("b,R,frontier", [(4, 8, "auto"), (6, 4, "off"), (5, 16, "push")])
def test_runs_in_one_handle_weighted_discounted(orc, b, R, frontier):
    """Sec. 6 weights and a Sec. 7 discount on rows of several runs: each run
    hashes the replicas with its own seed and keeps its own discounted
    accumulator; every run equals the weighted, discounted oracle run of its
    seed, and the statistics (the discounted one included) the oracle's."""
    off, tgt = graphs.rmat_graph(scale=11, edge_factor=8, seed=90 + b).numpy()
    n = off.size - 1
    w = np.random.default_rng(b + R).integers(0, 7, size=n).astype(np.int64)
    table = [1.0 / math.log(d + 1) for d in range(1, 65)]
    seeds = [500 + 13 * r for r in range(R)]
    hb = hbl.HyperBall.runs(*to_dev(off, tgt), b, seeds, n=n, frontier=frontier)
    hb.set_weights(torch.from_numpy(w).cuda())
    hb.set_discount(table)
    hb.run()
    check_wide(orc, hb, off, tgt, b, seeds, weights=w, discount=table)
    # a short table: distances beyond it contribute nothing; reset keeps both
    hb.set_discount([1.0, 0.5, 0.25])
    hb.reset(0)
    hb.run()
    check_wide(orc, hb, off, tgt, b, seeds, weights=w, discount=[1.0, 0.5, 0.25])
    # unit weights give the unweighted runs
    hb.set_weights(np.ones(n, dtype=np.int64))
    hb.set_discount([])
    hb.run()
    check_wide(orc, hb, off, tgt, b, seeds)
    hb.close()


@pytest.mark.parametrize("relabel,transpose", [(False, False), (True, True)])
def test_runs_in_one_handle_layouts(orc, relabel, transpose):
    """Without the degree relabelling, and with the transpose taken on the
    device (HB_TRANSPOSE): each run still equals its solo oracle run on the
    scanned graph."""
    g = graphs.rmat_graph(scale=11, edge_factor=8, seed=77)
    off, tgt = g.numpy()
    b, seeds = 5, [3, 4, 5, 6]
    if transpose:
        gt = graphs.transpose(g)          # hand over G^T, scan its transpose (= g)
        d_off, d_tgt = to_dev(*gt.numpy())
    else:
        d_off, d_tgt = to_dev(off, tgt)
    hb = hbl.HyperBall.runs(d_off, d_tgt, b, seeds, n=off.size - 1, relabel=relabel, transpose=transpose)
    hb.run()
    check_wide(orc, hb, off, tgt, b, seeds)
    hb.close()


def test_runs_in_one_handle_empty_and_edgeless():
    for n in (0, 5):
        off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        tgt = torch.zeros(0, dtype=torch.int32, device="cuda")
        hb = hbl.HyperBall.runs(off, tgt, 4, [1, 2], n=n)
        assert hb.run() == 1
        assert hb.run_steps() == [1, 1]
        mean, sd = hb.run_stats("closeness")
        assert mean.numel() == n and not mean.any() and not sd.any()
        hb.close()
