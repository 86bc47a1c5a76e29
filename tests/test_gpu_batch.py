"""Batched form: every graph in the mix gives the same result as when run
alone (registers, iteration counts and accumulators identical) and as the
oracle (bit-exact registers and counts, 1e-9 on accumulators)."""
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


def _mix(count=24, seed=0):
    """Graphs of uneven size and mixed log2m, some with split (heavy) nodes."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = i % 3
        if kind == 0:
            g = graphs.plain_graph(n=int(rng.integers(300, 5000)), seed=100 + i)
        elif kind == 1:
            g = graphs.rmat_graph(scale=int(rng.integers(8, 14)), edge_factor=int(rng.integers(4, 33)),
                                  seed=200 + i)
        else:
            g = graphs.from_edges(int(rng.integers(2, 40)),
                                  [(int(a), int(b)) for a, b in rng.integers(0, 2, size=(1, 2))])
        b = int(rng.choice([4, 5, 6, 7]))
        out.append((g, b, 1000 + i))
    # an empty graph and one hub-dominated graph
    out.append((graphs.from_edges(1, []), 4, 7))
    hub = [(v, 0) for v in range(1, 3000)] + [(0, v) for v in range(1, 3000, 7)]
    out.append((graphs.from_edges(3000, hub, keep_all=False), 6, 11))
    return out


def _descs(mix):
    return [(g.offsets.cuda(), g.targets.cuda(), g.n, b, s) for g, b, s in mix]


def test_batch_matches_solo_and_oracle(orc):
    mix = _mix()
    batch = hbl.HyperBallBatch(_descs(mix))
    iters = batch.run()
    it, active, arcs = batch.totals()
    assert active == 0 and it == iters
    total = 0
    for i, (g, b, s) in enumerate(mix):
        solo = hbl.HyperBall(g.offsets.cuda(), g.targets.cuda(), log2m=b, seed=s, n=g.n)
        steps = solo.run()
        info = batch.info(i)
        assert info["t"] == steps and info["converged"] == 1
        assert torch.equal(batch.registers(i), solo.registers())
        for x, y in zip(batch.accumulators(i), solo.accumulators()):
            assert torch.equal(x, y)
        total += info["total_arcs"]
        if i % 4 == 0:
            off, tgt = g.numpy()
            ref = orc.run(off, tgt, b, s)
            assert ref.steps == steps
            assert np.array_equal(batch.registers(i).cpu().numpy(), ref.regs)
            s_, h_ = batch.accumulators(i)
            np.testing.assert_allclose(s_.cpu().numpy(), ref.sumd, rtol=1e-9, atol=0)
            np.testing.assert_allclose(h_.cpu().numpy(), ref.harm, rtol=1e-9, atol=0)
            fin = orc.finalize(b, ref.regs, ref.sumd, ref.harm)
            cen = batch.centralities(i)
            for key in fin:
                np.testing.assert_allclose(cen[key].cpu().numpy(), fin[key], rtol=1e-9, atol=0)
        solo.close()
    assert total == arcs
    batch.close()


def test_batch_step_by_step_matches_solo_steps():
    mix = _mix(count=9, seed=3)
    batch = hbl.HyperBallBatch(_descs(mix))
    solos = [hbl.HyperBall(g.offsets.cuda(), g.targets.cuda(), log2m=b, seed=s, n=g.n) for g, b, s in mix]
    done = [False] * len(mix)
    for _ in range(200):
        active = batch.step()
        for i, h in enumerate(solos):
            if not done[i]:
                if h.step() == 0:
                    done[i] = True
            assert torch.equal(batch.registers(i), h.registers())
        assert active == sum(1 for d in done if not d)
        if active == 0:
            break
    assert all(done)
    for h in solos:
        h.close()
    batch.close()


def test_batch_reset_and_rerun_is_identical():
    mix = _mix(count=6, seed=5)
    batch = hbl.HyperBallBatch(_descs(mix), fp32=True)
    batch.run()
    first = [batch.registers(i).clone() for i in range(len(mix))]
    acc = [batch.accumulators(i) for i in range(len(mix))]
    batch.reset()
    batch.run()
    for i in range(len(mix)):
        assert torch.equal(batch.registers(i), first[i])
        for x, y in zip(batch.accumulators(i), acc[i]):
            assert torch.equal(x, y)
    batch.close()


def test_batch_rejects_bad_arguments():
    with pytest.raises(hbl.HBError):
        hbl.HyperBallBatch([])
    g = graphs.plain_graph(n=50, seed=1)
    with pytest.raises(hbl.HBError):
        hbl.HyperBallBatch([(g.offsets.cuda(), g.targets.cuda(), g.n, 3, 1)])


def test_batch_autotuner_keeps_results():
    mix = _mix(count=8, seed=9)
    batch = hbl.HyperBallBatch(_descs(mix))
    aps = batch.tune()
    assert aps in (1, 2, 4, 8, 16, 32, 64, 128)
    batch.run()
    for i, (g, b, s) in enumerate(mix):
        solo = hbl.HyperBall(g.offsets.cuda(), g.targets.cuda(), log2m=b, seed=s, n=g.n)
        solo.run()
        assert torch.equal(batch.registers(i), solo.registers())
        for x, y in zip(batch.accumulators(i), solo.accumulators()):
            assert torch.equal(x, y)
        solo.close()
    batch.close()


def test_batch_pushed_and_gathered_frontiers_agree_at_every_log2m(orc):
    """Frontier iterations done by the pushed union (default) and by the
    gather (HB_PULL_GATHER) give identical batch results, on a mix that spans
    every log2m from 4 to 12 (one gather kernel and item prefix per log2m)."""
    mix = [(graphs.rmat_graph(scale=10, edge_factor=8, seed=300 + i), b, 50 + i)
           for i, b in enumerate(range(4, 13))]
    res = []
    for pg in (False, True):
        batch = hbl.HyperBallBatch(_descs(mix), pull_gather=pg)
        batch.run()
        res.append([(batch.registers(i).cpu(), [x.cpu() for x in batch.accumulators(i)], batch.info(i)["t"])
                    for i in range(len(mix))])
        batch.close()
    for (r0, a0, t0), (r1, a1, t1) in zip(*res):
        assert t0 == t1 and torch.equal(r0, r1)
        for x, y in zip(a0, a1):
            assert torch.equal(x, y)
    for i in (0, 4, 8):
        g, b, s = mix[i]
        off, tgt = g.numpy()
        ref = orc.run(off, tgt, b, s)
        assert res[0][i][2] == ref.steps
        assert np.array_equal(res[0][i][0].numpy(), ref.regs)
        np.testing.assert_allclose(res[0][i][1][0].numpy(), ref.sumd, rtol=1e-9, atol=0)
