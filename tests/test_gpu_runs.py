"""Multiple runs of one graph (Sec. 5) in one batch, through the C ABI:
each run equals its solo run with the same seed (registers and iteration
counts bit-exact, accumulators within 1e-9), and the per-node mean and
empirical standard deviation of every centrality equal the oracle's over
the same seeds within 1e-9 of the mean."""
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
