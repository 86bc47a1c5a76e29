"""Accuracy of the GPU centralities against exact breadth-first values on
the encyclopedia-like graph (R-MAT, 4,206,785 nodes, 101,355,853 arcs drawn,
scanned as its transpose), the stand-in for the Wikipedia snapshot of the
paper's Sec. 8 experiments, at p = 64 registers.

Sec. 8 computes exact centralities for a random sample of nodes and finds
the estimates' relative error close to, and mostly below, the single-counter
bound 1.06/sqrt(p) of Sec. 4.1, shrinking when runs are averaged.  Here a
uniform sample of 1,000 nodes (seed 3) gets exact values from the oracle's
breadth-first visits along the scanned arcs, and the GPU's four
centralities over 16 hash seeds are held to a few times that bound."""
import math

import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl

pytestmark = pytest.mark.gpu

B = 6            # p = 64 registers
SEEDS = 16
SAMPLE = 1000


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


@pytest.fixture(scope="module")
def sample(orc):
    g = graphs.enwiki_graph(device="cuda")
    off, tgt = g.numpy()
    n = off.size - 1
    rng = np.random.default_rng(3)
    src = np.sort(rng.choice(n, size=SAMPLE, replace=False))
    exact = orc.exact_centralities(off, tgt, src)
    est = {k: [] for k in ("closeness", "harmonic", "lin", "reachable")}
    hb = hbl.HyperBall(g.offsets, g.targets, log2m=B, seed=1, n=n)
    idx = torch.from_numpy(src).cuda()
    for s in range(SEEDS):
        hbl.hb_reset(hb._h, 9000 + s)
        hb.run()
        cen = hb.centralities()
        for k in est:
            est[k].append(cen[k][idx].cpu().numpy())
    hb.close()
    return src, exact, {k: np.array(v) for k, v in est.items()}


def _exact_centrality(exact, key):
    s, r = exact["sumd"], exact["reach"]
    if key == "closeness":
        return np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    if key == "lin":
        return np.where(s > 0, r * r / np.where(s > 0, s, 1.0), 1.0)
    if key == "harmonic":
        return exact["harm"]
    return r


def test_sample_covers_small_and_large_balls(sample):
    _, exact, _ = sample
    assert (exact["reach"] >= 1).all()
    assert (exact["reach"] >= 1000).sum() > 100      # many sampled nodes reach many nodes


@pytest.mark.parametrize("key", ["closeness", "harmonic", "lin", "reachable"])
def test_rms_error_within_a_few_counter_bounds(sample, key):
    """Per node, the RMS relative error over 16 seeds: its median over the
    sampled nodes with at least 200 coreachable nodes within two times the
    single-counter bound 1.06/sqrt(p) ("a few times" the bound), the median
    bias over seeds within one bound, and a node that nothing else
    coreaches exact.  Sum-of-distance centralities combine the estimates of
    every iteration (sumd = T size(c_T) - sum over t < T of size(c_t)), so
    at p = 64 their error exceeds one counter's; the measured values are
    printed."""
    _, exact, est = sample
    bound = 1.06 / math.sqrt(1 << B)
    ex = _exact_centrality(exact, key)
    big = exact["reach"] >= 200
    e = est[key][:, big] / ex[big] - 1.0
    rms = np.sqrt((e ** 2).mean(axis=0))
    bias = np.median(e.mean(axis=0))
    print(f"{key}: median RMS relative error {np.median(rms):.4f} = {np.median(rms) / bound:.2f} x bound, "
          f"median bias {bias:+.4f}, nodes {int(big.sum())}")
    assert np.median(rms) <= 2.0 * bound, (key, np.median(rms), bound)
    assert abs(bias) <= bound, (key, bias)
    alone = exact["reach"] == 1
    if key in ("closeness", "harmonic"):
        assert (est[key][:, alone] == 0.0).all()
    elif key == "lin":
        assert (est[key][:, alone] == 1.0).all()


def test_averaging_seeds_shrinks_error(sample):
    """Sec. 8: averaging runs tightens the estimate.  Per node, the error of
    the mean of 16 runs against the RMS error of one run (most sampled nodes
    share one coreachable set, so within one run their errors are a single
    draw: the comparison is taken across runs).  16 runs: about 1/4 of one
    run's error plus the estimator's bias at p = 64; allow 1/2."""
    _, exact, est = sample
    big = exact["reach"] >= 200
    ex = exact["harm"][big]
    e = est["harmonic"][:, big] / ex - 1.0
    single = np.median(np.sqrt((e ** 2).mean(axis=0)))
    mean16 = np.median(np.abs(e.mean(axis=0)))
    assert mean16 < 0.5 * single, (mean16, single)
