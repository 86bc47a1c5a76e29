"""The switch of HB_FRONTIER_AUTO (hb_set_frontier_switch and
hb_options.frontier_switch): how the nodes to recompute are chosen each
iteration, pushing the last iteration's changed counters when their reverse
arcs are at most that fraction of m, else recomputing every node (the
modification tracking of Sec. 5 / 5.1).  It never changes what a node
computes, so counters must equal the oracle's at every iteration for every
switch value, including one changed between iterations, and the
accumulators must be bitwise equal across values (the same per-node
arithmetic in the same order)."""
import math

import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl
from tests.test_gpu_parity import walk_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


@pytest.mark.parametrize("frac", [1e-6, 0.0625, 0.25, 1.0, 1e6])
@pytest.mark.parametrize("pull_gather", [False, True])
def test_switch_values_against_oracle(orc, frac, pull_gather):
    off, tgt = graphs.rmat_graph(scale=12, edge_factor=8, seed=23).numpy()
    walk_parity(orc, off, tgt, 5, 19, frontier="auto", pull_gather=pull_gather, frontier_switch=frac)


def test_switch_reported_and_changed_between_iterations(orc):
    off, tgt = graphs.rmat_graph(scale=13, edge_factor=8, seed=7).numpy()
    n = off.size - 1
    h = hbl.HyperBall(torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda(), log2m=4, seed=3, n=n)
    assert h.info()["frontier_switch"] == 0.25
    c = orc.init(n, 4, 3)
    s, hm = np.zeros(n), np.zeros(n)
    fracs = [0.5, 1e-6, 4.0, 0.01, 0.25]
    modes = set()
    t = 0
    while True:
        h.set_frontier_switch(fracs[t % len(fracs)])
        assert h.info()["frontier_switch"] == fracs[t % len(fracs)]
        c, _, k = orc.step(off, tgt, 4, t, c, s, hm)
        assert h.step() == k
        modes.add(h.info()["last_sparse"])
        assert np.array_equal(h.registers().cpu().numpy(), c), t
        t += 1
        if k == 0:
            break
    assert modes == {0, 1}
    gs, gh = h.accumulators()
    np.testing.assert_allclose(gs.cpu().numpy(), s, rtol=1e-9, atol=0)
    np.testing.assert_allclose(gh.cpu().numpy(), hm, rtol=1e-9, atol=0)
    h.close()


def test_switch_values_bitwise_equal_at_scale():
    g = graphs.rmat_graph(scale=18, edge_factor=16, seed=5, device="cuda")
    ref = None
    for frac in (0.25, 1e-6, 0.05, 1.0, 8.0):
        h = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=9, n=g.n, fp32=True, frontier_switch=frac)
        steps = h.run()
        out = (steps, h.registers(), *h.accumulators(), h.centralities()["lin"])
        if ref is None:
            ref = out
        else:
            assert out[0] == ref[0]
            for x, y in zip(out[1:], ref[1:]):
                assert torch.equal(x, y), frac
        h.close()


def test_switch_refusals():
    g = graphs.rmat_graph(scale=10, edge_factor=8, seed=1, device="cuda")
    for bad in (-1.0, math.inf, math.nan):
        with pytest.raises(hbl.HBError) as e:
            hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=1, n=g.n, frontier_switch=bad)
        assert e.value.status == hbl.HB_ERR_INVALID
    h = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=1, n=g.n)
    for bad in (0.0, -0.5, math.inf, math.nan):
        with pytest.raises(hbl.HBError) as e:
            h.set_frontier_switch(bad)
        assert e.value.status == hbl.HB_ERR_INVALID
    assert h.info()["frontier_switch"] == 0.25
    h.close()
