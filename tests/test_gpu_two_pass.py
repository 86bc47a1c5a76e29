"""The hot range of the gather (hb_set_hot_nodes, the hot_nodes and
hot_passes options, hb_tune) against the oracle and against the plain
gather: one pass with L2 priorities (passes = 1) and the two-phase gather
(passes = 2).

The register-wise maximum does not depend on the order or the cache policy
of the reads, so both must give the oracle's counters bit for bit and, with
the same per-node tail, the same accumulators bit for bit as the plain
gather.  Cases: every log2m, hot ranges from one node to beyond n, heavy
(split) nodes, every class sizing, both precisions, every frontier policy,
changing the range and the mode between iterations, and the autotuner."""
import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl
from tests.test_gpu_parity import _degree_boundary_graph, walk_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("b", list(range(4, 13)))
def test_hot_range_every_log2m_against_oracle(orc, b, passes):
    off, tgt = graphs.rmat_graph(scale=11, edge_factor=8, seed=60 + b).numpy()
    n = off.size - 1
    walk_parity(orc, off, tgt, b, 700 + b, frontier="off", hot_nodes=n // 7, hot_passes=passes)


@pytest.mark.parametrize("frontier,pull_gather", [("auto", False), ("auto", True), ("push", False),
                                                  ("pull", False), ("off", False)])
@pytest.mark.parametrize("relabel", [True, False])
@pytest.mark.parametrize("passes", [1, 2])
def test_hot_range_frontier_policies(orc, frontier, pull_gather, relabel, passes):
    off, tgt = graphs.rmat_graph(scale=12, edge_factor=8, seed=21).numpy()
    walk_parity(orc, off, tgt, 5, 77, frontier=frontier, relabel=relabel, pull_gather=pull_gather,
                hot_nodes=500, hot_passes=passes)


@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("b", [4, 6, 9, 12])
def test_hot_range_degree_class_boundaries(orc, b, passes):
    # heavy nodes split into chunks (in both passes), every class boundary
    off, tgt = _degree_boundary_graph(b)
    n = off.size - 1
    walk_parity(orc, off, tgt, b, 5, check_every_step=(b <= 6), frontier="off", hot_nodes=n // 3,
                hot_passes=passes)


def _run_all(h):
    regs, ks = [], []
    while True:
        ks.append(h.step())
        regs.append(h.registers().clone())
        if ks[-1] == 0:
            break
    return ks, regs


@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("b", [4, 6])
def test_hot_range_equals_plain_gather_bitwise(fp32, b, passes):
    """Counters at every iteration, accumulators and centralities bitwise
    equal to the one-pass gather, for hot ranges of 1 node, a third, n - 1,
    n and beyond n, on an R-MAT graph with split nodes."""
    g = graphs.rmat_graph(scale=15, edge_factor=16, seed=9, device="cuda")
    n = g.n
    ref = hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=11, n=n, fp32=fp32, frontier="off")
    ks0, regs0 = _run_all(ref)
    acc0, cen0 = ref.accumulators(), ref.centralities()
    ref.close()
    for hot in (1, n // 3, n - 1, n, 2 * n):
        h = hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=11, n=n, fp32=fp32, frontier="off",
                          hot_nodes=hot, hot_passes=passes)
        assert h.info()["hot_nodes"] == min(hot, n) and h.info()["hot_passes"] == passes
        ks, regs = _run_all(h)
        assert ks == ks0, hot
        for x, y in zip(regs, regs0):
            assert torch.equal(x, y), hot
        for x, y in zip(h.accumulators(), acc0):
            assert torch.equal(x, y), hot
        cen = h.centralities()
        for key in cen0:
            assert torch.equal(cen[key], cen0[key]), (hot, key)
        h.close()


@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("aps", [1, 4, 16, 128])
def test_hot_range_every_class_sizing(aps, passes):
    g = graphs.rmat_graph(scale=14, edge_factor=12, seed=4, device="cuda")
    ref = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=2, n=g.n, frontier="off", arcs_per_slot=aps)
    ks0, regs0 = _run_all(ref)
    h = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=2, n=g.n, frontier="off", arcs_per_slot=aps,
                      hot_nodes=g.n // 5, hot_passes=passes)
    ks, regs = _run_all(h)
    assert ks == ks0
    assert all(torch.equal(x, y) for x, y in zip(regs, regs0))
    for x, y in zip(h.accumulators(), ref.accumulators()):
        assert torch.equal(x, y)
    ref.close()
    h.close()


def test_hot_range_changed_between_iterations(orc):
    off, tgt = graphs.rmat_graph(scale=12, edge_factor=10, seed=13).numpy()
    n = off.size - 1
    d_off, d_tgt = torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda()
    h = hbl.HyperBall(d_off, d_tgt, log2m=5, seed=3, n=n, frontier="auto")
    c = orc.init(n, 5, 3)
    s, hm = np.zeros(n), np.zeros(n)
    t = 0
    hots = [(0, 1), (n // 2, 2), (17, 1), (n, 2), (0, 2), (n // 9, 1), (n // 3, 2)]
    while True:
        h.set_hot_nodes(*hots[t % len(hots)])
        c, _, k = orc.step(off, tgt, 5, t, c, s, hm)
        assert h.step() == k
        assert np.array_equal(h.registers().cpu().numpy(), c), t
        t += 1
        if k == 0:
            break
    gs, gh = h.accumulators()
    np.testing.assert_allclose(gs.cpu().numpy(), s, rtol=1e-9, atol=0)
    np.testing.assert_allclose(gh.cpu().numpy(), hm, rtol=1e-9, atol=0)
    h.close()


def test_hot_range_rejected_where_it_does_not_apply():
    g = graphs.rmat_graph(scale=10, edge_factor=8, seed=1, device="cuda")
    h = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=1, n=g.n)
    with pytest.raises(hbl.HBError) as e:
        h.set_hot_nodes(-1)
    assert e.value.status == hbl.HB_ERR_INVALID
    with pytest.raises(hbl.HBError) as e:
        h.set_hot_nodes(10, 3)
    assert e.value.status == hbl.HB_ERR_INVALID
    h.close()
    with pytest.raises(hbl.HBError) as e:
        hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=1, n=g.n, hot_nodes=-5)
    assert e.value.status == hbl.HB_ERR_INVALID
    r = hbl.HyperBall.runs(g.offsets, g.targets, 4, [1, 2], n=g.n)
    with pytest.raises(hbl.HBError) as e:
        r.set_hot_nodes(100)
    assert e.value.status == hbl.HB_ERR_INVALID
    r.set_hot_nodes(0)
    r.close()


def test_tuner_chooses_a_hot_range_and_keeps_results(orc):
    # counters of 2^18 nodes x 1 KiB exceed L2, so the tuner tries hot ranges
    g = graphs.rmat_graph(scale=18, edge_factor=4, seed=17, device="cuda")
    ref = hbl.HyperBall(g.offsets, g.targets, log2m=10, seed=5, n=g.n)
    ks0, regs0 = _run_all(ref)
    h = hbl.HyperBall(g.offsets, g.targets, log2m=10, seed=5, n=g.n)
    aps = h.tune()
    info = h.info()
    assert info["arcs_per_slot"] == aps and info["t"] == 0
    assert 0 <= info["hot_nodes"] <= g.n and info["hot_passes"] in (1, 2)
    ks, regs = _run_all(h)
    assert ks == ks0
    assert all(torch.equal(x, y) for x, y in zip(regs, regs0))
    ref.close()
    h.close()
