"""The reverse CSR that pushed frontier iterations walk (Sec. 5 / 5.1:
changed counters are pushed to the predecessors that must be recomputed),
on graphs of 8-12M arcs with a hub whose reverse list holds up to 8.4M
repeated arcs, next to R-MAT arcs and sources of degree 0; also in the
caller's order (reverse lists counted by the library, not from the in-degree
precount) and for a graph the library transposes itself.  A missing,
duplicated or misplaced reverse arc changes the pushed union, so the
counters must equal the oracle's bit for bit with every iteration that can
push pushing.  Also the reverse lists built on a second stream under the
first iterations: pushed and automatic frontiers, the two-phase gather's
reordering of the target lists asked for before the first step, and
handles destroyed while the build may still run."""
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


def _csr(n, src, dst):
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, src + 1, 1)
    return np.cumsum(off), dst.astype(np.int32)


def _hub_graph(seed, n=1 << 20, hub_arcs=8, rmat_ef=4):
    """R-MAT(2^20) plus hub_arcs repeated arcs from every even node into one
    hub (4.2M arcs for 8, 8.4M for 16)."""
    rng = np.random.default_rng(seed)
    g = graphs.rmat_graph(scale=20, edge_factor=rmat_ef, seed=seed)
    off, tgt = g.numpy()
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    hub = int(rng.integers(n))
    hs = np.repeat(np.arange(0, n, 2, dtype=np.int64), hub_arcs)
    return _csr(n, np.concatenate([src, hs]), np.concatenate([tgt.astype(np.int64), np.full(hs.size, hub)]))


@pytest.mark.parametrize("hub_arcs,ef", [(0, 8), (8, 4), (16, 4)])
def test_hub_reverse_csr_against_oracle(orc, hub_arcs, ef):
    off, tgt = _hub_graph(31 + hub_arcs, hub_arcs=hub_arcs, rmat_ef=ef)
    walk_parity(orc, off, tgt, 4, 7, check_every_step=False, frontier="push")


def test_hub_reverse_csr_caller_order_and_transpose(orc):
    # the caller's order kept (no in-degree precount), and the scanned graph
    # built by the library's own transpose of G
    off, tgt = _hub_graph(5, hub_arcs=8)
    walk_parity(orc, off, tgt, 4, 3, check_every_step=False, frontier="push", relabel=False)
    n = off.size - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    toff, ttgt = _csr(n, tgt.astype(np.int64), src)   # G, whose transpose is (off, tgt)
    ref = orc.run(off, tgt, 4, 3)
    h = hbl.HyperBall(torch.from_numpy(toff).cuda(), torch.from_numpy(ttgt).cuda(), log2m=4, seed=3, n=n,
                      transpose=True, frontier="push")
    assert h.run() == ref.steps
    assert np.array_equal(h.registers().cpu().numpy(), ref.regs)
    h.close()


# Graphs of at least 2^20 arcs made through hb_create build their reverse
# lists on a second stream while the first iterations gather; the handle's
# stream waits for them before the first iteration that may push, before the
# two-phase gather reorders the target lists, and at destroy.

@pytest.mark.parametrize("frontier,hot_passes", [("push", 0), ("auto", 0), ("auto", 1), ("auto", 2)])
def test_reverse_lists_built_under_the_first_iterations(orc, frontier, hot_passes):
    off, tgt = graphs.rmat_graph(scale=18, edge_factor=16, seed=41).numpy()
    n = off.size - 1
    assert tgt.size >= 1 << 20
    hot = dict(hot_nodes=n // 8, hot_passes=hot_passes) if hot_passes else {}
    walk_parity(orc, off, tgt, 4, 9, frontier=frontier, **hot)


def test_targets_reordered_right_after_create(orc):
    # the two-phase gather's reordering of every target list, asked for
    # before the first step, while the reverse lists may still be built
    off, tgt = graphs.rmat_graph(scale=18, edge_factor=16, seed=43).numpy()
    n = off.size - 1
    d_off, d_tgt = torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda()
    h = hbl.HyperBall(d_off, d_tgt, log2m=5, seed=2, n=n, frontier="auto")
    h.set_hot_nodes(n // 5, 2)
    c = orc.init(n, 5, 2)
    s, hm = np.zeros(n), np.zeros(n)
    t = 0
    pushed = 0
    while True:
        c, _, k = orc.step(off, tgt, 5, t, c, s, hm)
        assert h.step() == k
        pushed += h.info()["last_sparse"]
        assert np.array_equal(h.registers().cpu().numpy(), c), t
        t += 1
        if k == 0:
            break
    assert pushed > 0
    h.close()


def test_destroy_while_reverse_lists_may_be_built(orc):
    g = graphs.rmat_graph(scale=20, edge_factor=16, seed=45, device="cuda")
    for seed in range(4):
        h = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=seed, n=g.n, frontier="push")
        h.close()
    off, tgt = g.numpy()
    ref = orc.run(off, tgt, 4, 6)
    h = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=6, n=g.n, frontier="push")
    assert h.run() == ref.steps
    assert np.array_equal(h.registers().cpu().numpy(), ref.regs)
    h.close()
