"""Create-time graph passes at larger sizes (2^19 and 2^20 nodes): the
in-degree histogram shared by the degree-sorted relabelling and the reverse
CSR, the relabelled arcs written in their own order, the reverse CSR of the
pushed frontier and the device transpose (HB_TRANSPOSE) give the oracle's
counters at every iteration, with duplicate arcs, self-loops, nodes without
in-arcs and with the relabelling off."""
import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl
from tests.test_gpu_parity import close, to_dev

pytestmark = pytest.mark.gpu

N_PLAIN = (1 << 19) + 1234


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


def with_duplicates(off, tgt):
    """The same graph with every 7th arc doubled and a self-loop on every
    5th node."""
    n = off.size - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    s_all = np.concatenate([src, src[::7], np.arange(0, n, 5)])
    d_all = np.concatenate([tgt, tgt[::7], np.arange(0, n, 5, dtype=np.int32)])
    order = np.argsort(s_all, kind="stable")
    off2 = np.zeros(n + 1, dtype=np.int64)
    off2[1:] = np.cumsum(np.bincount(s_all, minlength=n))
    return off2, d_all[order].astype(np.int32)


def transpose_np(off, tgt):
    """The transpose CSR, every arc kept."""
    n = off.size - 1
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(off))
    order = np.argsort(tgt, kind="stable")
    toff = np.zeros(n + 1, dtype=np.int64)
    toff[1:] = np.cumsum(np.bincount(tgt, minlength=n))
    return toff, src[order]


def walk(orc, hb, off, tgt, b, seed):
    """GPU and oracle side by side, one iteration at a time."""
    n = off.size - 1
    c = orc.init(n, b, seed)
    sumd, harm = np.zeros(n), np.zeros(n)
    t = 0
    while True:
        nxt, _, k = orc.step(off, tgt, b, t, c, sumd, harm)
        assert hb.step() == k, t
        assert np.array_equal(hb.registers().cpu().numpy(), nxt), t
        c = nxt
        t += 1
        if k == 0:
            break
    gs, gh = hb.accumulators()
    close(gs.cpu().numpy(), sumd)
    close(gh.cpu().numpy(), harm)
    return t


@pytest.mark.parametrize("kind,frontier,relabel", [("plain", "push", True), ("plain_dups", "auto", True),
                                                   ("plain_dups", "push", False), ("rmat", "push", True)])
def test_large_reverse_lists_and_relabelling(orc, kind, frontier, relabel):
    if kind.startswith("plain"):
        off, tgt = graphs.plain_graph(n=N_PLAIN, seed=3).numpy()
    else:
        off, tgt = graphs.rmat_graph(scale=20, edge_factor=4, seed=5).numpy()
    if kind.endswith("dups"):
        off, tgt = with_duplicates(off, tgt)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=11, n=off.size - 1, frontier=frontier,
                       relabel=relabel)
    assert walk(orc, hb, off, tgt, 4, 11) > 2
    hb.close()


def test_large_device_transpose(orc):
    off, tgt = with_duplicates(*graphs.plain_graph(n=N_PLAIN, seed=4).numpy())
    # hand over G^T; the library scans its transpose, the graph above
    hb = hbl.HyperBall(*to_dev(*transpose_np(off, tgt)), log2m=4, seed=12, n=off.size - 1, transpose=True,
                       frontier="push")
    walk(orc, hb, off, tgt, 4, 12)
    hb.close()


def test_large_host_upload_checked_by_chunks(orc):
    """Targets from host memory (2^23 arcs and more) are uploaded in chunks,
    each checked and counted as it arrives: pageable and pinned host CSRs
    give the oracle's run, and a target out of range in the last chunk is
    refused with HB_ERR_INVALID while the library stays usable."""
    off, tgt = graphs.rmat_graph(scale=21, edge_factor=6, seed=21).numpy()
    n = off.size - 1
    assert tgt.size >= 1 << 23
    ref = orc.run(off, tgt, 4, 5)
    for pinned in (False, True):
        o, t = torch.from_numpy(off), torch.from_numpy(tgt)
        if pinned:
            o, t = o.pin_memory(), t.pin_memory()
        hb = hbl.HyperBall(o, t, log2m=4, seed=5, n=n)
        assert hb.run() == ref.steps
        assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
        hb.close()
    bad = tgt.copy()
    bad[-3] = n
    with pytest.raises(hbl.HBError) as e:
        hbl.HyperBall(torch.from_numpy(off), torch.from_numpy(bad), log2m=4, seed=5, n=n)
    assert e.value.status == hbl.HB_ERR_INVALID
    assert "outside" in str(e.value)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=5, n=n)
    assert hb.run() == ref.steps
    hb.close()


@pytest.mark.parametrize("relabel,transpose", [(False, False), (False, True), (True, True)])
def test_sparse_graph_with_long_empty_runs(orc, relabel, transpose):
    """3,000 arcs over 60,000 nodes: a 2048-arc tile's sources span far more
    than 2048 nodes, so the arc passes (reverse lists of the graph in the
    caller's order, the device transpose) search all offsets per arc."""
    n = 60_000
    rng = np.random.default_rng(12)
    edges = list(zip(rng.integers(0, n, 3000).tolist(), rng.integers(0, n, 3000).tolist()))
    off, tgt = graphs.from_edges(n, edges, keep_all=True).numpy()
    given = transpose_np(off, tgt) if transpose else (off, tgt)
    hb = hbl.HyperBall(*to_dev(*given), log2m=4, seed=3, n=n, frontier="push", relabel=relabel,
                       transpose=transpose)
    assert walk(orc, hb, off, tgt, 4, 3) >= 2
    hb.close()
