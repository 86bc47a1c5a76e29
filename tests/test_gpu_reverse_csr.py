"""The reverse CSR that pushed frontier iterations walk (Sec. 5 / 5.1:
changed counters are pushed to the predecessors that must be recomputed),
on graphs of 8-12M arcs with a hub whose reverse list holds up to 8.4M
repeated arcs, next to R-MAT arcs and sources of degree 0; also in the
caller's order (reverse lists counted by the library, not from the in-degree
precount) and for a graph the library transposes itself.  A missing,
duplicated or misplaced reverse arc changes the pushed union, so the
counters must equal the oracle's bit for bit with every iteration that can
push pushing."""
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
