"""hb_step_noalloc, the iteration for callers that cannot allocate device
memory (it keeps its temporary data in a static device array), checked
against hb_step on a handle: the same counters, changed flags and
accumulators over two calls in a row.  Collected last on purpose, so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl

pytestmark = pytest.mark.gpu

RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


def _graph(kind):
    if kind == "zipf":
        return graphs.plain_graph(n=10_000, seed=1), 4
    # R-MAT with nodes above the split threshold (1024 arcs at p = 64)
    return graphs.rmat_graph(scale=14, edge_factor=24, seed=7), 6


@pytest.mark.parametrize("kind", ["zipf", "rmat"])
def test_noalloc_matches_hb_step_two_calls(kind):
    g, b = _graph(kind)
    off, tgt = g.offsets.cuda(), g.targets.cuda()
    n, m, p = g.n, g.m, 1 << b
    ref = hbl.HyperBall(off, tgt, log2m=b, seed=42, n=n)
    cur = ref.registers().contiguous()          # c_0 in the caller's order
    sumd = torch.zeros(n, dtype=torch.float64, device="cuda")
    harm = torch.zeros(n, dtype=torch.float64, device="cuda")
    for t in range(2):
        nxt = torch.empty((n, p), dtype=torch.uint8, device="cuda")
        changed = torch.empty(n, dtype=torch.uint8, device="cuda")
        k = hbl.hb_step_noalloc(off, tgt, n, m, b, t, cur, nxt, sumd, harm, changed)
        k_ref = ref.step()
        assert k == k_ref
        assert torch.equal(nxt, ref.registers())
        ch_ref, _ = ref.frontier()
        assert torch.equal(changed, ch_ref)
        s_ref, h_ref = ref.accumulators()
        np.testing.assert_allclose(sumd.cpu().numpy(), s_ref.cpu().numpy(), rtol=RTOL, atol=0)
        np.testing.assert_allclose(harm.cpu().numpy(), h_ref.cpu().numpy(), rtol=RTOL, atol=0)
        cur = nxt
    ref.close()


def test_noalloc_rejects_what_does_not_fit():
    # 9M nodes need 72 MB of cached estimates alone, above the 64 MiB maximum
    n = 9_000_000
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    tgt = torch.zeros(1, dtype=torch.int32, device="cuda")
    cur = torch.zeros((n, 16), dtype=torch.uint8, device="cuda")
    nxt = torch.empty_like(cur)
    sumd = torch.zeros(n, dtype=torch.float64, device="cuda")
    harm = torch.zeros_like(sumd)
    changed = torch.empty(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(hbl.HBError) as e:
        hbl.hb_step_noalloc(off, tgt, n, 0, 4, 0, cur, nxt, sumd, harm, changed)
    assert e.value.status == hbl.HB_ERR_INVALID
    assert "scratch" in str(e.value)


def test_noalloc_rejects_host_pointers():
    off = np.array([0, 1, 1], dtype=np.int64)
    tgt = np.array([1], dtype=np.int32)
    regs = np.zeros((2, 16), dtype=np.uint8)
    with pytest.raises(hbl.HBError) as e:
        hbl.hb_step_noalloc(off, tgt, 2, 1, 4, 0, regs, regs.copy(), np.zeros(2), np.zeros(2),
                            np.zeros(2, dtype=np.uint8))
    assert e.value.status == hbl.HB_ERR_INVALID
