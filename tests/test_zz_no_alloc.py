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


def _device_csr(off, tgt):
    return torch.from_numpy(np.ascontiguousarray(off)).cuda(), torch.from_numpy(np.ascontiguousarray(tgt)).cuda()


def _buffers(n, p):
    cur = torch.zeros((n, p), dtype=torch.uint8, device="cuda")
    return (cur, torch.empty_like(cur), torch.zeros(n, dtype=torch.float64, device="cuda"),
            torch.zeros(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("fault", ["offsets_end", "target_is_n", "offsets_decrease", "offsets_start"])
def test_noalloc_refuses_malformed_csr_before_any_gather(fault):
    # the CSR checks run before any kernel reads a counter; the buffers are
    # sized for the caller's stated n and m, so the checks stay in bounds
    off, tgt = graphs.plain_graph(n=2000, seed=3).numpy()
    off, tgt = off.copy(), tgt.copy()
    n, m = off.size - 1, tgt.size
    if fault == "offsets_end":
        off[-1] = m - 1
    elif fault == "target_is_n":
        tgt[m // 3] = n
    elif fault == "offsets_decrease":
        off[n // 2] = off[n // 2 + 1] + 1
    else:
        off[0] = 1
    d_off, d_tgt = _device_csr(off, tgt)
    cur, nxt, sumd, harm, changed = _buffers(n, 16)
    with pytest.raises(hbl.HBError) as e:
        hbl.hb_step_noalloc(d_off, d_tgt, n, m, 4, 0, cur, nxt, sumd, harm, changed)
    assert e.value.status == hbl.HB_ERR_INVALID
    assert "malformed CSR" in str(e.value)
    # nothing was written
    assert not sumd.any() and not harm.any()


def test_noalloc_refuses_overlapping_buffers():
    g = graphs.plain_graph(n=1000, seed=2)
    off, tgt = g.offsets.cuda(), g.targets.cuda()
    n, m = g.n, g.m
    cur, nxt, sumd, harm, changed = _buffers(n, 16)
    cases = {
        "next is cur": (cur, cur, sumd, harm, changed),
        "sumd is harm": (cur, nxt, sumd, sumd, changed),
        "changed inside next": (cur, nxt, sumd, harm, nxt.view(-1)[16:16 + n]),
        "sumd inside cur": (cur, nxt, cur.view(-1)[: 8 * n].view(torch.float64), harm, changed),
    }
    for name, (c, x, s, h, ch) in cases.items():
        with pytest.raises(hbl.HBError) as e:
            hbl.hb_step_noalloc(off, tgt, n, m, 4, 0, c, x, s, h, ch)
        assert e.value.status == hbl.HB_ERR_INVALID, name
        assert "overlap" in str(e.value), name


def test_noalloc_to_fixpoint_matches_oracle():
    import oracle
    g = graphs.rmat_graph(scale=13, edge_factor=8, seed=11)
    off_h, tgt_h = g.numpy()
    n, m, b = g.n, g.m, 5
    p = 1 << b
    c_ref = oracle.init(n, b, 42)
    s_ref, h_ref = np.zeros(n), np.zeros(n)
    hb = hbl.HyperBall(g.offsets.cuda(), g.targets.cuda(), log2m=b, seed=42, n=n)
    cur = hb.registers().contiguous()
    hb.close()
    assert np.array_equal(cur.cpu().numpy(), c_ref)
    off, tgt = g.offsets.cuda(), g.targets.cuda()
    sumd = torch.zeros(n, dtype=torch.float64, device="cuda")
    harm = torch.zeros_like(sumd)
    t = 0
    while True:
        nxt = torch.empty((n, p), dtype=torch.uint8, device="cuda")
        changed = torch.empty(n, dtype=torch.uint8, device="cuda")
        k = hbl.hb_step_noalloc(off, tgt, n, m, b, t, cur, nxt, sumd, harm, changed)
        c_ref, ch_ref, k_ref = oracle.step(off_h, tgt_h, b, t, c_ref, s_ref, h_ref)
        assert k == k_ref, t
        assert np.array_equal(nxt.cpu().numpy(), c_ref), t
        assert np.array_equal(changed.cpu().numpy(), ch_ref), t
        np.testing.assert_allclose(sumd.cpu().numpy(), s_ref, rtol=RTOL, atol=0)
        np.testing.assert_allclose(harm.cpu().numpy(), h_ref, rtol=RTOL, atol=0)
        cur = nxt
        t += 1
        if k == 0:
            break
    assert t >= 4


def test_noalloc_debug_build_keeps_error_word_clear():
    # the debug build checks every arc target in the gather; on a valid
    # graph the check never fires and the call returns HB_OK
    import os
    import subprocess
    import sys
    import textwrap
    from paper_1308_2144_gb300 import build
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib = build.build(debug=True)
    child = textwrap.dedent("""
        import numpy as np, torch
        import oracle
        from paper_1308_2144_gb300 import graphs, hyperball as hbl
        assert hbl.LIB_PATH.endswith("libhyperball_debug.so"), hbl.LIB_PATH
        g = graphs.plain_graph(n=3000, seed=4)
        off_h, tgt_h = g.numpy()
        n, m = g.n, g.m
        c = oracle.init(n, 4, 9)
        s, h = np.zeros(n), np.zeros(n)
        cur = torch.from_numpy(c).cuda()
        sumd = torch.zeros(n, dtype=torch.float64, device="cuda")
        harm = torch.zeros_like(sumd)
        for t in range(3):
            nxt = torch.empty_like(cur)
            changed = torch.empty(n, dtype=torch.uint8, device="cuda")
            k = hbl.hb_step_noalloc(g.offsets.cuda(), g.targets.cuda(), n, m, 4, t, cur, nxt, sumd, harm,
                                    changed)
            c, _, k_ref = oracle.step(off_h, tgt_h, 4, t, c, s, h)
            assert k == k_ref and np.array_equal(nxt.cpu().numpy(), c), t
            cur = nxt
        print("noalloc debug ok")
    """)
    env = dict(os.environ, HYPERBALL_LIB=lib, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", child], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "noalloc debug ok" in r.stdout
