"""Packed registers on the GPU (HB_PACKED_REGISTERS, Sec. 4.1 register
width: six bits per register, counters of 3p/4 bytes) against the oracle's
packed iteration and against the byte-register handle.

Packing changes how the registers are stored, never their values (every
register value, at most 64 - log2m, fits in six bits), so the counters at
every iteration must equal the oracle's packed counters unpacked, and the
accumulators and centralities must equal those of the same handle with
byte registers bit for bit (the same per-node arithmetic on the same
values).  Cases: every log2m, heavy (split) nodes and every degree-class
boundary, every class sizing, both precisions, both node orders, the
transposed graph, the discount and neighbourhood accumulators, reset and
the autotuner at a size whose counters exceed L2, the encyclopedia-like
graph, and every option the packed form refuses."""
import ctypes
import os

import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl
from tests.test_gpu_parity import _degree_boundary_graph, close, walk_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


def _packed_walk_parity(orc, off, tgt, b, seed, **opts):
    """GPU packed handle beside the oracle's packed iteration (step_packed),
    one iteration at a time."""
    n = off.size - 1
    d_off, d_tgt = torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda()
    h = hbl.HyperBall(d_off, d_tgt, log2m=b, seed=seed, n=n, frontier="off", packed=True, **opts)
    assert h.info()["packed"] == 1
    c = orc.pack6(orc.init(n, b, seed), b)
    sumd, harm = np.zeros(n), np.zeros(n)
    assert np.array_equal(h.registers().cpu().numpy(), orc.unpack6(c, b))
    t = 0
    while True:
        c, ch, k = orc.step_packed(off, tgt, b, t, c, sumd, harm)
        assert h.step() == k, t
        assert np.array_equal(h.registers().cpu().numpy(), orc.unpack6(c, b)), t
        gch, _ = h.frontier()
        assert np.array_equal(gch.cpu().numpy(), ch), t
        gs, gh = h.accumulators()
        close(gs.cpu().numpy(), sumd)
        close(gh.cpu().numpy(), harm)
        t += 1
        if k == 0:
            break
    fin = orc.finalize(b, orc.unpack6(c, b), sumd, harm)
    cen = {key: v.cpu().numpy() for key, v in h.centralities().items()}
    for key in ("closeness", "harmonic", "lin", "reachable"):
        close(cen[key], fin[key])
    h.close()
    return t


@pytest.mark.parametrize("b", list(range(4, 13)))
def test_packed_every_log2m_against_packed_oracle(orc, b):
    off, tgt = graphs.rmat_graph(scale=11, edge_factor=8, seed=80 + b).numpy()
    assert _packed_walk_parity(orc, off, tgt, b, 900 + b) > 3


@pytest.mark.parametrize("relabel", [True, False])
def test_packed_plain_workload_and_layouts(orc, relabel):
    off, tgt = graphs.plain_graph(n=10_000, seed=1).numpy()
    _packed_walk_parity(orc, off, tgt, 4, 42, relabel=relabel)


@pytest.mark.parametrize("b", [4, 6, 9, 12])
def test_packed_degree_class_boundaries(orc, b):
    # heavy nodes split into chunks, every class boundary (walk against the
    # byte-register oracle, frontier flags included)
    off, tgt = _degree_boundary_graph(b)
    walk_parity(orc, off, tgt, b, 5, check_every_step=(b <= 6), frontier="off", packed=True)


def test_packed_empty_and_isolated_graphs(orc):
    for n in (0, 1, 37):
        off = np.zeros(n + 1, dtype=np.int64)
        tgt = np.zeros(0, dtype=np.int32)
        h = hbl.HyperBall(torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda(), log2m=5, seed=3, n=n,
                          frontier="off", packed=True)
        assert h.step() == 0
        if n:
            regs = h.registers().cpu().numpy()
            assert np.array_equal(regs, orc.init(n, 5, 3))
        h.close()


def _run_all(h):
    regs, ks = [], []
    while True:
        ks.append(h.step())
        regs.append(h.registers().clone())
        if ks[-1] == 0:
            break
    return ks, regs


def _same_handles(g, b, seed, opts, check_regs=True):
    """A byte-register and a packed handle of the same graph and options:
    the same changed counts and counters at every iteration, bitwise equal
    accumulators and centralities."""
    ref = hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=seed, n=g.n, frontier="off", **opts)
    pk = hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=seed, n=g.n, frontier="off", packed=True, **opts)
    if check_regs:
        ks0, regs0 = _run_all(ref)
        ks, regs = _run_all(pk)
        assert ks == ks0
        for t, (x, y) in enumerate(zip(regs, regs0)):
            assert torch.equal(x, y), t
    else:
        assert pk.run() == ref.run()
        assert torch.equal(pk.registers(), ref.registers())
    for x, y in zip(pk.accumulators(), ref.accumulators()):
        assert torch.equal(x, y)
    c0, c1 = ref.centralities(), pk.centralities()
    for key in c0:
        assert torch.equal(c1[key], c0[key]), key
    return ref, pk


@pytest.mark.parametrize("relabel", [True, False])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("b", [4, 6, 9, 12])
def test_packed_equals_byte_registers_bitwise(b, fp32, relabel):
    g = graphs.rmat_graph(scale=15 if b < 12 else 13, edge_factor=16, seed=9, device="cuda")
    ref, pk = _same_handles(g, b, 11, dict(fp32=fp32, relabel=relabel))
    # the packed counters take 3/4 of the bytes
    info0, info1 = ref.info(), pk.info()
    assert info0["packed"] == 0 and info1["packed"] == 1
    saved = info0["device_bytes"] - info1["device_bytes"]
    assert abs(saved - 2 * g.n * (1 << b) // 4) <= 1024, (saved, g.n)
    ref.close()
    pk.close()


@pytest.mark.parametrize("aps", [1, 4, 16, 128])
def test_packed_every_class_sizing(aps):
    g = graphs.rmat_graph(scale=14, edge_factor=12, seed=4, device="cuda")
    ref, pk = _same_handles(g, 5, 2, dict(arcs_per_slot=aps))
    assert pk.info()["arcs_per_slot"] == aps
    ref.close()
    pk.close()


def test_packed_transpose_discount_neighbourhood_reset():
    g = graphs.rmat_graph(scale=13, edge_factor=10, seed=31, device="cuda")
    opts = dict(transpose=True, neighbourhood=True)
    ref = hbl.HyperBall(g.offsets, g.targets, log2m=6, seed=7, n=g.n, frontier="off", **opts)
    pk = hbl.HyperBall(g.offsets, g.targets, log2m=6, seed=7, n=g.n, frontier="off", packed=True, **opts)
    f = np.array([1.0, 0.5, 0.25, 0.125, 1.0 / 16])
    for seed in (7, 1234):
        for h in (ref, pk):
            h.reset(seed)
            h.set_discount(f)
            h.run()
        assert torch.equal(pk.registers(), ref.registers())
        assert torch.equal(pk.discounted(), ref.discounted())
        assert np.array_equal(pk.neighbourhood(), ref.neighbourhood())
        for x, y in zip(pk.accumulators(), ref.accumulators()):
            assert torch.equal(x, y)
    ref.close()
    pk.close()


def test_packed_tuner_keeps_results():
    # 2^18 nodes x 768 bytes exceed L2: the tuner sizes the classes only
    g = graphs.rmat_graph(scale=18, edge_factor=4, seed=17, device="cuda")
    ref = hbl.HyperBall(g.offsets, g.targets, log2m=10, seed=5, n=g.n, frontier="off")
    ks0, regs0 = _run_all(ref)
    pk = hbl.HyperBall(g.offsets, g.targets, log2m=10, seed=5, n=g.n, frontier="off", packed=True)
    aps = pk.tune()
    info = pk.info()
    assert info["arcs_per_slot"] == aps and info["hot_nodes"] == 0 and info["t"] == 0
    ks, regs = _run_all(pk)
    assert ks == ks0
    assert all(torch.equal(x, y) for x, y in zip(regs, regs0))
    ref.close()
    pk.close()


def test_packed_refusals(tmp_path):
    g = graphs.rmat_graph(scale=10, edge_factor=8, seed=1, device="cuda")

    def status(fn):
        with pytest.raises(hbl.HBError) as e:
            fn()
        return e.value.status

    for frontier in ("auto", "pull", "push"):
        assert status(lambda: hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=1, n=g.n, frontier=frontier,
                                            packed=True)) == hbl.HB_ERR_INVALID
    assert status(lambda: hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=1, n=g.n, frontier="off",
                                        packed=True, hot_nodes=100)) == hbl.HB_ERR_INVALID
    assert status(lambda: hbl.HyperBall.runs(g.offsets, g.targets, 4, [1, 2], n=g.n, frontier="off",
                                             packed=True)) == hbl.HB_ERR_INVALID
    assert status(lambda: hbl.HyperBallBatch([(g.offsets, g.targets, g.n, 4, 1)], frontier="off",
                                             packed=True)) == hbl.HB_ERR_INVALID
    h = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=1, n=g.n, frontier="off", packed=True)
    assert status(lambda: h.set_hot_nodes(10)) == hbl.HB_ERR_STATE
    h.set_hot_nodes(0)
    assert status(lambda: h.set_weights(torch.ones(g.n, dtype=torch.int64))) == hbl.HB_ERR_STATE
    path = str(tmp_path / "ck.bin")
    assert status(lambda: h.save(path)) == hbl.HB_ERR_STATE
    assert not os.path.exists(path) or os.path.getsize(path) == 0
    ref = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=1, n=g.n, frontier="off")
    ref.save(path)
    assert status(lambda: hbl.hb_load(path, hbl.make_options(frontier="off", packed=True))) == hbl.HB_ERR_INVALID
    # the handle still works after every refusal
    assert h.run() == ref.run()
    assert torch.equal(h.registers(), ref.registers())
    h.close()
    ref.close()


def test_packed_server_refused():
    L = hbl.load()
    o = hbl.ServerOptions()
    L.hb_server_default_options(ctypes.byref(o))
    o.flags = hbl.HB_PACKED_REGISTERS
    h = hbl._vp()
    assert L.hb_server_create(ctypes.byref(o), ctypes.byref(h)) == hbl.HB_ERR_INVALID
    assert not h.value


def test_packed_encyclopedia_like_full_size():
    """The encyclopedia-like graph (4,206,785 nodes, about 10^8 arcs) at
    p = 64: fixpoint, counters, accumulators and centralities of the packed
    handle equal the byte-register handle's bit for bit."""
    g = graphs.enwiki_graph(device="cuda")
    ref, pk = _same_handles(g, 6, 1, dict(), check_regs=False)
    assert pk.info()["total_arcs"] == ref.info()["total_arcs"]
    ref.close()
    pk.close()


def test_packed_profile_counts_packed_bytes():
    """HB_PROFILE's algorithmic bytes count a packed counter read or write
    as 3p/4 bytes: against byte registers, every dense launch (all of them
    with HB_FRONTIER_OFF) differs by (m + 2 N) p/4, N the nodes recomputed."""
    g = graphs.rmat_graph(scale=14, edge_factor=8, seed=12, device="cuda")
    b = 6
    infos = []
    for packed in (False, True):
        h = hbl.HyperBall(g.offsets, g.targets, log2m=b, seed=4, n=g.n, frontier="off", profile=True, packed=packed)
        h.run()
        infos.append(h.info())
        h.close()
    ib, ip = infos
    assert ib["kernel_launches"] == ip["kernel_launches"] == ib["t"]
    diff = ib["kernel_bytes"] - ip["kernel_bytes"]
    want = ib["kernel_launches"] * (g.m + 2 * ib["last_nodes"]) * (1 << b) / 4
    assert diff == pytest.approx(want, rel=1e-12)
