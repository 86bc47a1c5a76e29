"""GPU path against the oracle, element by element, through the C ABI.

Bar: registers, changed sets, must-check sets and iteration counts
bit-exact; FP64 accumulators and centralities within 1e-9 relative (the
only difference allowed is the last bit of the natural logarithm in the
small-range estimator: glibc and CUDA's log may differ by an ulp).
"""
import math
import os

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


def close(a, b, rtol=RTOL):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape
    np.testing.assert_allclose(a, b, rtol=rtol, atol=0)


def to_dev(off, tgt):
    return torch.from_numpy(np.ascontiguousarray(off)).cuda(), torch.from_numpy(np.ascontiguousarray(tgt)).cuda()


def walk_parity(orc, off, tgt, b, seed, check_every_step=True, **opts):
    """Run GPU and oracle side by side, one iteration at a time."""
    n = off.size - 1
    d_off, d_tgt = to_dev(off, tgt)
    hb = hbl.HyperBall(d_off, d_tgt, log2m=b, seed=seed, n=n, **opts)
    c = orc.init(n, b, seed)
    sumd = np.zeros(n)
    harm = np.zeros(n)
    assert np.array_equal(hb.registers().cpu().numpy(), c)
    t = 0
    while True:
        nxt, ch, k = orc.step(off, tgt, b, t, c, sumd, harm)
        kg = hb.step()
        assert kg == k, (t, kg, k)
        if check_every_step or k == 0:
            assert np.array_equal(hb.registers().cpu().numpy(), nxt), t
            gch, gmust = hb.frontier()
            assert np.array_equal(gch.cpu().numpy(), ch), t
            assert np.array_equal(gmust.cpu().numpy(), orc.must_check(off, tgt, ch)), t
            gs, gh = hb.accumulators()
            close(gs.cpu().numpy(), sumd)
            close(gh.cpu().numpy(), harm)
        c = nxt
        t += 1
        if k == 0:
            break
    info = hb.info()
    assert info["t"] == t and info["converged"] == 1
    fin = orc.finalize(b, c, sumd, harm)
    cen = {k: v.cpu().numpy() for k, v in hb.centralities().items()}
    for key in ("closeness", "harmonic", "lin", "reachable"):
        close(cen[key], fin[key])
    hb.close()
    return t


# ------------------------------------------------------------- workloads --

@pytest.fixture(scope="module")
def plain():
    return graphs.plain_graph(n=10_000, seed=1).numpy()


def test_plain_workload_every_step(orc, plain):
    """The 10,000-node Zipf(2.1) workload, log2m = 4, hash seed 42."""
    off, tgt = plain
    steps = walk_parity(orc, off, tgt, 4, 42)
    assert steps > 3


@pytest.mark.parametrize("b", list(range(4, 13)))
def test_every_log2m(orc, b):
    off, tgt = graphs.plain_graph(n=1500, seed=b).numpy()
    walk_parity(orc, off, tgt, b, 1000 + b)


@pytest.mark.parametrize("frontier,pull_gather", [("auto", False), ("auto", True), ("push", False),
                                                  ("push", True), ("pull", False), ("off", False)])
@pytest.mark.parametrize("relabel", [True, False])
def test_frontier_policies_and_layouts(orc, frontier, pull_gather, relabel):
    off, tgt = graphs.rmat_graph(scale=12, edge_factor=8, seed=21).numpy()
    walk_parity(orc, off, tgt, 5, 77, frontier=frontier, relabel=relabel, pull_gather=pull_gather)


@pytest.mark.parametrize("b", list(range(4, 13)))
def test_pushed_union_every_log2m(orc, b):
    """Every iteration after the first is a frontier iteration (push policy),
    done by the pushed union: counters, frontier and accumulators equal the
    oracle's full recomputation at every step, for every log2m."""
    off, tgt = graphs.rmat_graph(scale=11, edge_factor=8, seed=30 + b).numpy()
    walk_parity(orc, off, tgt, b, 500 + b, frontier="push")


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("frontier", ["auto", "push"])
def test_pushed_and_gathered_frontiers_agree_bitwise(fp32, frontier):
    """Pushing last iteration's changed counters and gathering every
    successor give the same union, so the two runs agree bit for bit in
    counters, frontier, accumulators and centralities (both precisions)."""
    g = graphs.rmat_graph(scale=14, edge_factor=12, seed=5, device="cuda")
    hs = [hbl.HyperBall(g.offsets, g.targets, log2m=6, seed=3, n=g.n, fp32=fp32, frontier=frontier,
                        pull_gather=pg) for pg in (False, True)]
    while True:
        ks = [h.step() for h in hs]
        assert ks[0] == ks[1]
        assert torch.equal(hs[0].registers(), hs[1].registers())
        f0, f1 = hs[0].frontier(), hs[1].frontier()
        assert torch.equal(f0[0], f1[0]) and torch.equal(f0[1], f1[1])
        if ks[0] == 0:
            break
    for x, y in zip(hs[0].accumulators(), hs[1].accumulators()):
        assert torch.equal(x, y)
    c0, c1 = hs[0].centralities(), hs[1].centralities()
    for key in c0:
        assert torch.equal(c0[key], c1[key])
    i0, i1 = hs[0].info(), hs[1].info()
    assert i0["t"] == i1["t"] and i0["total_arcs"] <= i1["total_arcs"]
    for h in hs:
        h.close()


def _degree_boundary_graph(b, seed=3):
    """Nodes whose degrees sit on every class boundary of the step kernel
    for every class sizing: 0, 1, 2^k - 1, 2^k, 2^k + 1 up to the heavy
    threshold, the heavy threshold +-1, several heavy chunks."""
    p = 1 << b
    L = min(p // 16, 32)
    smax = 32 // L
    chunk = 64 * smax
    heavy = 2 * chunk
    # light class bounds are aps * 2^k (aps and 2^k powers of two)
    degs = [0, 3, heavy - 1, heavy, heavy + 1, 3 * chunk + 5, 7 * chunk]
    k = 1
    while k < heavy:
        degs += [k - 1, k, k + 1]
        k *= 2
    degs = sorted(set(d for d in degs if d >= 0))
    n = max(4 * max(degs), 5000)
    rng = np.random.default_rng(seed)
    edges = []
    for i, d in enumerate(degs):
        for tgt in rng.choice(n, size=d, replace=False):
            edges.append((i, int(tgt)))
    for v in range(len(degs), n):   # background: small random out-degrees
        for tgt in rng.integers(0, n, size=int(rng.integers(0, 4))):
            edges.append((v, int(tgt)))
    return graphs.from_edges(n, edges, keep_all=True).numpy()


@pytest.mark.parametrize("b", [4, 6, 9, 12])
def test_degree_class_boundaries(orc, b):
    off, tgt = _degree_boundary_graph(b)
    walk_parity(orc, off, tgt, b, 5, check_every_step=(b <= 6))


def test_hub_with_many_predecessors(orc):
    # one node reached from almost every node: exercises the grid-wide push
    n = 6000
    rng = np.random.default_rng(8)
    edges = [(v, 0) for v in range(1, n)] + [(0, int(w)) for w in rng.integers(1, n, 50)]
    edges += [(int(u), int(w)) for u, w in rng.integers(1, n, size=(3 * n, 2))]
    off, tgt = graphs.from_edges(n, edges, keep_all=False).numpy()
    walk_parity(orc, off, tgt, 4, 9, frontier="push")
    walk_parity(orc, off, tgt, 4, 9, frontier="push", pull_gather=True)


@pytest.mark.parametrize("name", ["path", "cycle", "star_out", "star_in", "complete", "loops_dups",
                                  "isolated"])
def test_small_structured_graphs(orc, name):
    from tests.test_oracle_hyperball import SMALL
    off, tgt = SMALL[name]
    walk_parity(orc, off, tgt, 4, 42)


def test_empty_graph():
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    tgt = torch.zeros(0, dtype=torch.int32, device="cuda")
    hb = hbl.HyperBall(off, tgt, log2m=4, seed=1, n=0)
    assert hb.run() == 1
    assert hb.registers().numel() == 0
    hb.close()


# ------------------------------------------------------------ interfaces --

def test_host_and_device_pointers_int32_and_int64(orc, plain):
    off, tgt = plain
    ref = orc.run(off, tgt, 4, 42)
    variants = [
        dict(offsets=off, targets=tgt),                                        # host, int64
        dict(offsets=off.astype(np.int32), targets=tgt),                        # host, int32
        dict(offsets=torch.from_numpy(off.astype(np.int32)).cuda(), targets=torch.from_numpy(tgt).cuda()),
        dict(offsets=torch.from_numpy(off).cuda(), targets=torch.from_numpy(tgt).cuda(), borrow=True),
    ]
    for v in variants:
        o, t_ = v.pop("offsets"), v.pop("targets")
        hb = hbl.HyperBall(o, t_, log2m=4, seed=42, n=off.size - 1, **v)
        assert hb.run() == ref.steps
        assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
        s, h = hb.accumulators(device="cpu")
        close(s.numpy(), ref.sumd)
        close(h.numpy(), ref.harm)
        hb.close()


def test_transpose_flag_matches_transposed_input(orc):
    g = graphs.rmat_graph(scale=11, edge_factor=6, seed=5)        # this is S = G^T
    gt = graphs.transpose(g)                                        # G
    off, tgt = g.numpy()
    ref = orc.run(off, tgt, 6, 3)
    o2, t2 = gt.numpy()
    hb = hbl.HyperBall(*to_dev(o2, t2), log2m=6, seed=3, n=g.n, transpose=True)
    assert hb.run() == ref.steps
    assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
    hb.close()


def test_max_steps_and_continue(orc, plain):
    off, tgt = plain
    ref = orc.run(off, tgt, 4, 42)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=42, n=off.size - 1, max_steps=2)
    with pytest.raises(hbl.HBNotConverged):
        hb.run()
    assert hb.info()["t"] == 2
    while hb.step() != 0:
        pass
    assert hb.info()["t"] == ref.steps
    assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
    hb.close()


def test_step_after_convergence_changes_nothing(orc, plain):
    off, tgt = plain
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=42, n=off.size - 1)
    hb.run()
    regs = hb.registers().cpu().numpy()
    s0, h0 = hb.accumulators(device="cpu")
    assert hb.step() == 0
    assert np.array_equal(hb.registers().cpu().numpy(), regs)
    s1, h1 = hb.accumulators(device="cpu")
    assert torch.equal(s0, s1) and torch.equal(h0, h1)
    hb.close()


def test_reset_equals_fresh_handle(orc, plain):
    off, tgt = plain
    ref = orc.run(off, tgt, 4, 1234)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=42, n=off.size - 1)
    hb.run()
    hb.reset(1234)
    assert hb.run() == ref.steps
    assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
    hb.close()


@pytest.mark.parametrize("frontier", ["auto", "pull"])
def test_checkpoint_resume_is_bit_identical(tmp_path, plain, frontier):
    off, tgt = plain
    full = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=42, n=off.size - 1, frontier=frontier)
    full.run()
    a = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=42, n=off.size - 1, frontier=frontier)
    for _ in range(3):
        a.step()
    path = str(tmp_path / "hb.ckpt")
    a.save(path)
    a.close()
    with pytest.raises(hbl.HBError) as e:   # a class sizing that is no candidate
        hbl.hb_load(path, hbl.make_options(frontier=frontier, arcs_per_slot=3))
    assert e.value.status == hbl.HB_ERR_INVALID
    # the loaded handle takes its class sizing from the options (results never depend on it)
    h = hbl.hb_load(path, hbl.make_options(frontier=frontier, arcs_per_slot=64 if frontier == "auto" else 0))
    b = hbl.HyperBall.__new__(hbl.HyperBall)
    b._h, b.n, b.p, b.log2m = h, off.size - 1, 16, 4
    b.run()
    assert b.info()["t"] == full.info()["t"]
    assert torch.equal(b.registers(), full.registers())
    for x, y in zip(b.accumulators(), full.accumulators()):
        assert torch.equal(x, y)
    b.close()
    full.close()


@pytest.mark.parametrize("bad", ["first", "last", "decrease", "target_high", "target_neg"])
@pytest.mark.parametrize("where", ["device", "host"])
def test_malformed_csr_is_rejected(bad, where):
    off = np.array([0, 2, 3, 5, 6], dtype=np.int64)
    tgt = np.array([1, 2, 0, 3, 1, 2], dtype=np.int32)
    n, m = 4, 6
    if bad == "first":
        off[0] = 1
    elif bad == "last":
        off[-1] = 5
    elif bad == "decrease":
        off[2] = 1
    elif bad == "target_high":
        tgt[3] = 4
    else:
        tgt[0] = -1
    o, t = torch.from_numpy(off), torch.from_numpy(tgt)
    if where == "device":
        o, t = o.cuda(), t.cuda()
    with pytest.raises(hbl.HBError) as e:
        hbl.hb_create(o, t, n, m, 4, 1)
    assert e.value.status == hbl.HB_ERR_INVALID


# --------------------------------------------------------- precision form --

def test_fp32_estimate_form(orc, plain):
    """FP32 estimates and deltas, FP64 accumulators: registers, changed sets
    and iteration counts stay bit-exact; accumulators within the FP32 bound
    (per step, each estimate has relative error <= 2^-22, so with a factor
    two for estimates that exceed the final one, the sum of distances moves
    by at most 2^-20 * reach * steps^2 and the harmonic sum by
    2^-20 * reach * (1 + ln steps))."""
    off, tgt = plain
    n = off.size - 1
    ref = orc.run(off, tgt, 4, 42, keep_changed=True)
    fin = orc.finalize(4, ref.regs, ref.sumd, ref.harm)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=42, n=n, fp32=True)
    t = 0
    while True:
        k = hb.step()
        ch, _ = hb.frontier()
        assert np.array_equal(ch.cpu().numpy(), ref.changed_hist[t])
        t += 1
        if k == 0:
            break
    assert t == ref.steps
    assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
    s, h = (x.cpu().numpy() for x in hb.accumulators())
    T = ref.steps
    reach = fin["reachable"]
    bound_s = 2.0 ** -20 * reach * T * T + 1e-12
    bound_h = 2.0 ** -20 * reach * (1 + math.log(T)) + 1e-12
    assert np.all(np.abs(s - ref.sumd) <= bound_s)
    assert np.all(np.abs(h - ref.harm) <= bound_h)
    cen = {k: v.cpu().numpy() for k, v in hb.centralities().items()}
    rel = np.abs(cen["reachable"] - reach) / reach
    assert rel.max() < 2e-7
    hb.close()


# -------------------------------------------------------------- autotuner --

@pytest.mark.parametrize("b", [4, 6, 9])
@pytest.mark.parametrize("relabel", [True, False])
def test_every_class_sizing_gives_the_same_result(orc, b, relabel):
    """The autotuner's choice changes only how lanes are grouped, never the
    result: every candidate class sizing, and the tuned one, match the
    oracle."""
    off, tgt = _degree_boundary_graph(b, seed=11)
    ref = orc.run(off, tgt, b, 3)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=b, seed=3, n=off.size - 1, relabel=relabel)
    for aps in (1, 2, 4, 8, 16, 32, 64, 128, None):
        if aps is None:
            assert hb.tune() in (1, 2, 4, 8, 16, 32, 64, 128)
        else:
            hb.set_class_sizing(aps)
        assert hb.run() == ref.steps
        assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
        s, h = hb.accumulators(device="cpu")
        close(s.numpy(), ref.sumd)
        close(h.numpy(), ref.harm)
        hb.reset(3)
    with pytest.raises(hbl.HBError):
        hb.set_class_sizing(3)
    hb.close()
    # the sizing given at creation (hb_options.arcs_per_slot) is the same
    for aps in (1, 128):
        hb = hbl.HyperBall(*to_dev(off, tgt), log2m=b, seed=3, n=off.size - 1, relabel=relabel, arcs_per_slot=aps)
        assert hb.run() == ref.steps
        assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
        hb.close()
    with pytest.raises(hbl.HBError) as e:
        hbl.HyperBall(*to_dev(off, tgt), log2m=b, seed=3, n=off.size - 1, arcs_per_slot=3)
    assert e.value.status == hbl.HB_ERR_INVALID


def test_pinned_host_outputs(orc, plain):
    """Outputs in pinned host memory (as the end-to-end path delivers them)
    equal the device outputs and the oracle, for the centralities,
    accumulators, registers, frontier and a runs handle's statistics."""
    off, tgt = plain
    n = off.size - 1
    ref = orc.run(off, tgt, 4, 42)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=4, seed=42, n=n)
    hb.run()

    def pinned(shape, dtype):
        return torch.full(shape if isinstance(shape, tuple) else (shape,), 7, dtype=dtype).pin_memory()

    cen = {k: pinned(n, torch.float64) for k in ("closeness", "harmonic", "lin", "reachable")}
    hbl.hb_get_centralities(hb._h, cen["closeness"], cen["harmonic"], cen["lin"], cen["reachable"])
    dev = hb.centralities()
    for k in cen:
        assert torch.equal(cen[k], dev[k].cpu()), k
    s, h = pinned(n, torch.float64), pinned(n, torch.float64)
    hbl.hb_get_accumulators(hb._h, s, h)
    close(s.numpy(), ref.sumd)
    close(h.numpy(), ref.harm)
    regs = pinned((n, 16), torch.uint8)
    hbl.hb_get_registers(hb._h, regs)
    assert np.array_equal(regs.numpy(), ref.regs)
    ch, mk = pinned(n, torch.uint8), pinned(n, torch.uint8)
    hbl.hb_get_frontier(hb._h, ch, mk)
    d_ch, d_mk = hb.frontier()
    assert torch.equal(ch, d_ch.cpu()) and torch.equal(mk, d_mk.cpu())
    hb.close()
    runs = hbl.HyperBall.runs(*to_dev(off, tgt), 4, [1, 2, 3, 4], n=n)
    runs.run()
    mean, sd = pinned(n, torch.float64), pinned(n, torch.float64)
    hbl._check(hbl.load().hb_get_run_stats(runs._h, 1, hbl._ptr(mean), hbl._ptr(sd)))
    d_mean, d_sd = runs.run_stats("harmonic")
    assert torch.equal(mean, d_mean.cpu()) and torch.equal(sd, d_sd.cpu())
    runs.close()


def test_centralities_to_host_in_chunks_equal_device():
    """More nodes than one staging chunk (2^24): centralities delivered to
    host memory (pinned and pageable, chunk by chunk, copies overlapping the
    next chunk's computation) equal those delivered to device memory bit for
    bit, in the caller's node order, also with an output left out."""
    n = (1 << 24) * 2 + 12345          # two full chunks and a ragged third
    g = graphs.rmat_graph(scale=26, edge_factor=1, seed=3, n=n, device="cuda")
    hb = hbl.HyperBall(g.offsets, g.targets, log2m=4, seed=8, n=g.n)
    hb.run()
    dev = hb.centralities()
    pinned = {k: torch.empty(g.n, dtype=torch.float64).pin_memory() for k in dev}
    pageable = {k: torch.empty(g.n, dtype=torch.float64) for k in dev}
    for out in (pinned, pageable):
        hbl.hb_get_centralities(hb._h, out["closeness"], out["harmonic"], out["lin"], out["reachable"])
        for k in dev:
            assert torch.equal(out[k], dev[k].cpu()), k
    part = torch.full((g.n,), -1.0, dtype=torch.float64)
    hbl.hb_get_centralities(hb._h, None, part, None, None)
    assert torch.equal(part, dev["harmonic"].cpu())
    hb.close()
