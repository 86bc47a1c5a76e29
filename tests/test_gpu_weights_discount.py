"""Node weights (Sec. 6) and discount functions (Sec. 7) on the GPU against
the oracle, through the C ABI: registers, changed sets and iteration counts
bit-exact at every iteration; the three accumulators (sum of distances,
harmonic, discounted) and the centralities within 1e-9 relative."""
import math

import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl
from tests.test_gpu_parity import close, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


LOG_DISCOUNT = [1.0 / math.log(d + 1) for d in range(1, 65)]   # Sec. 7's logarithmic discount


def weights_of(n, seed, hi=6, zeros=True):
    return np.random.default_rng(seed).integers(0 if zeros else 1, hi + 1, size=n).astype(np.int64)


def walk(orc, off, tgt, b, seed, w, table, fp32=False, **opts):
    """GPU and oracle side by side, one iteration at a time."""
    n = off.size - 1
    d_off, d_tgt = to_dev(off, tgt)
    hb = hbl.HyperBall(d_off, d_tgt, log2m=b, seed=seed, n=n, fp32=fp32, **opts)
    if w is not None:
        hb.set_weights(torch.from_numpy(w).cuda())
    if table is not None:
        hb.set_discount(table)
    c = orc.init_weighted(n, b, seed, w) if w is not None else orc.init(n, b, seed)
    sumd, harm, disc = np.zeros(n), np.zeros(n), np.zeros(n)
    assert np.array_equal(hb.registers().cpu().numpy(), c)
    t = 0
    while True:
        f = orc.discount(table, t + 1) if table is not None else 0.0
        nxt, ch, k = orc.step(off, tgt, b, t, c, sumd, harm, disc, f)
        assert hb.step() == k, t
        assert np.array_equal(hb.registers().cpu().numpy(), nxt), t
        assert np.array_equal(hb.frontier()[0].cpu().numpy(), ch), t
        if not fp32:
            gs, gh = hb.accumulators()
            close(gs.cpu().numpy(), sumd)
            close(gh.cpu().numpy(), harm)
            if table is not None:
                close(hb.discounted().cpu().numpy(), disc)
        c = nxt
        t += 1
        if k == 0:
            break
    out = dict(steps=t, regs=c, sumd=sumd, harm=harm, disc=disc, hb=hb)
    return out


@pytest.mark.parametrize("frontier,pull_gather,relabel", [("auto", False, True), ("auto", True, True),
                                                          ("pull", False, True), ("off", False, True),
                                                          ("auto", False, False)])
def test_weighted_discounted_plain_workload(orc, frontier, pull_gather, relabel):
    off, tgt = graphs.plain_graph(n=10_000, seed=1).numpy()
    w = weights_of(off.size - 1, 5)
    r = walk(orc, off, tgt, 4, 42, w, LOG_DISCOUNT, frontier=frontier, pull_gather=pull_gather,
             relabel=relabel)
    fin = orc.finalize(4, r["regs"], r["sumd"], r["harm"])
    cen = {k: v.cpu().numpy() for k, v in r["hb"].centralities().items()}
    for key in ("closeness", "harmonic", "lin", "reachable"):
        close(cen[key], fin[key])
    r["hb"].close()


@pytest.mark.parametrize("b", [5, 6, 9, 12])
def test_weighted_split_nodes(orc, b):
    """R-MAT hubs above the split threshold: partial counters of split nodes
    and the pushed union carry the weighted counters."""
    off, tgt = graphs.rmat_graph(scale=13, edge_factor=16, seed=40 + b).numpy()
    w = weights_of(off.size - 1, b, hi=9, zeros=False)
    r = walk(orc, off, tgt, b, 900 + b, w, [1.0 / (d * d) for d in range(1, 40)])
    r["hb"].close()


def test_short_table_and_fp32_form(orc):
    off, tgt = graphs.rmat_graph(scale=12, edge_factor=8, seed=3).numpy()
    n = off.size - 1
    w = weights_of(n, 8)
    # distances beyond the table contribute nothing
    r = walk(orc, off, tgt, 6, 17, w, [1.0, 0.5])
    r["hb"].close()
    # FP32 estimates: counters, frontier and counts stay exact; each estimate
    # is within 2^-22 of the FP64 one (three roundings), so each layer's
    # delta within 2^-21 reach and the discounted sum within
    # 2^-21 reach T max|f| (written with 2^-20 for slack, as for sumd)
    r = walk(orc, off, tgt, 6, 17, w, LOG_DISCOUNT, fp32=True)
    ref = orc.run(off, tgt, 6, 17, weights=w, discount=LOG_DISCOUNT)
    reach = orc.finalize(6, ref.regs, ref.sumd, ref.harm)["reachable"]
    got = r["hb"].discounted().cpu().numpy()
    bound = 2.0 ** -20 * reach * ref.steps * max(LOG_DISCOUNT) + 1e-12
    assert np.all(np.abs(got - ref.disc) <= bound)
    r["hb"].close()


def test_unit_weights_and_reset(orc):
    off, tgt = graphs.plain_graph(n=3000, seed=2).numpy()
    n = off.size - 1
    d_off, d_tgt = to_dev(off, tgt)
    hb = hbl.HyperBall(d_off, d_tgt, log2m=5, seed=9, n=n)
    plain_steps = hb.run()
    plain_regs = hb.registers().cpu().numpy()
    hb.set_weights(np.ones(n, dtype=np.int64))          # host weights, unit: the same run
    assert hb.run() == plain_steps
    assert np.array_equal(hb.registers().cpu().numpy(), plain_regs)
    w = weights_of(n, 4)
    hb.set_weights(w)
    hb.set_discount(LOG_DISCOUNT)
    steps = hb.run()
    ref = orc.run(off, tgt, 5, 9, weights=w, discount=LOG_DISCOUNT)
    assert steps == ref.steps and np.array_equal(hb.registers().cpu().numpy(), ref.regs)
    close(hb.discounted().cpu().numpy(), ref.disc)
    # a reset keeps weights and discount, with the new seed
    hb.reset(31)
    hb.run()
    ref = orc.run(off, tgt, 5, 31, weights=w, discount=LOG_DISCOUNT)
    assert np.array_equal(hb.registers().cpu().numpy(), ref.regs)
    close(hb.discounted().cpu().numpy(), ref.disc)
    # removing them gives back the plain run of that seed
    hb.set_weights(None)
    hb.set_discount(None)
    hb.run()
    assert np.array_equal(hb.registers().cpu().numpy(), orc.run(off, tgt, 5, 31).regs)
    with pytest.raises(hbl.HBError) as e:
        hb.discounted()
    assert e.value.status == hbl.HB_ERR_STATE
    hb.close()


def test_bad_weights_rejected_handle_unchanged(orc):
    off, tgt = graphs.plain_graph(n=2000, seed=6).numpy()
    n = off.size - 1
    d_off, d_tgt = to_dev(off, tgt)
    hb = hbl.HyperBall(d_off, d_tgt, log2m=4, seed=3, n=n)
    hb.step()
    before = hb.registers().cpu().numpy()
    for bad in (-1, 1 << 31):
        w = np.ones(n, dtype=np.int64)
        w[n // 2] = bad
        with pytest.raises(hbl.HBError) as e:
            hb.set_weights(w)
        assert e.value.status == hbl.HB_ERR_INVALID
    assert hb.info()["t"] == 1
    assert np.array_equal(hb.registers().cpu().numpy(), before)
    hb.run()
    assert np.array_equal(hb.registers().cpu().numpy(), orc.run(off, tgt, 4, 3).regs)
    hb.close()


def test_checkpoint_keeps_weights_and_discount(orc, tmp_path):
    off, tgt = graphs.rmat_graph(scale=11, edge_factor=8, seed=12).numpy()
    n = off.size - 1
    w = weights_of(n, 12)
    d_off, d_tgt = to_dev(off, tgt)
    hb = hbl.HyperBall(d_off, d_tgt, log2m=6, seed=5, n=n)
    hb.set_weights(w)
    hb.set_discount(LOG_DISCOUNT)
    hb.step()
    hb.step()
    path = str(tmp_path / "wd.ckpt")
    hb.save(path)
    h2 = hbl.hb_load(path)
    hb.run()
    hbl.hb_run_to_fixpoint(h2)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    hbl.hb_get_discounted(h2, out)
    regs = torch.empty((n, 64), dtype=torch.uint8, device="cuda")
    hbl.hb_get_registers(h2, regs)
    assert torch.equal(regs, hb.registers())
    assert torch.equal(out, hb.discounted())
    ref = orc.run(off, tgt, 6, 5, weights=w, discount=LOG_DISCOUNT)
    assert np.array_equal(regs.cpu().numpy(), ref.regs)
    close(out.cpu().numpy(), ref.disc)
    hbl.hb_destroy(h2)
    hb.close()


# ------------------------------------------------ neighbourhood function --

@pytest.mark.parametrize("b,frontier", [(4, "auto"), (8, "off"), (6, "pull")])
def test_neighbourhood_function(orc, b, frontier):
    """N(t) after every iteration equals the oracle's sum of size() over all
    counters within 1e-9, in the same order of magnitude of terms; the
    device sum has a fixed order, so two runs agree bit for bit."""
    off, tgt = graphs.plain_graph(n=10_000, seed=3).numpy()
    n = off.size - 1
    ref = orc.neighbourhood_function(off, tgt, b, 42)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=b, seed=42, n=n, frontier=frontier, neighbourhood=True)
    hb.run()
    nf = hb.neighbourhood()
    assert nf.size == ref.size
    close(nf, ref)
    hb.reset(42)
    hb.run()
    assert np.array_equal(hb.neighbourhood(), nf)
    hb.close()


def test_neighbourhood_function_weighted_fp32_checkpoint(orc, tmp_path):
    off, tgt = graphs.rmat_graph(scale=12, edge_factor=8, seed=5).numpy()
    n = off.size - 1
    w = weights_of(n, 3)
    ref = orc.neighbourhood_function(off, tgt, 6, 7, weights=w)
    hb = hbl.HyperBall(*to_dev(off, tgt), log2m=6, seed=7, n=n, neighbourhood=True)
    hb.set_weights(w)
    hb.step()
    hb.step()
    path = str(tmp_path / "nf.ckpt")
    hb.save(path)
    hb.run()
    close(hb.neighbourhood(), ref)
    h2 = hbl.hb_load(path)
    hbl.hb_run_to_fixpoint(h2)
    assert np.array_equal(hbl.hb_get_neighbourhood(h2), hb.neighbourhood())
    hbl.hb_destroy(h2)
    hb.close()
    # FP32 estimates: each within 2^-22 relative, so the sum too
    h32 = hbl.HyperBall(*to_dev(off, tgt), log2m=6, seed=7, n=n, fp32=True, neighbourhood=True)
    h32.set_weights(w)
    h32.run()
    got = h32.neighbourhood()
    assert got.size == ref.size and np.all(np.abs(got / ref - 1) < 2.0 ** -21)
    h32.close()
    plain = hbl.HyperBall(*to_dev(off, tgt), log2m=6, seed=7, n=n)
    with pytest.raises(hbl.HBError) as e:
        plain.neighbourhood()
    assert e.value.status == hbl.HB_ERR_STATE
    plain.close()
