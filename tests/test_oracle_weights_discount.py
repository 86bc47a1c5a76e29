"""Pins for the oracle's node weights (Sec. 6, replicas) and discount
functions (Sec. 7), against brute force that shares no code with it.

* After t iterations with weights w, every counter equals the HyperLogLog
  counter of the replicas of the nodes in the breadth-first ball of radius t
  (the weighted ball of Sec. 6, by its definition).
* Under a seed where every replica has its own register, a counter holding
  K replicas is estimated by linear counting as p ln(p/(p-K)), so the
  accumulators are closed-form sums over exact weighted layer sizes, for any
  discount table.
* Discounts that reduce to the Sec. 5 accumulators (f(d) = d, f(d) = 1/d),
  and the constant discount, which telescopes to the growth of the counter.
* Weighted reachable-set estimates stay within the counter's error bound of
  the exact weighted sums."""
import math

import numpy as np
import pytest

from paper_1308_2144_gb300 import graphs
from tests import brute
from tests.test_oracle_hyperball import SMALL


def _weights(n, seed, lo=0, hi=4):
    return np.random.default_rng(seed).integers(lo, hi + 1, size=n).astype(np.int64)


def _walk(orc, off, tgt, b, seed, weights, table=None, max_steps=10_000):
    n = off.size - 1
    c = orc.init_weighted(n, b, seed, weights)
    sumd, harm, disc = np.zeros(n), np.zeros(n), np.zeros(n)
    hist, changed = [c], []
    for t in range(max_steps):
        f = orc.discount(table, t + 1) if table is not None else 0.0
        nxt, ch, k = orc.step(off, tgt, b, t, hist[-1], sumd, harm, disc, f)
        changed.append(ch)
        hist.append(nxt)
        if k == 0:
            break
    return hist, changed, sumd, harm, disc


@pytest.mark.parametrize("name", ["path", "cycle", "star_in", "dag", "loops_dups", "zipf", "rmat"])
@pytest.mark.parametrize("b,seed", [(4, 42), (7, 5)])
def test_weighted_counters_equal_hll_of_replica_balls(orc, name, b, seed):
    off, tgt = SMALL[name]
    n = off.size - 1
    w = _weights(n, seed)
    starts = brute.replica_starts(w)
    adj = brute.adjacency(off, tgt)
    dists = [brute.bfs_dist(adj, x) for x in range(n)]
    hist, changed, _, _, _ = _walk(orc, off, tgt, b, seed, w)
    for t, c in enumerate(hist):
        for v in range(n):
            items = brute.replica_items(brute.ball(dists[v], t), w, starts)
            assert np.array_equal(c[v], brute.hll_of_items(items, b, seed)), (name, t, v)
    # the loop ends at the first iteration that leaves every weighted ball unchanged
    T = 0
    while any(not np.array_equal(
            brute.hll_of_items(brute.replica_items(brute.ball(dists[v], T + 1), w, starts), b, seed),
            brute.hll_of_items(brute.replica_items(brute.ball(dists[v], T), w, starts), b, seed))
            for v in range(n)):
        T += 1
    assert len(changed) == T + 1


def test_unit_weights_give_the_unweighted_counters(orc):
    off, tgt = SMALL["zipf"]
    n = off.size - 1
    for b, seed in ((4, 1), (9, 77)):
        assert np.array_equal(orc.init_weighted(n, b, seed, np.ones(n, dtype=np.int64)),
                              orc.init(n, b, seed))
        ref = orc.run(off, tgt, b, seed)
        res = orc.run(off, tgt, b, seed, weights=np.ones(n, dtype=np.int64))
        assert res.steps == ref.steps and np.array_equal(res.regs, ref.regs)
        assert np.array_equal(res.sumd, ref.sumd) and np.array_equal(res.harm, ref.harm)


def _distinct_items_seed(total, b, start):
    seed = start
    while True:
        idx = {brute.split_bits(brute.node_hash(seed, x), b)[0] for x in range(total)}
        if len(idx) == total:
            return seed
        seed += 1


TABLES = {
    "log": [1.0 / math.log(d + 1) for d in range(1, 40)],      # Sec. 7's logarithmic discount
    "quadratic": [1.0 / (d * d) for d in range(1, 40)],        # Sec. 7's quadratic discount
    "short": [1.0, 0.5, 0.25],                                  # longer distances count 0
}


@pytest.mark.parametrize("table", sorted(TABLES))
@pytest.mark.parametrize("n,b,gseed", [(10, 8, 1), (14, 9, 2)])
def test_weighted_discounted_accumulators_closed_form(orc, table, n, b, gseed):
    """Every replica in its own register and at most p/2 of them: a ball
    whose nodes weigh K in all is estimated as p ln(p/(p-K)), and every
    accumulator is the discounted sum of exact weighted layer sizes:
    sum_y w(y) f(d(y,x)) in its estimated form (Sec. 7)."""
    p = 1 << b
    rng = np.random.default_rng(gseed)
    edges = [(int(u), int(v)) for u, v in rng.integers(0, n, size=(2 * n, 2)) if u != v]
    off, tgt = graphs.from_edges(n, edges).numpy()
    w = _weights(n, gseed, 0, 6)
    total = int(w.sum())
    assert total <= p // 2
    seed = _distinct_items_seed(total, b, 1000 * gseed)
    f = TABLES[table]
    res = orc.run(off, tgt, b, seed, weights=w, discount=f)
    adj = brute.adjacency(off, tgt)

    def fd(d):
        return f[d - 1] if 1 <= d <= len(f) else 0.0

    for v in range(n):
        dist = brute.bfs_dist(adj, v)
        R = max(dist.values())
        K = [sum(int(w[y]) for y, d in dist.items() if d <= r) for r in range(R + 2)]
        E = [brute.linear_counting(p, k) for k in K]
        layers = range(len(E) - 1)
        assert res.sumd[v] == pytest.approx(sum((t + 1) * (E[t + 1] - E[t]) for t in layers),
                                            rel=1e-12, abs=1e-12)
        assert res.harm[v] == pytest.approx(sum((E[t + 1] - E[t]) / (t + 1) for t in layers),
                                            rel=1e-12, abs=1e-12)
        assert res.disc[v] == pytest.approx(sum(fd(t + 1) * (E[t + 1] - E[t]) for t in layers),
                                            rel=1e-12, abs=1e-12)
        fin = orc.finalize(b, res.regs[v:v + 1], res.sumd[v:v + 1], res.harm[v:v + 1])
        assert fin["reachable"][0] == pytest.approx(E[-1], rel=1e-13)


@pytest.mark.parametrize("name", ["zipf", "rmat", "dag"])
def test_discounts_that_reduce_to_the_accumulators(orc, name):
    off, tgt = SMALL[name]
    n = off.size - 1
    w = _weights(n, 3, 1, 5)
    b, seed = 6, 9
    ref = orc.run(off, tgt, b, seed, weights=w)
    L = ref.steps + 2
    # f(d) = d is the sum of distances, term by term
    lin = orc.run(off, tgt, b, seed, weights=w, discount=[float(d) for d in range(1, L)])
    assert np.array_equal(lin.disc, ref.sumd)
    # f(d) = 1/d is the harmonic sum (one more rounding: f is rounded first)
    rec = orc.run(off, tgt, b, seed, weights=w, discount=[1.0 / d for d in range(1, L)])
    np.testing.assert_allclose(rec.disc, ref.harm, rtol=1e-12, atol=1e-12)
    # f = 1 telescopes: the growth of each counter's estimate
    one = orc.run(off, tgt, b, seed, weights=w, discount=[1.0] * L)
    c0 = orc.init_weighted(n, b, seed, w)
    growth = np.array([orc.size(ref.regs[v], b) - orc.size(c0[v], b) for v in range(n)])
    np.testing.assert_allclose(one.disc, growth, rtol=1e-9, atol=1e-9)
    # distances beyond the table contribute nothing
    short = orc.run(off, tgt, b, seed, weights=w, discount=[1.0, 1.0])
    hist, _, _, _, _ = _walk(orc, off, tgt, b, seed, w)
    two = np.array([orc.size(hist[min(2, len(hist) - 1)][v], b) - orc.size(c0[v], b)
                    for v in range(n)])
    np.testing.assert_allclose(short.disc, two, rtol=1e-9, atol=1e-9)
    # none of this changes counters or iteration counts
    for r in (lin, rec, one, short):
        assert r.steps == ref.steps and np.array_equal(r.regs, ref.regs)


def test_weighted_reach_within_counter_error(orc):
    """Across hash seeds, each node's weighted reachable-set estimate has RMS
    relative error within the counter bound 1.06/sqrt(p) of the exact
    sum of the weights it coreaches (Sec. 4.1, Sec. 6), without bias."""
    g = graphs.plain_graph(n=1500, seed=7)
    off, tgt = g.numpy()
    n = off.size - 1
    w = _weights(n, 11, 1, 8)
    adj = brute.adjacency(off, tgt)
    exact = np.array([sum(int(w[y]) for y in brute.bfs_dist(adj, v)) for v in range(n)], float)
    big = exact >= 400
    assert big.sum() > 300
    # nodes of the giant component share one coreachable set, so a run
    # gives one draw of their error: K runs must pin the RMS by themselves
    b, K = 7, 96
    bound = 1.06 / math.sqrt(1 << b)
    errs = []
    for k in range(K):
        res = orc.run(off, tgt, b, 300 + k, weights=w)
        reach = orc.finalize(b, res.regs, res.sumd, res.harm)["reachable"]
        errs.append(reach[big] / exact[big] - 1)
    e = np.array(errs)
    assert np.median(np.sqrt((e ** 2).mean(axis=0))) <= 1.15 * bound
    assert abs(np.median(e.mean(axis=0))) <= 3 * bound / math.sqrt(K)


# ------------------------------------------------ neighbourhood function --

@pytest.mark.parametrize("name", ["path", "dag", "star_in", "loops_dups", "zipf"])
def test_neighbourhood_function_is_sum_of_ball_counters(orc, name):
    """N(t) is the sum over nodes of size() of the HyperLogLog counter of the
    BFS ball of radius t, at every t of the run."""
    off, tgt = SMALL[name]
    n = off.size - 1
    b, seed = 6, 21
    nf = orc.neighbourhood_function(off, tgt, b, seed)
    adj = brute.adjacency(off, tgt)
    dists = [brute.bfs_dist(adj, x) for x in range(n)]
    for t, N in enumerate(nf):
        balls = np.array([brute.hll_of_set(brute.ball(dists[v], t), b, seed) for v in range(n)])
        expect = sum(orc.size(balls[v], b) for v in range(n))
        assert N == pytest.approx(expect, rel=1e-13)


def test_neighbourhood_function_closed_form(orc):
    """Every node in its own register: N(t) is the sum over nodes of
    p ln(p/(p - |B(v,t)|)) with exact ball sizes, non-decreasing in t."""
    n, b = 20, 9
    p = 1 << b
    rng = np.random.default_rng(4)
    edges = [(int(u), int(v)) for u, v in rng.integers(0, n, size=(2 * n, 2)) if u != v]
    off, tgt = graphs.from_edges(n, edges).numpy()
    seed = _distinct_items_seed(n, b, 300)
    nf = orc.neighbourhood_function(off, tgt, b, seed)
    adj = brute.adjacency(off, tgt)
    dists = [brute.bfs_dist(adj, x) for x in range(n)]
    for t, N in enumerate(nf):
        expect = sum(brute.linear_counting(p, len(brute.ball(dists[v], t))) for v in range(n))
        assert N == pytest.approx(expect, rel=1e-12)
    assert np.all(np.diff(nf) >= 0)


def test_neighbourhood_function_accuracy(orc):
    """Against the exact neighbourhood function (the sum of BFS ball
    sizes): within the counter's error bound at every t (Sec. 4.1)."""
    off, tgt = graphs.plain_graph(n=2000, seed=5).numpy()
    n = off.size - 1
    adj = brute.adjacency(off, tgt)
    dists = [brute.bfs_dist(adj, x) for x in range(n)]
    b = 8
    nf = orc.neighbourhood_function(off, tgt, b, 77)
    for t in range(1, len(nf)):
        exact = sum(sum(1 for d in dv.values() if d <= t) for dv in dists)
        # a sum of per-node estimates: the relative error stays below one counter's
        assert abs(nf[t] / exact - 1) < 3 * 1.06 / math.sqrt(1 << b), t
