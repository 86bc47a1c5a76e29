"""Pins for the oracle's HyperBall loop (Sec. 4.2, Algorithm 2) and its
accumulators (Sec. 5), against brute force that shares no code with it:
after t iterations every counter must equal the HyperLogLog counter built
directly from the breadth-first ball of radius t."""
import math

import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from tests import brute


def _edges_graph(n, edges):
    return graphs.from_edges(n, edges).numpy()


def _small_graphs():
    rng = np.random.default_rng(5)
    G = {}
    G["path"] = _edges_graph(12, [(i, i + 1) for i in range(11)])
    G["cycle"] = _edges_graph(9, [(i, (i + 1) % 9) for i in range(9)])
    G["star_out"] = _edges_graph(11, [(0, i) for i in range(1, 11)])
    G["star_in"] = _edges_graph(11, [(i, 0) for i in range(1, 11)])
    G["complete"] = _edges_graph(7, [(i, j) for i in range(7) for j in range(7) if i != j])
    dag = [(i, j) for i in range(30) for j in range(i + 1, 30) if rng.random() < 0.12]
    G["dag"] = _edges_graph(30, dag)
    G["empty"] = _edges_graph(0, [])
    G["isolated"] = _edges_graph(5, [])
    G["loops_dups"] = _edges_graph(6, [(0, 0), (0, 1), (0, 1), (1, 2), (2, 2), (2, 0), (3, 4),
                                       (3, 4), (4, 4), (5, 3)])
    G["zipf"] = graphs.plain_graph(n=300, seed=9).numpy()
    G["rmat"] = graphs.rmat_graph(scale=8, edge_factor=4, seed=13).numpy()
    return G


SMALL = _small_graphs()


def _walk(orc, off, tgt, b, seed, max_steps=10_000):
    """Iterate the oracle step by step; return the list of counters c_0..c_T,
    the changed sets and the accumulators."""
    n = off.size - 1
    c = orc.init(n, b, seed)
    sumd = np.zeros(n)
    harm = np.zeros(n)
    hist, changed = [c], []
    for t in range(max_steps):
        nxt, ch, k = orc.step(off, tgt, b, t, hist[-1], sumd, harm)
        changed.append(ch)
        hist.append(nxt)
        if k == 0:
            break
    return hist, changed, sumd, harm


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("b,seed", [(4, 42), (7, 5)])
def test_counters_equal_hll_of_balls(orc, name, b, seed):
    off, tgt = SMALL[name]
    n = off.size - 1
    adj = brute.adjacency(off, tgt)
    dists = [brute.bfs_dist(adj, x) for x in range(n)]
    hist, changed, _, _ = _walk(orc, off, tgt, b, seed)
    steps = len(changed)
    for t, c in enumerate(hist):
        for v in range(n):
            expect = brute.hll_of_set(brute.ball(dists[v], t), b, seed)
            assert np.array_equal(c[v], expect), (name, t, v)
    # changed sets are exactly the counters that differ between iterations
    for t, ch in enumerate(changed):
        assert np.array_equal(ch.astype(bool), (hist[t + 1] != hist[t]).any(axis=1))
    # first iteration that leaves every ball-HLL unchanged ends the loop
    T = 0
    while any(not np.array_equal(brute.hll_of_set(brute.ball(dists[v], T + 1), b, seed),
                                 brute.hll_of_set(brute.ball(dists[v], T), b, seed))
              for v in range(n)):
        T += 1
    assert steps == T + 1
    ecc = max((max(d.values()) for d in dists), default=0)
    assert steps <= ecc + 1
    # monotone registers, idempotent fixpoint
    for t in range(len(hist) - 1):
        assert (hist[t + 1] >= hist[t]).all()
    s2, h2 = np.zeros(n), np.zeros(n)
    again, ch, k = orc.step(off, tgt, b, steps, hist[-1], s2, h2)
    assert k == 0 and np.array_equal(again, hist[-1]) and not s2.any() and not h2.any()


@pytest.mark.parametrize("name", ["zipf", "rmat", "dag", "cycle", "loops_dups"])
def test_must_check_is_sound(orc, name):
    # Only nodes with a changed successor can change in the next iteration.
    off, tgt = SMALL[name]
    _, changed, _, _ = _walk(orc, off, tgt, 5, 77)
    for t in range(len(changed) - 1):
        must = orc.must_check(off, tgt, changed[t])
        assert not (changed[t + 1].astype(bool) & ~must.astype(bool)).any()
    if len(changed) > 2:
        # and the rule really skips nodes on these graphs
        assert any(orc.must_check(off, tgt, c).sum() < off.size - 1 for c in changed[1:])


def test_must_check_definition(orc):
    off, tgt = SMALL["zipf"]
    n = off.size - 1
    rng = np.random.default_rng(1)
    ch = (rng.random(n) < 0.05).astype(np.uint8)
    must = orc.must_check(off, tgt, ch)
    adj = brute.adjacency(off, tgt)
    assert [int(any(ch[w] for w in adj[v])) for v in range(n)] == must.tolist()


def _distinct_index_seed(n, b, start=1):
    seed = start
    while True:
        idx = {brute.split_bits(brute.node_hash(seed, v), b)[0] for v in range(n)}
        if len(idx) == n:
            return seed
        seed += 1


@pytest.mark.parametrize("n,b,gseed", [(8, 7, 1), (40, 12, 2), (60, 12, 3)])
def test_accumulators_closed_form(orc, n, b, gseed):
    """With a seed under which all n nodes use distinct registers, a ball of
    k nodes has exactly k nonzero registers and (k <= p/2) is estimated by
    linear counting as p ln(p/(p-k)).  The Sec. 5 accumulators are then
    sums over exact BFS layer sizes."""
    p = 1 << b
    rng = np.random.default_rng(gseed)
    edges = [(int(u), int(v)) for u, v in rng.integers(0, n, size=(3 * n, 2)) if u != v]
    off, tgt = _edges_graph(n, edges)
    seed = _distinct_index_seed(n, b, start=100 * gseed)
    res = orc.run(off, tgt, b, seed)
    adj = brute.adjacency(off, tgt)
    for v in range(n):
        d = brute.bfs_dist(adj, v)
        sizes = [sum(1 for x in d.values() if x <= r) for r in range(max(d.values()) + 2)]
        E = [brute.linear_counting(p, k) for k in sizes]
        sumd = sum((t + 1) * (E[t + 1] - E[t]) for t in range(len(E) - 1))
        harm = sum((E[t + 1] - E[t]) / (t + 1) for t in range(len(E) - 1))
        assert res.sumd[v] == pytest.approx(sumd, rel=1e-12, abs=1e-12)
        assert res.harm[v] == pytest.approx(harm, rel=1e-12, abs=1e-12)
        fin = orc.finalize(b, res.regs[v:v + 1], res.sumd[v:v + 1], res.harm[v:v + 1])
        assert fin["reachable"][0] == pytest.approx(brute.linear_counting(p, len(d)), rel=1e-13)


def test_finalize_special_cases(orc):
    b, p = 6, 64
    off, tgt = _edges_graph(4, [(0, 1), (1, 2)])    # node 3 isolated, node 2 a sink
    res = orc.run(off, tgt, b, 42)
    fin = orc.finalize(b, res.regs, res.sumd, res.harm)
    for v in (2, 3):                                # nothing else reached: sumd = 0
        assert res.sumd[v] == 0.0 and res.harm[v] == 0.0
        assert fin["closeness"][v] == 0.0 and fin["lin"][v] == 1.0
        assert fin["harmonic"][v] == 0.0
        assert fin["reachable"][v] == pytest.approx(p * math.log(p / (p - 1)))
    for v in (0, 1):
        assert fin["closeness"][v] == 1.0 / res.sumd[v]
        assert fin["lin"][v] == fin["reachable"][v] ** 2 / res.sumd[v]
        assert fin["harmonic"][v] == res.harm[v]


@pytest.mark.parametrize("name", ["zipf", "path", "dag", "star_in"])
def test_run_matches_stepwise(orc, name):
    off, tgt = SMALL[name]
    hist, changed, sumd, harm = _walk(orc, off, tgt, 6, 3)
    res = orc.run(off, tgt, 6, 3, keep_changed=True)
    assert res.converged and res.steps == len(changed)
    assert np.array_equal(res.regs, hist[-1])
    assert np.array_equal(res.sumd, sumd) and np.array_equal(res.harm, harm)
    assert np.array_equal(res.changed_hist, np.stack(changed))
    if len(changed) > 2:
        short = orc.run(off, tgt, 6, 3, max_steps=2)
        assert not short.converged and short.steps == 2
        assert np.array_equal(short.regs, hist[2])


def test_thread_count_does_not_change_results(orc):
    off, tgt = graphs.plain_graph(n=3000, seed=4).numpy()
    outs = []
    for k in (1, 3, 8):
        orc.set_threads(k)
        outs.append(orc.run(off, tgt, 5, 11))
    orc.set_threads(0)
    for r in outs[1:]:
        assert r.steps == outs[0].steps
        assert np.array_equal(r.regs, outs[0].regs)
        assert np.array_equal(r.sumd, outs[0].sumd) and np.array_equal(r.harm, outs[0].harm)


def _exact_by_brute_force(off, tgt, sources):
    """Sum of distances, sum of reciprocal distances over y != x, number of
    nodes at finite distance (x included) and eccentricity, from the
    brute-force breadth-first distances along the scanned graph's arcs
    (Sec. 3's definitions of closeness, harmonic and Lin centrality)."""
    adj = brute.adjacency(off, tgt)
    out = {"sumd": [], "harm": [], "reach": [], "ecc": []}
    for x in sources:
        d = brute.bfs_dist(adj, int(x))
        out["sumd"].append(float(sum(d.values())))
        out["harm"].append(sum(1.0 / k for k in d.values() if k > 0))
        out["reach"].append(float(len(d)))
        out["ecc"].append(max(d.values()))
    return {k: np.array(v) for k, v in out.items()}


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("with_sources", [False, True])
def test_exact_centralities_equal_brute_force_bfs(orc, name, with_sources):
    """The exact-BFS checker behind the accuracy pins, against breadth-first
    distances computed independently, on every small graph: all nodes, and
    a shuffled subset of sources with a repeat."""
    off, tgt = SMALL[name]
    n = off.size - 1
    if with_sources:
        rng = np.random.default_rng(n + 1)
        src = rng.permutation(n)[: max(1, (2 * n) // 3)] if n else np.zeros(0, dtype=np.int64)
        if n:
            src = np.concatenate([src, src[:1]])
    else:
        src = np.arange(n)
    got = orc.exact_centralities(off, tgt, src if with_sources else None)
    exp = _exact_by_brute_force(off, tgt, src)
    assert np.array_equal(got["reach"], exp["reach"]), name
    assert np.array_equal(got["ecc"], exp["ecc"]), name
    assert np.array_equal(got["sumd"], exp["sumd"]), name
    np.testing.assert_allclose(got["harm"], exp["harm"], rtol=1e-12, atol=0)
