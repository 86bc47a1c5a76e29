"""Pins for the oracle's packed registers (Sec. 4.1, register width: a
register needs only about log2 log2 n bits).  Six bits per register, register
j at bits 6j .. 6j+5 of the counter's bit string.

What pins it: (a) the packed form holds every register value the method can
produce (rho+ <= 64 - b <= 60 < 64), so unpacking a packed counter gives it
back, for every log2m and every position, and a value that does not fit is
refused; (b) the bit layout against the counter read as one little-endian
integer; (c) the packed iteration, step by step, equals the HyperLogLog built
directly from each node's breadth-first ball (brute force, no oracle code),
and the unpacked oracle run bit for bit."""
import numpy as np
import pytest

from tests import brute
from tests.test_oracle_hyperball import SMALL


@pytest.mark.parametrize("b", list(range(4, 13)))
def test_round_trip_every_position_and_value(orc, b):
    p = 1 << b
    rng = np.random.default_rng(b)
    # every value 0 .. 64-b at every position, and random counters
    vals = np.arange(0, 64 - b + 1, dtype=np.uint8)
    rows = np.zeros((len(vals), p), dtype=np.uint8)
    for k, v in enumerate(vals):
        rows[k] = np.roll(np.full(p, v, dtype=np.uint8) * (np.arange(p) % 3 == k % 3), k)
    rows = np.vstack([rows, rng.integers(0, 64 - b + 1, size=(50, p)).astype(np.uint8),
                      np.full((1, p), 63, dtype=np.uint8)])
    packed = orc.pack6(rows, b)
    assert packed.shape == (rows.shape[0], 3 * p // 4)
    assert np.array_equal(orc.unpack6(packed, b), rows)


def test_a_register_that_does_not_fit_is_refused(orc):
    M = np.zeros((1, 16), dtype=np.uint8)
    M[0, 7] = 64
    with pytest.raises(ValueError):
        orc.pack6(M, 4)


@pytest.mark.parametrize("b", [4, 6, 9])
def test_bit_layout_is_the_little_endian_bit_string(orc, b):
    p = 1 << b
    rng = np.random.default_rng(100 + b)
    M = rng.integers(0, 61, size=(8, p)).astype(np.uint8)
    packed = orc.pack6(M, b)
    for row, pk in zip(M, packed):
        as_int = int.from_bytes(bytes(pk), "little")
        for j in range(p):
            assert (as_int >> (6 * j)) & 63 == row[j]
        assert as_int >> (6 * p) == 0


def _packed_walk(orc, off, tgt, b, seed):
    n = off.size - 1
    c = orc.pack6(orc.init(n, b, seed), b)
    sumd, harm = np.zeros(n), np.zeros(n)
    hist = [c]
    for t in range(10_000):
        nxt, ch, k = orc.step_packed(off, tgt, b, t, hist[-1], sumd, harm)
        hist.append(nxt)
        if k == 0:
            break
    return hist, sumd, harm


@pytest.mark.parametrize("name", ["path", "cycle", "dag", "loops_dups", "zipf", "rmat"])
@pytest.mark.parametrize("b,seed", [(4, 42), (6, 5)])
def test_packed_counters_equal_hll_of_balls(orc, name, b, seed):
    off, tgt = SMALL[name]
    n = off.size - 1
    adj = brute.adjacency(off, tgt)
    dists = [brute.bfs_dist(adj, x) for x in range(n)]
    hist, sumd, harm = _packed_walk(orc, off, tgt, b, seed)
    for t, c in enumerate(hist):
        regs = orc.unpack6(c, b) if n else np.zeros((0, 1 << b), dtype=np.uint8)
        for v in range(n):
            assert np.array_equal(regs[v], brute.hll_of_set(brute.ball(dists[v], t), b, seed)), (name, t, v)
    ref = orc.run(off, tgt, b, seed)
    assert len(hist) - 1 == ref.steps
    if n:
        assert np.array_equal(orc.unpack6(hist[-1], b), ref.regs)
    np.testing.assert_array_equal(sumd, ref.sumd)
    np.testing.assert_array_equal(harm, ref.harm)
