"""Pins for the oracle's HyperLogLog counter (Sec. 4.1, Algorithm 1).

The oracle is checked against things other than itself: bit-string
definitions, closed forms, an exact rational sum, the paper's printed
relative standard deviations and the alpha constants of Flajolet et al.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            parts = line.split()
            vals[parts[0]] = parts[1:]
    return vals


PAPER = _golden("paper_values.txt")
FFGH = _golden("ffgh_alpha.txt")


# ------------------------------------------------------------------ hash --

def test_hash_matches_bigint_splitmix(orc):
    rng = np.random.default_rng(7)
    seeds = [0, 1, 42, 2**63, 2**64 - 1] + [int(x) for x in rng.integers(0, 2**63, 20)]
    vs = [0, 1, 2, 10**6, 2**32, 2**40 + 3] + [int(x) for x in rng.integers(0, 2**40, 50)]
    for s in seeds:
        for v in vs:
            assert orc.hash64(s, v) == brute.node_hash(s, v)


def test_hash_is_injective_on_a_range(orc):
    # SplitMix64's output function is a bijection of 64-bit words, so node
    # hashes of distinct ids never collide.
    hs = {orc.hash64(42, v) for v in range(20000)}
    assert len(hs) == 20000


def test_hash_bits_are_balanced(orc):
    hs = np.array([orc.hash64(12345, v) for v in range(20000)], dtype=np.uint64)
    bits = np.unpackbits(hs.view(np.uint8)).reshape(-1, 64).mean(axis=0)
    # each bit is 1 with probability 1/2: 20000 samples, 5 sigma = 0.018
    assert np.all(np.abs(bits - 0.5) < 0.018)


# --------------------------------------------------------- index and rho+ --

def test_rho_plus_paper_example(orc):
    # Sec. 4.1: rho+(00101) = 3.  Put the 5-bit string right after a b-bit
    # index and pad the word with zeros.
    word_bits, expected = "00101", int(PAPER["rho_plus_00101"][0])
    for b in range(4, 13):
        idx = (1 << b) - 3 if b > 2 else 0
        s = format(idx, f"0{b}b") + word_bits + "0" * (64 - b - 5)
        x = int(s, 2)
        assert orc.hash_split(x, b) == (idx, expected)


@pytest.mark.parametrize("b", list(range(4, 13)))
def test_split_crafted_words(orc, b):
    top = 1 << (63 - b)                      # first bit after the index
    cases = [0, 2**64 - 1, top, top - 1, 1, 1 << 63, (1 << 63) | 1,
             ((1 << b) - 1) << (64 - b), (((1 << b) - 1) << (64 - b)) | 1]
    for x in cases:
        assert orc.hash_split(x, b) == brute.split_bits(x, b), hex(x)
    # all-zero remainder: capped at 64 - b; top remainder bit set: rho+ = 1
    assert orc.hash_split(0, b)[1] == 64 - b
    assert orc.hash_split(top, b)[1] == 1
    assert orc.hash_split(1, b)[1] == 64 - b   # 63-b zeros then a one: rho+ = 64-b


def test_split_random_words(orc):
    rng = np.random.default_rng(3)
    for b in (4, 6, 7, 12):
        for x in rng.integers(0, 2**63, 300, dtype=np.uint64):
            x = int(x) << int(rng.integers(0, 2))
            # sparse words exercise long zero runs
            y = int(x) >> int(rng.integers(0, 60))
            for w in (x & brute.M64, y):
                assert orc.hash_split(w, b) == brute.split_bits(w, b)


def test_index_and_rho_distribution(orc):
    # index uniform over p registers, rho+ geometric: P(rho+ = k) = 2^-k
    b, N = 4, 40000
    idx = np.zeros(16)
    rho = np.zeros(70)
    for v in range(N):
        i, r = orc.hash_split(orc.hash64(99, v), b)
        idx[i] += 1
        rho[r] += 1
    chi2 = ((idx - N / 16) ** 2 / (N / 16)).sum()
    assert chi2 < 45          # 15 dof: p-value ~ 1e-4
    for k in range(1, 8):
        expect = N * 2.0 ** -k
        assert abs(rho[k] - expect) < 5 * math.sqrt(expect)


# -------------------------------------------------------------- estimator --

def test_alpha_constants(orc):
    for p in (16, 32, 64):
        assert orc.alpha(p) == float(FFGH[str(p)][0])
    c0, c1 = map(float, FFGH["formula"])
    for b in range(7, 13):
        p = 1 << b
        assert orc.alpha(p) == c0 / (1 + c1 / p)


@pytest.mark.parametrize("b", list(range(4, 13)))
def test_size_closed_forms(orc, b):
    p = 1 << b
    M = np.zeros(p, dtype=np.uint8)
    assert orc.size(M, b) == 0.0                          # empty counter
    for r in (1, 3, 20, 64 - b):
        M = np.zeros(p, dtype=np.uint8)
        M[p // 3] = r                                      # one register set
        assert orc.size(M, b) == pytest.approx(p * math.log(p / (p - 1)), rel=1e-14)
    for k in (2, p // 4, p // 2):
        M = np.zeros(p, dtype=np.uint8)
        M[:k] = 1                                          # k registers = 1
        raw = brute.alpha_ffgh(p) * p * p / (p - k + k / 2)
        assert raw <= 2.5 * p
        assert orc.size(M, b) == pytest.approx(brute.linear_counting(p, k), rel=1e-14)
    for r in (4, 9, 30):
        M = np.full(p, r, dtype=np.uint8)                  # all registers = r
        expect = brute.alpha_ffgh(p) * p * 2.0 ** r
        assert expect > 2.5 * p
        assert orc.size(M, b) == pytest.approx(expect, rel=1e-15)


def test_small_range_switch(orc):
    b, p = 4, 16
    # one empty register left and a raw estimate below 5p/2: linear counting
    M = np.full(p, 1, dtype=np.uint8)
    M[0] = 0
    raw = brute.alpha_ffgh(p) * p * p / (1 + 15 / 2)
    assert raw <= 2.5 * p
    assert orc.size(M, b) == pytest.approx(p * math.log(p), rel=1e-14)
    # one empty register but a raw estimate above 5p/2: the raw estimate
    M = np.full(p, 3, dtype=np.uint8)
    M[0] = 0
    raw = brute.alpha_ffgh(p) * p * p / (1 + 15 / 8)
    assert 2.5 * p < raw < 5 * p
    assert orc.size(M, b) == pytest.approx(raw, rel=1e-15)


def test_register_sum_exact(orc):
    rng = np.random.default_rng(11)
    for b in (4, 5, 6, 7, 10, 12):
        p = 1 << b
        for _ in range(50):
            M = rng.integers(0, 64 - b + 1, size=p).astype(np.uint8)
            M[rng.random(p) < 0.3] = 0
            exact = sum(Fraction(1, 2 ** int(m)) for m in M)
            got, V = orc.register_sum(M, b)
            assert V == int((M == 0).sum())
            # two roundings (integer-to-double, then the add): within 2 ulp
            assert abs(Fraction(got) - exact) <= 2 * Fraction(math.ulp(float(exact)))


def _rsd(orc, b, N, trials, seed):
    rng = np.random.default_rng(seed)
    p = 1 << b
    est = np.empty(trials)
    for k in range(trials):
        M = np.zeros(p, dtype=np.uint8)
        orc.add_stream(M, b, rng.integers(0, 2**64 - 1, size=N, dtype=np.uint64, endpoint=True))
        est[k] = orc.size(M, b)
    return est.mean() / N, est.std(ddof=1) / N


def test_rsd_p64_matches_paper(orc):
    # Sec. 8: p = 64 registers give a relative standard deviation of 13.18%.
    target = float(PAPER["rsd_p64"][0])
    mean, rsd = _rsd(orc, 6, 20000, 3000, 1)
    assert abs(mean - 1) < 0.012
    assert abs(rsd - target) < 0.008     # sampling error of the std ~ 0.0017


def test_rsd_p4096_matches_paper(orc):
    # Sec. 8: p = 4096 registers give 1.62%; and every RSD <= 1.06/sqrt(p).
    target = float(PAPER["rsd_p4096"][0])
    mean, rsd = _rsd(orc, 12, 200000, 300, 2)
    assert abs(mean - 1) < 0.004
    assert abs(rsd - target) < 0.0025
    assert rsd <= float(PAPER["rsd_bound_coeff"][0]) / 64 + 0.0025


def test_node_hash_estimates_distinct_ids(orc):
    # The node hash behaves like a random hash: counting n distinct ids with
    # many seeds has the RSD of Sec. 4.1.
    b, p, N = 5, 32, 2000
    est = []
    for seed in range(200):
        M = np.zeros(p, dtype=np.uint8)
        for v in range(N):
            orc.add(M, b, orc.hash64(seed * 7919 + 1, v))
        est.append(orc.size(M, b))
    est = np.array(est) / N
    assert abs(est.mean() - 1) < 0.03
    assert est.std(ddof=1) < 1.06 / math.sqrt(p) * 1.15
