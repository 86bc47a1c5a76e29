"""Brute-force restatements used to pin the oracle (no oracle code is used).

* ``splitmix64`` -- the published SplitMix64 output function with Python
  integers masked to 64 bits;
* ``split_bits`` -- h_b and rho+ of Sec. 4.1 from the 64-character bit
  string of the word;
* ``hll_of_set`` -- Algorithm 1's add() applied to every element of a set;
* ``ball_layers`` -- breadth-first layers along the scanned graph's arcs
  (B(x, r) of Sec. 2 / 4.2 by its definition, not by the recurrence).
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, k: int) -> int:
    """Output number k (1-based) of SplitMix64 seeded with `seed`."""
    z = (seed + k * GOLDEN) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def node_hash(seed: int, v: int) -> int:
    return splitmix64(seed, v + 1)


def split_bits(x: int, b: int) -> tuple[int, int]:
    """(index, rho+) from the bit string: index = leftmost b bits, rho+ =
    leading zeros of the rest plus one, capped at 64 - b."""
    s = format(x & M64, "064b")
    index = int(s[:b], 2)
    rest = s[b:]
    rho = rest.index("1") + 1 if "1" in rest else len(rest) + 1
    return index, min(rho, 64 - b)


def hll_of_set(nodes, b: int, seed: int) -> np.ndarray:
    M = np.zeros(1 << b, dtype=np.uint8)
    for v in nodes:
        i, r = split_bits(node_hash(seed, int(v)), b)
        if r > M[i]:
            M[i] = r
    return M


def adjacency(offsets, targets):
    off = np.asarray(offsets, dtype=np.int64)
    tgt = np.asarray(targets, dtype=np.int64)
    return [tgt[off[v]:off[v + 1]].tolist() for v in range(off.size - 1)]


def bfs_dist(adj, x: int) -> dict:
    dist = {x: 0}
    q = deque([x])
    while q:
        u = q.popleft()
        for w in adj[u]:
            if w not in dist:
                dist[w] = dist[u] + 1
                q.append(w)
    return dist


def ball(dist: dict, r: int):
    return [y for y, d in dist.items() if d <= r]


def alpha_ffgh(p: int) -> float:
    table = {16: 0.673, 32: 0.697, 64: 0.709}
    return table.get(p, 0.7213 / (1 + 1.079 / p))


def linear_counting(p: int, k: int) -> float:
    """Estimate of a counter with k distinct nonzero registers (and its raw
    estimate below 5p/2): p ln(p / (p - k))."""
    return p * math.log(p / (p - k))


def replica_starts(weights) -> list[int]:
    """First replica item of each node: the running total of the weights of
    the nodes before it (Sec. 6 asks only that distinct nodes have disjoint
    replicas; consecutive numbering is the reading taken)."""
    starts, run = [], 0
    for w in weights:
        starts.append(run)
        run += int(w)
    return starts


def hll_of_items(items, b: int, seed: int) -> np.ndarray:
    """Algorithm 1's add() applied to items hashed like node ids."""
    M = np.zeros(1 << b, dtype=np.uint8)
    for x in items:
        i, r = split_bits(node_hash(seed, int(x)), b)
        if r > M[i]:
            M[i] = r
    return M


def replica_items(nodes, weights, starts):
    return [starts[y] + k for y in nodes for k in range(int(weights[y]))]
