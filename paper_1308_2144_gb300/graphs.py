"""Seeded synthetic graph generators (inputs only).

These build the power-law workloads the HyperBall step is measured on:

* ``plain``  -- 10,000 nodes, out-degree Zipf(2.1) on {1..1000}, uniform
  targets; the small correctness workload.
* ``enwiki`` -- R-MAT (0.57, 0.19, 0.19, 0.05) at scale 23, keeping arcs whose
  endpoints are both below 4,206,785 until 101,355,853 are drawn: a stand-in
  with the node and arc counts of the Wikipedia snapshot of the paper's
  Sec. 8 (the snapshot itself is not available here).
* ``web``    -- R-MAT at scale 28 with edge factor 16 (2^32 arcs drawn), int64
  offsets: a GPU-memory-scale stand-in for the paper's ClueWeb09 run.

Labels are permuted (Graph500 style), self-loops and duplicate arcs are
dropped and the resulting arc count is reported.  Centralities are
in-centralities (Sec. 3 footnote, Sec. 5), so each workload is handed to
HyperBall as the transpose S = G^T of the generated graph.

All randomness comes from one counter-based generator, the MurmurHash3
64-bit finaliser applied to a keyed Weyl sequence, written with torch int64
operations so the same graph comes out on the CPU and on the GPU.  This
module holds none of HyperBall's arithmetic; both the CUDA path and the
oracle only consume what it produces.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

_M64 = (1 << 64) - 1


def _s64(c: int) -> int:
    """Two's-complement int64 value of a 64-bit constant."""
    c &= _M64
    return c - (1 << 64) if c >= (1 << 63) else c


_FM1 = _s64(0xFF51AFD7ED558CCD)
_FM2 = _s64(0xC4CEB9FE1A85EC53)
_WEYL = _s64(0xD1B54A32D192ED03)
_KEY = _s64(0xA0761D6478BD642F)


def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def _fmix64(x: torch.Tensor) -> torch.Tensor:
    x = x ^ _srl(x, 33)
    x = x * _FM1
    x = x ^ _srl(x, 33)
    x = x * _FM2
    return x ^ _srl(x, 33)


def _key(seed: int, stream: int) -> int:
    k = torch.tensor([_s64(seed * 0x100000001B3 + stream * 0x9FB21C651E98DF25)], dtype=torch.int64)
    return int(_fmix64(k ^ _KEY)[0])


def rand_u64(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """64-bit random words (as int64) for counter indices ``idx``."""
    k = _key(seed, stream)
    return _fmix64(idx * _WEYL + k)


def rand_uniform(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return _srl(rand_u64(seed, stream, idx), 11).to(torch.float64) * (2.0 ** -53)


@dataclass
class CSRGraph:
    """A directed graph in CSR form: successors of v are
    targets[offsets[v]:offsets[v+1]]."""
    n: int
    offsets: torch.Tensor
    targets: torch.Tensor
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.targets.numel())

    def to(self, device) -> "CSRGraph":
        return CSRGraph(self.n, self.offsets.to(device), self.targets.to(device), self.name,
                        dict(self.meta))

    def numpy(self):
        return self.offsets.cpu().numpy(), self.targets.cpu().numpy()

    def degrees(self) -> torch.Tensor:
        return (self.offsets[1:] - self.offsets[:-1]).to(torch.int64)


# --------------------------------------------------------------- assembly --

def arcs_to_csr(src: torch.Tensor, dst: torch.Tensor, n: int, *, transpose: bool = False,
                offsets_dtype=torch.int64, name: str = "", drop_self_loops: bool = True,
                dedup: bool = True, bucket_bits: int = 0) -> CSRGraph:
    """CSR of the arcs src->dst (or of their transpose), with sorted
    successor lists, self-loops and duplicates optionally removed.

    ``bucket_bits`` > 0 processes rows in 2^bucket_bits groups to bound the
    temporary memory of very large graphs."""
    rows, cols = (dst, src) if transpose else (src, dst)
    device = rows.device
    shift = max(1, int(n - 1).bit_length())
    if bucket_bits <= 0:
        rows64 = rows.to(torch.int64)
        cols64 = cols.to(torch.int64)
        if drop_self_loops:
            keep = rows64 != cols64
            rows64, cols64 = rows64[keep], cols64[keep]
        key = (rows64 << shift) | cols64
        del rows64, cols64
        key = torch.unique(key, sorted=True) if dedup else torch.sort(key).values
        r = key >> shift
        tgt = (key & ((1 << shift) - 1)).to(torch.int32)
        counts = torch.bincount(r, minlength=n)
        del key, r
    else:
        parts_t, parts_c = [], []
        nb = 1 << bucket_bits
        rshift = max(0, shift - bucket_bits)
        rows_per = 1 << rshift
        for bk in range(nb):
            sel = (rows >> rshift) == bk
            r = rows[sel].to(torch.int64)
            c = cols[sel].to(torch.int64)
            del sel
            if drop_self_loops:
                keep = r != c
                r, c = r[keep], c[keep]
            key = ((r - bk * rows_per) << shift) | c
            del r, c
            key = torch.unique(key, sorted=True) if dedup else torch.sort(key).values
            lr = key >> shift
            parts_t.append((key & ((1 << shift) - 1)).to(torch.int32))
            lo = bk * rows_per
            hi = min(n, lo + rows_per)
            if hi > lo:
                parts_c.append(torch.bincount(lr, minlength=hi - lo)[: hi - lo])
            del key, lr
        tgt = torch.cat(parts_t) if parts_t else torch.zeros(0, dtype=torch.int32, device=device)
        counts = torch.cat(parts_c) if parts_c else torch.zeros(n, dtype=torch.int64, device=device)
        counts = counts[:n]
        if counts.numel() < n:
            counts = torch.cat([counts, torch.zeros(n - counts.numel(), dtype=torch.int64,
                                                    device=device)])
    off = torch.zeros(n + 1, dtype=torch.int64, device=device)
    off[1:] = torch.cumsum(counts, 0)
    return CSRGraph(n, off.to(offsets_dtype), tgt.contiguous(), name)


def transpose(g: CSRGraph, offsets_dtype=None) -> CSRGraph:
    """The transpose graph (arcs reversed), keeping every arc."""
    src = torch.repeat_interleave(torch.arange(g.n, device=g.targets.device, dtype=torch.int32),
                                  g.degrees())
    return arcs_to_csr(src, g.targets, g.n, transpose=True,
                       offsets_dtype=offsets_dtype or g.offsets.dtype, name=g.name + "^T",
                       drop_self_loops=False, dedup=False)


def from_edges(n: int, edges, *, offsets_dtype=torch.int64, keep_all: bool = True,
               name: str = "") -> CSRGraph:
    """CSR from a small explicit arc list (tests).  ``keep_all`` keeps
    self-loops and duplicate arcs exactly as given."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    src = torch.from_numpy(e[:, 0].copy())
    dst = torch.from_numpy(e[:, 1].copy())
    return arcs_to_csr(src, dst, n, offsets_dtype=offsets_dtype, name=name,
                       drop_self_loops=not keep_all, dedup=not keep_all)


def induced_subgraph(g: CSRGraph, nodes: torch.Tensor) -> CSRGraph:
    """Arcs of g between the given nodes, relabelled 0..k-1 in the order given."""
    dev = g.targets.device
    nodes = nodes.to(dev, torch.int64)
    k = nodes.numel()
    newid = torch.full((g.n,), -1, dtype=torch.int64, device=dev)
    newid[nodes] = torch.arange(k, device=dev)
    deg = g.degrees()
    src = torch.repeat_interleave(torch.arange(g.n, device=dev), deg)
    s2 = newid[src]
    d2 = newid[g.targets.to(torch.int64)]
    keep = (s2 >= 0) & (d2 >= 0)
    return arcs_to_csr(s2[keep], d2[keep], k, offsets_dtype=g.offsets.dtype,
                       name=g.name + f"[{k}]", drop_self_loops=False, dedup=False)


def permutation(n: int, seed: int, stream: int, device="cpu") -> torch.Tensor:
    """A seeded random permutation of 0..n-1 (argsort of random keys)."""
    keys = rand_u64(seed, stream, torch.arange(n, device=device, dtype=torch.int64))
    return torch.argsort(keys, stable=True)


# --------------------------------------------------------------- families --

_STREAM_DEG, _STREAM_TGT, _STREAM_PERM, _STREAM_RMAT = 1, 2, 3, 16


def zipf_arcs(n: int, s: float = 2.1, kmax: int = 1000, seed: int = 1, min_degree: int = 1,
              device="cpu"):
    """Out-degree ~ Zipf(s) on {min_degree..kmax}, uniform targets."""
    ks = torch.arange(min_degree, kmax + 1, dtype=torch.float64, device=device)
    pmf = ks ** (-s)
    cdf = torch.cumsum(pmf, 0) / pmf.sum()
    cdf[-1] = 1.0
    u = rand_uniform(seed, _STREAM_DEG, torch.arange(n, device=device, dtype=torch.int64))
    deg = torch.searchsorted(cdf, u, right=True).clamp_max(kmax - min_degree) + min_degree
    src = torch.repeat_interleave(torch.arange(n, device=device, dtype=torch.int64), deg)
    j = torch.arange(src.numel(), device=device, dtype=torch.int64)
    dst = torch.floor(rand_uniform(seed, _STREAM_TGT, j) * n).to(torch.int64).clamp_max(n - 1)
    return src, dst


def rmat_arcs(scale: int, count: int, a=0.57, b=0.19, c=0.19, seed: int = 2, start: int = 0,
              device="cpu"):
    """Arcs number start..start+count-1 of a seeded R-MAT stream: each of the
    `scale` levels picks a quadrant with probabilities (a, b, c, d)."""
    idx = torch.arange(start, start + count, device=device, dtype=torch.int64)
    tA = int(a * 2 ** 32)
    tB = int((a + b) * 2 ** 32)
    tC = int((a + b + c) * 2 ** 32)
    src = torch.zeros(count, dtype=torch.int64, device=device)
    dst = torch.zeros(count, dtype=torch.int64, device=device)
    for lvl in range(0, scale, 2):
        w = rand_u64(seed, _STREAM_RMAT + lvl // 2, idx)
        for half in range(2):
            level = lvl + half
            if level >= scale:
                break
            u = _srl(w, 32) if half == 0 else (w & 0xFFFFFFFF)
            row = (u >= tB).to(torch.int64)
            col = ((u >= tA) & (u < tB)) | (u >= tC)
            bit = scale - 1 - level
            src |= row << bit
            dst |= col.to(torch.int64) << bit
            del u, row, col
        del w
    return src, dst


def plain_graph(n: int = 10_000, seed: int = 1, min_degree: int = 1, device="cpu") -> CSRGraph:
    """Zipf(2.1) out-degree workload, handed over as S = G^T."""
    src, dst = zipf_arcs(n, seed=seed, min_degree=min_degree, device=device)
    g = arcs_to_csr(src, dst, n, transpose=True, offsets_dtype=torch.int64,
                    name=f"zipf2.1-n{n}-seed{seed}^T")
    g.meta.update(kind="plain", seed=seed, arcs_drawn=int(src.numel()))
    return g


def enwiki_graph(n: int = 4_206_785, m_draw: int = 101_355_853, scale: int = 23, seed: int = 2,
                 device="cpu", chunk: int = 1 << 25) -> CSRGraph:
    """R-MAT stand-in with Wikipedia's node and arc counts, as S = G^T."""
    srcs, dsts, got, start = [], [], 0, 0
    while got < m_draw:
        s, d = rmat_arcs(scale, chunk, seed=seed, start=start, device=device)
        keep = (s < n) & (d < n)
        s, d = s[keep], d[keep]
        need = m_draw - got
        s, d = s[:need], d[:need]
        srcs.append(s.to(torch.int32))
        dsts.append(d.to(torch.int32))
        got += s.numel()
        start += chunk
    src = torch.cat(srcs).to(torch.int64)
    dst = torch.cat(dsts).to(torch.int64)
    del srcs, dsts
    perm = permutation(n, seed, _STREAM_PERM, device=device)
    src, dst = perm[src], perm[dst]
    g = arcs_to_csr(src, dst, n, transpose=True, offsets_dtype=torch.int32,
                    name=f"rmat23-enwiki-n{n}^T")
    g.meta.update(kind="enwiki", seed=seed, arcs_drawn=m_draw)
    return g


def web_graph(scale: int = 28, edge_factor: int = 16, seed: int = 4, device="cuda",
              chunk: int = 1 << 27, bucket_bits: int = 6) -> CSRGraph:
    """R-MAT scale-28 stand-in for a web graph (2^scale * edge_factor arcs
    drawn), int64 offsets, as S = G^T."""
    n = 1 << scale
    total = n * edge_factor
    src = torch.empty(total, dtype=torch.int32, device=device)
    dst = torch.empty(total, dtype=torch.int32, device=device)
    perm = permutation(n, seed, _STREAM_PERM, device=device).to(torch.int32)
    for start in range(0, total, chunk):
        cnt = min(chunk, total - start)
        s, d = rmat_arcs(scale, cnt, seed=seed, start=start, device=device)
        src[start:start + cnt] = perm[s]
        dst[start:start + cnt] = perm[d]
        del s, d
    del perm
    g = arcs_to_csr(src, dst, n, transpose=True, offsets_dtype=torch.int64,
                    name=f"rmat{scale}-ef{edge_factor}^T", bucket_bits=bucket_bits)
    del src, dst
    g.meta.update(kind="web", seed=seed, arcs_drawn=total)
    return g


def rmat_graph(scale: int, edge_factor: int, seed: int, n: int | None = None, device="cpu",
               offsets_dtype=torch.int64) -> CSRGraph:
    """A smaller R-MAT graph (batched and served workloads), as S = G^T.  If
    n < 2^scale, arcs touching nodes >= n are dropped."""
    full = 1 << scale
    n = full if n is None else n
    s, d = rmat_arcs(scale, full * edge_factor if n == full else n * edge_factor,
                     seed=seed, device=device)
    keep = (s < n) & (d < n)
    s, d = s[keep], d[keep]
    perm = permutation(n, seed, _STREAM_PERM, device=device)
    g = arcs_to_csr(perm[s], perm[d], n, transpose=True, offsets_dtype=offsets_dtype,
                    name=f"rmat{scale}-n{n}-ef{edge_factor}-s{seed}^T")
    g.meta.update(kind="rmat", seed=seed)
    return g
