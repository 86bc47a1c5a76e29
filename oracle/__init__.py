"""CPU oracle for HyperBall (Boldi & Vigna, arXiv:1308.2144).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the CUDA library and its Python
binding never do.  It shares no code with the CUDA path.

The arithmetic lives in ``hb_oracle.c`` (plain C loops in fp64, compiled with
``-ffp-contract=off``); this module only compiles it with gcc and wraps its
functions with ctypes and numpy.  See the header of ``hb_oracle.c`` for the
passages each function follows and the readings taken where the paper is
silent.  Every function here is pinned by the ``-m "not gpu"`` tests against
closed forms, the paper's printed values and brute-force ball counting.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hb_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile hb_oracle.c into a shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load(path: str):
    """Open a compiled oracle library and declare its C signatures."""
    L = ctypes.CDLL(path)
    L.orc_hash.restype = ctypes.c_uint64
    L.orc_hash.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    L.orc_hash_split.restype = None
    L.orc_hash_split.argtypes = [ctypes.c_uint64, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_uint32),
                                 ctypes.POINTER(ctypes.c_uint32)]
    L.orc_alpha.restype = ctypes.c_double
    L.orc_alpha.argtypes = [ctypes.c_int]
    L.orc_add.restype = None
    L.orc_add.argtypes = [_u8p, ctypes.c_int, ctypes.c_uint64]
    L.orc_add_stream.restype = None
    L.orc_add_stream.argtypes = [_u8p, ctypes.c_int, _u64p, ctypes.c_int64]
    L.orc_register_sum.restype = ctypes.c_double
    L.orc_register_sum.argtypes = [_u8p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.orc_size.restype = ctypes.c_double
    L.orc_size.argtypes = [_u8p, ctypes.c_int]
    L.orc_set_threads.restype = None
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_get_threads.restype = ctypes.c_int
    L.orc_get_threads.argtypes = []
    L.orc_init.restype = None
    L.orc_init.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, _u8p]
    L.orc_init_weighted.restype = None
    L.orc_init_weighted.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, _i64p, _u8p]
    L.orc_step_ex.restype = ctypes.c_int64
    L.orc_step_ex.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int, ctypes.c_int32,
                              _u8p, _u8p, _f64p, _f64p, ctypes.c_double, _f64p, _u8p]
    L.orc_pack6.restype = ctypes.c_int
    L.orc_pack6.argtypes = [_u8p, ctypes.c_int, _u8p]
    L.orc_unpack6.restype = None
    L.orc_unpack6.argtypes = [_u8p, ctypes.c_int, _u8p]
    L.orc_step_packed.restype = ctypes.c_int64
    L.orc_step_packed.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int, ctypes.c_int32,
                                  _u8p, _u8p, _f64p, _f64p, _u8p]
    L.orc_discount.restype = ctypes.c_double
    L.orc_discount.argtypes = [_f64p, ctypes.c_int32, ctypes.c_int64]
    L.orc_run_ex.restype = ctypes.c_int
    L.orc_run_ex.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int, ctypes.c_uint64,
                             _i64p, _f64p, ctypes.c_int32, ctypes.c_int32, _u8p, _f64p, _f64p,
                             _f64p, _i32p, _u8p]
    L.orc_step.restype = ctypes.c_int64
    L.orc_step.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int, ctypes.c_int32,
                           _u8p, _u8p, _f64p, _f64p, _u8p]
    L.orc_run.restype = ctypes.c_int
    L.orc_run.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int, ctypes.c_uint64,
                          ctypes.c_int32, _u8p, _f64p, _f64p, _i32p, _u8p]
    L.orc_finalize.restype = None
    L.orc_finalize.argtypes = [ctypes.c_int64, ctypes.c_int, _u8p, _f64p, _f64p,
                               _f64p, _f64p, _f64p, _f64p]
    L.orc_neighbourhood.restype = ctypes.c_double
    L.orc_neighbourhood.argtypes = [ctypes.c_int64, ctypes.c_int, _u8p]
    L.orc_must_check.restype = None
    L.orc_must_check.argtypes = [ctypes.c_int64, _i64p, _i32p, _u8p, _u8p]
    L.orc_exact_centralities.restype = ctypes.c_int
    L.orc_exact_centralities.argtypes = [ctypes.c_int64, _i64p, _i32p, _i64p,
                                         ctypes.c_int64, _f64p, _f64p, _f64p, _i32p]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t) if a is not None else None


def _csr(offsets, targets):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    tgt = np.ascontiguousarray(targets, dtype=np.int32)
    return off, tgt


# ----------------------------------------------------------------- counter --

def hash64(seed: int, v: int) -> int:
    """h(v): SplitMix64 output number v+1 for a generator seeded with `seed`."""
    return int(lib().orc_hash(seed & (2**64 - 1), v & (2**64 - 1)))


def hash_split(x: int, b: int) -> tuple[int, int]:
    """(h_b(x), rho+(h^b(x))) for a 64-bit word x (Sec. 4.1)."""
    i = ctypes.c_uint32()
    r = ctypes.c_uint32()
    lib().orc_hash_split(x & (2**64 - 1), b, ctypes.byref(i), ctypes.byref(r))
    return int(i.value), int(r.value)


def alpha(p: int) -> float:
    return float(lib().orc_alpha(p))


def add(M: np.ndarray, b: int, x: int) -> None:
    assert M.dtype == np.uint8 and M.flags.c_contiguous and M.size == 1 << b
    lib().orc_add(_p(M, _u8p), b, x & (2**64 - 1))


def add_stream(M: np.ndarray, b: int, xs: np.ndarray) -> None:
    assert M.dtype == np.uint8 and M.flags.c_contiguous and M.size == 1 << b
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    lib().orc_add_stream(_p(M, _u8p), b, _p(xs, _u64p), xs.size)


def register_sum(M: np.ndarray, b: int) -> tuple[float, int]:
    M = np.ascontiguousarray(M, dtype=np.uint8)
    V = ctypes.c_int()
    s = lib().orc_register_sum(_p(M, _u8p), b, ctypes.byref(V))
    return float(s), int(V.value)


def size(M: np.ndarray, b: int) -> float:
    M = np.ascontiguousarray(M, dtype=np.uint8)
    assert M.size == 1 << b
    return float(lib().orc_size(_p(M, _u8p), b))


def set_threads(k: int) -> None:
    lib().orc_set_threads(int(k))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# --------------------------------------------------------------- HyperBall --

def init(n: int, b: int, seed: int) -> np.ndarray:
    c = np.zeros((n, 1 << b), dtype=np.uint8)
    lib().orc_init(n, b, seed & (2**64 - 1), _p(c, _u8p))
    return c


def init_weighted(n: int, b: int, seed: int, weights) -> np.ndarray:
    """Initial counters with node weights simulated by replicas (Sec. 6)."""
    w = np.ascontiguousarray(weights, dtype=np.int64)
    assert w.size == n and (w >= 0).all()
    c = np.zeros((n, 1 << b), dtype=np.uint8)
    lib().orc_init_weighted(n, b, seed & (2**64 - 1), _p(w, _i64p), _p(c, _u8p))
    return c


def discount(table, d: int) -> float:
    """f(d) of a discount table: table[d-1] for 1 <= d <= len, else 0."""
    f = np.ascontiguousarray(table, dtype=np.float64)
    return float(lib().orc_discount(_p(f, _f64p), f.size, d))


def step(offsets, targets, b: int, t: int, cur: np.ndarray,
         sumd: np.ndarray, harm: np.ndarray, disc: np.ndarray | None = None,
         fdist: float = 0.0):
    """One Algorithm 2 iteration at loop index t.  Returns (next, changed,
    n_changed); sumd and harm (and disc, with discount fdist = f(t+1), when
    given) are updated in place."""
    off, tgt = _csr(offsets, targets)
    n = off.size - 1
    cur = np.ascontiguousarray(cur, dtype=np.uint8)
    nxt = np.empty_like(cur)
    changed = np.zeros(n, dtype=np.uint8)
    assert sumd.dtype == np.float64 and harm.dtype == np.float64
    if disc is None:
        k = lib().orc_step(n, _p(off, _i64p), _p(tgt, _i32p), b, t, _p(cur, _u8p),
                           _p(nxt, _u8p), _p(sumd, _f64p), _p(harm, _f64p), _p(changed, _u8p))
    else:
        assert disc.dtype == np.float64 and disc.flags.c_contiguous
        k = lib().orc_step_ex(n, _p(off, _i64p), _p(tgt, _i32p), b, t, _p(cur, _u8p),
                              _p(nxt, _u8p), _p(sumd, _f64p), _p(harm, _f64p), float(fdist),
                              _p(disc, _f64p), _p(changed, _u8p))
    return nxt, changed, int(k)


def pack6(regs: np.ndarray, b: int) -> np.ndarray:
    """Counters (rows of p registers) packed six bits per register (Sec. 4.1
    register width): rows of 3p/4 bytes.  ValueError if a register > 63."""
    regs = np.ascontiguousarray(regs, dtype=np.uint8).reshape(-1, 1 << b)
    out = np.zeros((regs.shape[0], 3 * (1 << b) // 4), dtype=np.uint8)
    for v in range(regs.shape[0]):
        if lib().orc_pack6(_p(regs[v], _u8p), b, _p(out[v], _u8p)) != 0:
            raise ValueError("a register does not fit six bits")
    return out


def unpack6(packed: np.ndarray, b: int) -> np.ndarray:
    """The inverse of pack6."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8).reshape(-1, 3 * (1 << b) // 4)
    out = np.zeros((packed.shape[0], 1 << b), dtype=np.uint8)
    for v in range(packed.shape[0]):
        lib().orc_unpack6(_p(packed[v], _u8p), b, _p(out[v], _u8p))
    return out


def step_packed(offsets, targets, b: int, t: int, cur: np.ndarray, sumd: np.ndarray, harm: np.ndarray):
    """One Algorithm 2 iteration on packed counters (rows of 3p/4 bytes).
    Returns (next, changed, n_changed)."""
    off, tgt = _csr(offsets, targets)
    n = off.size - 1
    cur = np.ascontiguousarray(cur, dtype=np.uint8)
    nxt = np.empty_like(cur)
    changed = np.zeros(n, dtype=np.uint8)
    k = lib().orc_step_packed(n, _p(off, _i64p), _p(tgt, _i32p), b, t, _p(cur, _u8p), _p(nxt, _u8p),
                              _p(sumd, _f64p), _p(harm, _f64p), _p(changed, _u8p))
    if k < 0:
        raise ValueError("a register does not fit six bits")
    return nxt, changed, int(k)


class RunResult:
    def __init__(self, regs, sumd, harm, steps, converged, changed_hist, disc=None):
        self.regs = regs
        self.sumd = sumd
        self.harm = harm
        self.steps = steps
        self.converged = converged
        self.changed_hist = changed_hist
        self.disc = disc


def run(offsets, targets, b: int, seed: int, max_steps: int = 1 << 20,
        keep_changed: bool = False, weights=None, discount=None) -> RunResult:
    """Algorithm 2 to its fixpoint (or max_steps iterations).  ``weights``
    (one non-negative integer per node, Sec. 6) and ``discount`` (a table
    f(1), f(2), ...; Sec. 7, which adds the ``disc`` accumulator) are
    optional."""
    off, tgt = _csr(offsets, targets)
    n = off.size - 1
    p = 1 << b
    regs = np.zeros((n, p), dtype=np.uint8)
    sumd = np.zeros(n, dtype=np.float64)
    harm = np.zeros(n, dtype=np.float64)
    steps = ctypes.c_int32()
    hist = None
    cap = max_steps
    if keep_changed:
        cap = min(max_steps, 4096)
        hist = np.zeros((cap, n), dtype=np.uint8)
    w = None
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.int64)
        assert w.size == n and (w >= 0).all()
    f, disc = None, None
    if discount is not None:
        f = np.ascontiguousarray(discount, dtype=np.float64)
        disc = np.zeros(n, dtype=np.float64)
    rc = lib().orc_run_ex(n, _p(off, _i64p), _p(tgt, _i32p), b, seed & (2**64 - 1),
                          _p(w, _i64p), _p(f, _f64p), 0 if f is None else f.size, cap,
                          _p(regs, _u8p), _p(sumd, _f64p), _p(harm, _f64p), _p(disc, _f64p),
                          ctypes.byref(steps), _p(hist, _u8p) if hist is not None else None)
    if rc < 0:
        raise MemoryError("oracle run: allocation failed")
    s = int(steps.value)
    return RunResult(regs, sumd, harm, s, rc == 0, hist[:s] if hist is not None else None, disc)


def finalize(b: int, regs: np.ndarray, sumd: np.ndarray, harm: np.ndarray):
    """Sec. 3 centralities: dict with closeness, harmonic, lin, reachable."""
    regs = np.ascontiguousarray(regs, dtype=np.uint8)
    n = regs.shape[0]
    out = {k: np.empty(n, dtype=np.float64) for k in ("closeness", "harmonic", "lin", "reachable")}
    lib().orc_finalize(n, b, _p(regs, _u8p), _p(np.ascontiguousarray(sumd), _f64p),
                       _p(np.ascontiguousarray(harm), _f64p), _p(out["closeness"], _f64p),
                       _p(out["harmonic"], _f64p), _p(out["lin"], _f64p),
                       _p(out["reachable"], _f64p))
    return out


def must_check(offsets, targets, changed: np.ndarray) -> np.ndarray:
    off, tgt = _csr(offsets, targets)
    n = off.size - 1
    ch = np.ascontiguousarray(changed, dtype=np.uint8)
    must = np.zeros(n, dtype=np.uint8)
    lib().orc_must_check(n, _p(off, _i64p), _p(tgt, _i32p), _p(ch, _u8p), _p(must, _u8p))
    return must


def exact_centralities(offsets, targets, sources=None):
    """Exact Sec. 3 ingredients by BFS along the scanned graph's arcs.
    Returns dict sumd, harm, reach, ecc (one entry per source)."""
    off, tgt = _csr(offsets, targets)
    n = off.size - 1
    src = None if sources is None else np.ascontiguousarray(sources, dtype=np.int64)
    k = n if src is None else src.size
    out = {"sumd": np.zeros(k), "harm": np.zeros(k), "reach": np.zeros(k),
           "ecc": np.zeros(k, dtype=np.int32)}
    rc = lib().orc_exact_centralities(n, _p(off, _i64p), _p(tgt, _i32p),
                                      _p(src, _i64p) if src is not None else None, k,
                                      _p(out["sumd"], _f64p), _p(out["harm"], _f64p),
                                      _p(out["reach"], _f64p), _p(out["ecc"], _i32p))
    if rc != 0:
        raise MemoryError("oracle exact BFS: allocation failed")
    return out


def run_stats(offsets, targets, b: int, seeds, which: str, weights=None, discount=None):
    """Sec. 5, multiple runs: per node, the mean and the empirical (sample,
    divisor R-1) standard deviation of one centrality over independent runs
    of Algorithm 2 with the given hash seeds (numpy's mean and std).
    ``which`` = "discounted" takes the Sec. 7 accumulator of ``discount``."""
    vals = []
    for s in seeds:
        res = run(offsets, targets, b, s, weights=weights, discount=discount)
        vals.append(res.disc if which == "discounted" else finalize(b, res.regs, res.sumd, res.harm)[which])
    vals = np.array(vals)
    sd = vals.std(axis=0, ddof=1) if len(seeds) > 1 else np.zeros(vals.shape[1])
    return vals.mean(axis=0), sd


def neighbourhood(regs: np.ndarray, b: int) -> float:
    """N(t) = sum over nodes of size(c_t[v]) for the counters c_t given."""
    regs = np.ascontiguousarray(regs, dtype=np.uint8)
    return float(lib().orc_neighbourhood(regs.shape[0], b, _p(regs, _u8p)))


def neighbourhood_function(offsets, targets, b: int, seed: int, weights=None):
    """N(0), N(1), ..., N(T) along a whole run of Algorithm 2 (T = the
    iteration count): the estimate after every iteration."""
    off, tgt = _csr(offsets, targets)
    n = off.size - 1
    c = init(n, b, seed) if weights is None else init_weighted(n, b, seed, weights)
    sumd, harm = np.zeros(n), np.zeros(n)
    out = [neighbourhood(c, b)]
    t = 0
    while True:
        c, _, k = step(off, tgt, b, t, c, sumd, harm)
        out.append(neighbourhood(c, b))
        t += 1
        if k == 0:
            return np.array(out)
