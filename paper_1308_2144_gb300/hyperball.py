"""ctypes binding of the HyperBall C ABI (``include/hyperball.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libhyperball.so``.  The functions keep the C names
(``hb_create``, ``hb_step``, ``hb_run_to_fixpoint``, ``hb_get_centralities``,
...); tensors are passed by ``data_ptr()`` (device) or as host buffers (CPU
tensors, numpy arrays), and streams as ``torch.cuda.Stream``.  If the
library is missing or cannot load, these functions raise: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# HYPERBALL_LIB selects another build of the same library (tuning sweeps)
LIB_PATH = os.environ.get("HYPERBALL_LIB") or os.path.join(_HERE, "libhyperball.so")

HB_OK = 0
HB_ERR_INVALID = -1
HB_ERR_OOM = -2
HB_ERR_CUDA = -3
HB_ERR_NOT_CONVERGED = -4
HB_ERR_TIMEOUT = -5
HB_ERR_STATE = -6

HB_TRANSPOSE = 0x1
HB_BORROW_DEVICE_PTRS = 0x2
HB_FP32_ESTIMATE = 0x4
HB_NO_RELABEL = 0x8
HB_PROFILE = 0x10
HB_PULL_GATHER = 0x20
HB_NEIGHBOURHOOD = 0x40
HB_PACKED_REGISTERS = 0x80

FRONTIER = {"auto": 0, "pull": 1, "push": 2, "off": 3}

HB_REQ_QUEUED, HB_REQ_RUNNING, HB_REQ_DONE, HB_REQ_FAILED, HB_REQ_CANCELLED = 0, 1, 2, 3, 4

# every symbol include/hyperball.h declares
EXPORTS = ["hb_default_options", "hb_create", "hb_create32", "hb_step", "hb_run_to_fixpoint",
           "hb_get_centralities", "hb_get_accumulators", "hb_get_registers", "hb_get_frontier",
           "hb_get_info", "hb_reset", "hb_trim_memory", "hb_set_weights", "hb_set_discount", "hb_get_discounted",
           "hb_get_neighbourhood", "hb_create_runs", "hb_get_run_steps", "hb_get_run_centralities",
           "hb_get_run_accumulators", "hb_get_run_discounted", "hb_get_run_stats",
           "hb_save", "hb_load", "hb_destroy", "hb_last_error",
           "hb_version", "hb_step_noalloc", "hb_batch_create", "hb_batch_step", "hb_batch_run",
           "hb_batch_reset", "hb_batch_get_centralities", "hb_batch_get_registers",
           "hb_batch_get_accumulators", "hb_batch_get_info", "hb_batch_get_totals",
           "hb_batch_destroy", "hb_batch_create_runs", "hb_batch_get_run_stats", "hb_tune", "hb_set_class_sizing", "hb_set_hot_nodes", "hb_set_frontier_switch", "hb_set_l2_fetch_bytes", "hb_batch_tune", "hb_server_default_options", "hb_server_create",
           "hb_server_add_graph", "hb_server_submit", "hb_server_wait", "hb_server_cancel", "hb_server_take",
           "hb_server_stats", "hb_server_destroy"]


class HBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class HBNotConverged(HBError):
    pass


class Options(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("frontier", ctypes.c_int32),
                ("max_steps", ctypes.c_int32), ("stream", ctypes.c_void_p), ("arcs_per_slot", ctypes.c_int32),
                ("hot_nodes", ctypes.c_int32), ("hot_passes", ctypes.c_int32),
                ("frontier_switch", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("log2m", ctypes.c_int32),
                ("t", ctypes.c_int32), ("last_changed", ctypes.c_int64),
                ("last_nodes", ctypes.c_int64), ("last_arcs", ctypes.c_int64),
                ("total_arcs", ctypes.c_int64), ("last_sparse", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double), ("kernel_bytes", ctypes.c_double),
                ("push_launches", ctypes.c_int64), ("push_ms", ctypes.c_double),
                ("push_bytes", ctypes.c_double), ("arcs_per_slot", ctypes.c_int32),
                ("hot_nodes", ctypes.c_int32), ("hot_passes", ctypes.c_int32),
                ("packed", ctypes.c_int32), ("frontier_switch", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOptions(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("flags", ctypes.c_uint32), ("max_steps", ctypes.c_int32),
                ("reserve_bytes", ctypes.c_int64), ("large_arcs", ctypes.c_int64), ("large_slots", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("steps", ctypes.c_int32), ("arcs", ctypes.c_int64),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GraphDesc(ctypes.Structure):
    _fields_ = [("offsets", ctypes.c_void_p), ("targets", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("m", ctypes.c_int64), ("log2m", ctypes.c_int32), ("seed", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p


def load():
    """Load libhyperball.so (build it first with ``paper_1308_2144_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing; build it with "
                               "`python -m paper_1308_2144_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        st = ctypes.c_int
        L.hb_default_options.restype = None
        L.hb_default_options.argtypes = [ctypes.POINTER(Options)]
        for name in ("hb_create", "hb_create32"):
            f = getattr(L, name)
            f.restype = st
            f.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                          ctypes.POINTER(Options), ctypes.POINTER(_vp)]
        L.hb_step.restype = st
        L.hb_step.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
        L.hb_run_to_fixpoint.restype = st
        L.hb_run_to_fixpoint.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
        L.hb_get_centralities.restype = st
        L.hb_get_centralities.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.hb_get_accumulators.restype = st
        L.hb_get_accumulators.argtypes = [_vp, _vp, _vp]
        L.hb_get_registers.restype = st
        L.hb_get_registers.argtypes = [_vp, _vp]
        L.hb_get_frontier.restype = st
        L.hb_get_frontier.argtypes = [_vp, _vp, _vp]
        L.hb_get_info.restype = st
        L.hb_get_info.argtypes = [_vp, ctypes.POINTER(Info)]
        L.hb_reset.restype = st
        L.hb_reset.argtypes = [_vp, ctypes.c_uint64]
        L.hb_create_runs.restype = st
        L.hb_create_runs.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Options), ctypes.POINTER(_vp)]
        L.hb_get_run_steps.restype = st
        L.hb_get_run_steps.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
        L.hb_get_run_centralities.restype = st
        L.hb_get_run_centralities.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp]
        L.hb_get_run_accumulators.restype = st
        L.hb_get_run_accumulators.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
        L.hb_get_run_discounted.restype = st
        L.hb_get_run_discounted.argtypes = [_vp, ctypes.c_int32, _vp]
        L.hb_get_run_stats.restype = st
        L.hb_get_run_stats.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
        L.hb_get_neighbourhood.restype = st
        L.hb_get_neighbourhood.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.hb_set_weights.restype = st
        L.hb_set_weights.argtypes = [_vp, _vp]
        L.hb_set_discount.restype = st
        L.hb_set_discount.argtypes = [_vp, _vp, ctypes.c_int32]
        L.hb_get_discounted.restype = st
        L.hb_get_discounted.argtypes = [_vp, _vp]
        L.hb_set_class_sizing.restype = st
        L.hb_set_class_sizing.argtypes = [_vp, ctypes.c_int32]
        L.hb_set_l2_fetch_bytes.restype = st
        L.hb_set_l2_fetch_bytes.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.hb_set_hot_nodes.restype = st
        L.hb_set_hot_nodes.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32]
        L.hb_set_frontier_switch.restype = st
        L.hb_set_frontier_switch.argtypes = [_vp, ctypes.c_double]
        L.hb_tune.restype = st
        L.hb_tune.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
        L.hb_batch_tune.restype = st
        L.hb_batch_tune.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
        L.hb_save.restype = st
        L.hb_save.argtypes = [_vp, ctypes.c_char_p]
        L.hb_load.restype = st
        L.hb_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(Options), ctypes.POINTER(_vp)]
        L.hb_destroy.restype = None
        L.hb_destroy.argtypes = [_vp]
        L.hb_trim_memory.restype = st
        L.hb_trim_memory.argtypes = []
        L.hb_last_error.restype = ctypes.c_char_p
        L.hb_last_error.argtypes = []
        L.hb_version.restype = ctypes.c_char_p
        L.hb_version.argtypes = []
        L.hb_batch_create.restype = st
        L.hb_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(GraphDesc), ctypes.POINTER(Options),
                                      ctypes.POINTER(_vp)]
        L.hb_batch_create_runs.restype = st
        L.hb_batch_create_runs.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Options),
                                           ctypes.POINTER(_vp)]
        L.hb_batch_get_run_stats.restype = st
        L.hb_batch_get_run_stats.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
        L.hb_batch_step.restype = st
        L.hb_batch_step.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
        L.hb_batch_run.restype = st
        L.hb_batch_run.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
        L.hb_batch_reset.restype = st
        L.hb_batch_reset.argtypes = [_vp, _vp]
        L.hb_batch_get_centralities.restype = st
        L.hb_batch_get_centralities.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.hb_batch_get_registers.restype = st
        L.hb_batch_get_registers.argtypes = [_vp, ctypes.c_int, _vp]
        L.hb_batch_get_accumulators.restype = st
        L.hb_batch_get_accumulators.argtypes = [_vp, ctypes.c_int, _vp, _vp]
        L.hb_batch_get_info.restype = st
        L.hb_batch_get_info.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(Info)]
        L.hb_batch_get_totals.restype = st
        L.hb_batch_get_totals.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int64)]
        L.hb_batch_destroy.restype = None
        L.hb_batch_destroy.argtypes = [_vp]
        L.hb_server_default_options.restype = None
        L.hb_server_default_options.argtypes = [ctypes.POINTER(ServerOptions)]
        L.hb_server_create.restype = st
        L.hb_server_create.argtypes = [ctypes.POINTER(ServerOptions), ctypes.POINTER(_vp)]
        L.hb_server_add_graph.restype = st
        L.hb_server_add_graph.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int32)]
        L.hb_server_submit.restype = st
        L.hb_server_submit.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_int64)]
        L.hb_server_wait.restype = st
        L.hb_server_wait.argtypes = [_vp, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(RequestInfo)]
        L.hb_server_cancel.restype = st
        L.hb_server_cancel.argtypes = [_vp, ctypes.c_int64]
        L.hb_server_take.restype = st
        L.hb_server_take.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
        L.hb_server_stats.restype = st
        L.hb_server_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
        L.hb_server_destroy.restype = None
        L.hb_server_destroy.argtypes = [_vp]
        L.hb_step_noalloc.restype = st
        L.hb_step_noalloc.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_int32, _vp, _vp, _vp, _vp, _vp,
                                      ctypes.POINTER(ctypes.c_int64), _vp]
        _lib = L
        return L


def _check(status: int):
    if status == HB_OK:
        return
    msg = load().hb_last_error().decode(errors="replace")
    if status == HB_ERR_NOT_CONVERGED:
        raise HBNotConverged(status, msg)
    raise HBError(status, msg)


def _ptr(x):
    """Pointer of a tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"expected a tensor or an ndarray, got {type(x)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_options(*, transpose=False, borrow=False, fp32=False, relabel=True, frontier="auto",
                 max_steps=1 << 20, stream=None, profile=False, pull_gather=False,
                 neighbourhood=False, arcs_per_slot=0, hot_nodes=0, hot_passes=1, packed=False,
                 frontier_switch=0.0) -> Options:
    o = Options()
    load().hb_default_options(ctypes.byref(o))
    o.flags = ((HB_TRANSPOSE if transpose else 0) | (HB_BORROW_DEVICE_PTRS if borrow else 0)
               | (HB_FP32_ESTIMATE if fp32 else 0) | (0 if relabel else HB_NO_RELABEL)
               | (HB_PROFILE if profile else 0) | (HB_PULL_GATHER if pull_gather else 0)
               | (HB_NEIGHBOURHOOD if neighbourhood else 0) | (HB_PACKED_REGISTERS if packed else 0))
    o.frontier = FRONTIER[frontier] if isinstance(frontier, str) else int(frontier)
    o.max_steps = int(max_steps)
    o.stream = _stream_ptr(stream)
    o.arcs_per_slot = int(arcs_per_slot)
    o.hot_nodes = int(hot_nodes)
    o.hot_passes = int(hot_passes)
    o.frontier_switch = float(frontier_switch)
    return o


# ------------------------------------------------------------ C-ABI calls --

def hb_create(offsets, targets, n: int, m: int, log2m: int, seed: int, options: Options | None = None):
    """Create a handle; int64 offsets use hb_create, int32 offsets hb_create32."""
    L = load()
    h = _vp()
    dt = offsets.dtype
    is32 = dt in (torch.int32, np.int32)
    fn = L.hb_create32 if is32 else L.hb_create
    _check(fn(_ptr(offsets), _ptr(targets), int(n), int(m), int(log2m), int(seed) & (2**64 - 1),
              ctypes.byref(options) if options is not None else None, ctypes.byref(h)))
    return h


def hb_step(h) -> int:
    k = ctypes.c_int64()
    _check(load().hb_step(h, ctypes.byref(k)))
    return int(k.value)


def hb_run_to_fixpoint(h) -> int:
    s = ctypes.c_int32()
    _check(load().hb_run_to_fixpoint(h, ctypes.byref(s)))
    return int(s.value)


def hb_get_centralities(h, closeness=None, harmonic=None, lin=None, reachable=None):
    _check(load().hb_get_centralities(h, _ptr(closeness), _ptr(harmonic), _ptr(lin), _ptr(reachable)))


def hb_get_accumulators(h, sumd=None, harm=None):
    _check(load().hb_get_accumulators(h, _ptr(sumd), _ptr(harm)))


def hb_get_registers(h, out):
    _check(load().hb_get_registers(h, _ptr(out)))


def hb_get_frontier(h, changed=None, must_check=None):
    _check(load().hb_get_frontier(h, _ptr(changed), _ptr(must_check)))


def hb_get_info(h) -> dict:
    info = Info()
    _check(load().hb_get_info(h, ctypes.byref(info)))
    return info.as_dict()


def hb_reset(h, seed: int):
    _check(load().hb_reset(h, int(seed) & (2**64 - 1)))


def hb_set_weights(h, weights=None):
    """Integer node weights (n int64 values in [0, 2^31), Sec. 6); None
    restores unit weights.  Restarts the computation."""
    _check(load().hb_set_weights(h, _ptr(weights)))


def hb_set_discount(h, f=None):
    """Discount table f(1), f(2), ... (float64, Sec. 7); None removes it.
    Restarts the computation."""
    _check(load().hb_set_discount(h, _ptr(f), 0 if f is None else int(f.shape[0])))


def hb_get_discounted(h, out):
    _check(load().hb_get_discounted(h, _ptr(out)))


def hb_get_neighbourhood(h) -> np.ndarray:
    """N(0), ..., N(T) recorded so far (handle created with neighbourhood=True)."""
    k = ctypes.c_int32()
    _check(load().hb_get_neighbourhood(h, None, 0, ctypes.byref(k)))
    out = np.zeros(k.value, dtype=np.float64)
    _check(load().hb_get_neighbourhood(h, _ptr(out), k.value, ctypes.byref(k)))
    return out


def hb_set_l2_fetch_bytes(nbytes: int) -> int:
    """Set the L2 fetch granularity of this process's context on the current
    device (32, 64 or 128 bytes; 0 only reads it); returns the value before."""
    prev = ctypes.c_int32()
    _check(load().hb_set_l2_fetch_bytes(int(nbytes), ctypes.byref(prev)))
    return int(prev.value)


def hb_tune(h) -> int:
    """Autotune the degree-class sizing; returns the chosen arcs per slot."""
    a = ctypes.c_int32()
    _check(load().hb_tune(h, ctypes.byref(a)))
    return int(a.value)


def hb_save(h, path: str):
    _check(load().hb_save(h, path.encode()))


def hb_load(path: str, options: Options | None = None):
    h = _vp()
    _check(load().hb_load(path.encode(), ctypes.byref(options) if options is not None else None,
                          ctypes.byref(h)))
    return h


def hb_destroy(h):
    if h:
        load().hb_destroy(h)


def hb_trim_memory():
    """Return the device memory cached in the library's pools (freed by
    destroyed handles) to the device."""
    _check(load().hb_trim_memory())


def hb_version() -> str:
    return load().hb_version().decode()


def hb_step_noalloc(offsets, targets, n: int, m: int, log2m: int, t: int, cur, nxt, sumd, harm,
                    changed, stream=None) -> int:
    """One iteration that allocates no device memory (all tensors on the
    GPU; scratch comes from a static device array).  Returns the number of
    changed nodes."""
    k = ctypes.c_int64()
    _check(load().hb_step_noalloc(_ptr(offsets), _ptr(targets), int(n), int(m), int(log2m), int(t),
                                  _ptr(cur), _ptr(nxt), _ptr(sumd), _ptr(harm), _ptr(changed),
                                  ctypes.byref(k), _stream_ptr(stream)))
    return int(k.value)


class HyperBallBatch:
    """Many graphs advanced together (the batched form).  ``graphs`` is a
    list of (offsets, targets, n, log2m, seed) with tensors kept alive by
    this object."""

    CENTRALITIES = ("closeness", "harmonic", "lin", "reachable")

    def __init__(self, graphs, **opts):
        self._keep = []
        descs = (GraphDesc * len(graphs))()
        self.sizes = []
        for i, (off, tgt, n, log2m, seed) in enumerate(graphs):
            self._keep += [off, tgt]
            descs[i] = GraphDesc(_ptr(off).value, _ptr(tgt).value if tgt.numel() else None, int(n),
                                 int(tgt.shape[0]), int(log2m), int(seed) & (2**64 - 1))
            self.sizes.append((int(n), 1 << int(log2m)))
        self.k = len(graphs)
        self.options = make_options(**opts)
        self._h = _vp()
        _check(load().hb_batch_create(self.k, descs, ctypes.byref(self.options), ctypes.byref(self._h)))

    @classmethod
    def runs(cls, offsets, targets, n: int, log2m: int, seeds, **opts) -> "HyperBallBatch":
        """Multiple runs of one graph (Sec. 5): run r uses seeds[r]; the runs
        share one device copy of the graph."""
        if offsets.dtype in (torch.int32, np.int32):   # the entry point takes int64 offsets
            offsets = offsets.to(torch.int64) if isinstance(offsets, torch.Tensor) else offsets.astype(np.int64)
        self = cls.__new__(cls)
        self._keep = [offsets, targets]
        self.k = len(seeds)
        self.sizes = [(int(n), 1 << int(log2m))] * self.k
        self.options = make_options(**opts)
        self._h = _vp()
        arr = (ctypes.c_uint64 * self.k)(*[int(x) & (2**64 - 1) for x in seeds])
        _check(load().hb_batch_create_runs(_ptr(offsets), _ptr(targets) if targets.shape[0] else None,
                                           int(n), int(targets.shape[0]), int(log2m), self.k, arr,
                                           ctypes.byref(self.options), ctypes.byref(self._h)))
        return self

    def run_stats(self, which, device="cuda"):
        """Per-node mean and empirical standard deviation over the graphs
        of the batch of one centrality ("closeness", "harmonic", "lin",
        "reachable")."""
        n, _ = self.sizes[0]
        w = self.CENTRALITIES.index(which) if isinstance(which, str) else int(which)
        mean = torch.empty(n, dtype=torch.float64, device=device)
        sd = torch.empty(n, dtype=torch.float64, device=device)
        _check(load().hb_batch_get_run_stats(self._h, w, _ptr(mean), _ptr(sd)))
        return mean, sd

    def step(self) -> int:
        a = ctypes.c_int32()
        _check(load().hb_batch_step(self._h, ctypes.byref(a)))
        return int(a.value)

    def run(self) -> int:
        it = ctypes.c_int32()
        _check(load().hb_batch_run(self._h, ctypes.byref(it)))
        return int(it.value)

    def tune(self) -> int:
        a = ctypes.c_int32()
        _check(load().hb_batch_tune(self._h, ctypes.byref(a)))
        return int(a.value)

    def reset(self, seeds=None):
        arr = None
        if seeds is not None:
            arr = (ctypes.c_uint64 * self.k)(*[int(x) & (2**64 - 1) for x in seeds])
        _check(load().hb_batch_reset(self._h, arr))

    def totals(self):
        it, act, arcs = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().hb_batch_get_totals(self._h, ctypes.byref(it), ctypes.byref(act), ctypes.byref(arcs)))
        return int(it.value), int(act.value), int(arcs.value)

    def info(self, i) -> dict:
        info = Info()
        _check(load().hb_batch_get_info(self._h, i, ctypes.byref(info)))
        return info.as_dict()

    def registers(self, i, device="cuda"):
        n, p = self.sizes[i]
        out = torch.empty((n, p), dtype=torch.uint8, device=device)
        _check(load().hb_batch_get_registers(self._h, i, _ptr(out)))
        return out

    def accumulators(self, i, device="cuda"):
        n, _ = self.sizes[i]
        s = torch.empty(n, dtype=torch.float64, device=device)
        h = torch.empty(n, dtype=torch.float64, device=device)
        _check(load().hb_batch_get_accumulators(self._h, i, _ptr(s), _ptr(h)))
        return s, h

    def centralities(self, i, device="cuda") -> dict:
        n, _ = self.sizes[i]
        out = {k: torch.empty(n, dtype=torch.float64, device=device)
               for k in ("closeness", "harmonic", "lin", "reachable")}
        _check(load().hb_batch_get_centralities(self._h, i, _ptr(out["closeness"]), _ptr(out["harmonic"]),
                                                _ptr(out["lin"]), _ptr(out["reachable"])))
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().hb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HyperBallServer:
    """The serving form: a request loop with continuous batching over a
    pool of device-resident graphs (see hb_server_* in hyperball.h)."""

    def __init__(self, slots=32, fp32=False, max_steps=1 << 16, reserve_bytes=4 << 30, large_slots=0,
                 large_arcs=None):
        L = load()
        o = ServerOptions()
        L.hb_server_default_options(ctypes.byref(o))
        o.slots, o.flags, o.max_steps, o.reserve_bytes = int(slots), HB_FP32_ESTIMATE if fp32 else 0, \
            int(max_steps), int(reserve_bytes)
        o.large_slots = int(large_slots)
        if large_arcs is not None:
            o.large_arcs = int(large_arcs)
        self._h = _vp()
        _check(L.hb_server_create(ctypes.byref(o), ctypes.byref(self._h)))
        self.sizes = []

    def add_graph(self, offsets, targets, n, log2ms=(4,)) -> int:
        arr = (ctypes.c_int32 * len(log2ms))(*[int(x) for x in log2ms])
        gid = ctypes.c_int32()
        _check(load().hb_server_add_graph(self._h, _ptr(offsets), _ptr(targets) if targets.shape[0] else None,
                                          int(n), int(targets.shape[0]), arr, len(log2ms), ctypes.byref(gid)))
        self.sizes.append(int(n))
        return int(gid.value)

    def submit(self, graph_id, log2m, seed) -> int:
        rid = ctypes.c_int64()
        _check(load().hb_server_submit(self._h, int(graph_id), int(log2m), int(seed) & (2**64 - 1),
                                       ctypes.byref(rid)))
        return int(rid.value)

    def wait(self, request_id, timeout=-1.0) -> dict:
        info = RequestInfo()
        _check(load().hb_server_wait(self._h, int(request_id), float(timeout), ctypes.byref(info)))
        return info.as_dict()

    def cancel(self, request_id):
        _check(load().hb_server_cancel(self._h, int(request_id)))

    def take(self, request_id, n, out=None) -> dict:
        """Copy a finished request's centralities into `out` (a dict of
        float64 buffers of n entries: numpy, or torch on the host (pinned is
        fastest) or the GPU), allocated here if None."""
        if out is None:
            out = {k: np.empty(n, dtype=np.float64) for k in ("closeness", "harmonic", "lin", "reachable")}
        _check(load().hb_server_take(self._h, int(request_id), _ptr(out["closeness"]), _ptr(out["harmonic"]),
                                     _ptr(out["lin"]), _ptr(out["reachable"])))
        return out

    def stats(self) -> dict:
        c, it, a = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        busy, clock = ctypes.c_double(), ctypes.c_double()
        _check(load().hb_server_stats(self._h, ctypes.byref(c), ctypes.byref(it), ctypes.byref(a),
                                      ctypes.byref(busy), ctypes.byref(clock)))
        return {"completed": c.value, "iterations": it.value, "arcs": a.value, "busy_s": busy.value,
                "clock_s": clock.value}

    def close(self):
        if getattr(self, "_h", None):
            load().hb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- convenience --

class HyperBall:
    """One graph's HyperBall state on the GPU (owns an hb_graph handle).

    ``offsets``/``targets`` describe the scanned graph S in CSR form (torch
    tensors on the GPU or the CPU, or numpy arrays); pass ``transpose=True``
    to hand over G and scan G^T (the in-centralities of Sec. 3).
    """

    def __init__(self, offsets, targets, log2m: int = 4, seed: int = 42, n: int | None = None,
                 **opts):
        self.n = int(offsets.shape[0] - 1) if n is None else int(n)
        self.m = int(targets.shape[0])
        self.log2m = log2m
        self.p = 1 << log2m
        self.options = make_options(**opts)
        self._h = hb_create(offsets, targets, self.n, self.m, log2m, seed, self.options)

    @classmethod
    def from_graph(cls, g, **kw):
        return cls(g.offsets, g.targets, n=g.n, **kw)

    @classmethod
    def runs(cls, offsets, targets, log2m: int, seeds, n: int | None = None, **opts) -> "HyperBall":
        """Several runs of one graph in one handle (hb_create_runs): run r
        uses seeds[r]; rows hold len(seeds) counters of 2^log2m registers."""
        if offsets.dtype in (torch.int32, np.int32):   # the entry point takes int64 offsets
            offsets = offsets.to(torch.int64) if isinstance(offsets, torch.Tensor) else offsets.astype(np.int64)
        self = cls.__new__(cls)
        self.n = int(offsets.shape[0] - 1) if n is None else int(n)
        self.m = int(targets.shape[0])
        self.log2m = log2m
        self.nruns = len(seeds)
        self.p = self.nruns << log2m
        self.options = make_options(**opts)
        self._h = _vp()
        arr = (ctypes.c_uint64 * self.nruns)(*[int(x) & (2**64 - 1) for x in seeds])
        _check(load().hb_create_runs(_ptr(offsets), _ptr(targets) if self.m else None, self.n, self.m,
                                     int(log2m), self.nruns, arr, ctypes.byref(self.options),
                                     ctypes.byref(self._h)))
        return self

    def run_steps(self) -> list:
        arr = (ctypes.c_int32 * self.nruns)()
        _check(load().hb_get_run_steps(self._h, arr))
        return list(arr)

    def run_centralities(self, r: int, device="cuda") -> dict:
        out = {k: self._out(self.n, torch.float64, device)
               for k in ("closeness", "harmonic", "lin", "reachable")}
        _check(load().hb_get_run_centralities(self._h, int(r), _ptr(out["closeness"]), _ptr(out["harmonic"]),
                                              _ptr(out["lin"]), _ptr(out["reachable"])))
        return out

    def run_accumulators(self, r: int, device="cuda"):
        sumd = self._out(self.n, torch.float64, device)
        harm = self._out(self.n, torch.float64, device)
        _check(load().hb_get_run_accumulators(self._h, int(r), _ptr(sumd), _ptr(harm)))
        return sumd, harm

    def run_discounted(self, r: int, device="cuda") -> torch.Tensor:
        out = self._out(self.n, torch.float64, device)
        _check(load().hb_get_run_discounted(self._h, int(r), _ptr(out)))
        return out

    def run_stats(self, which, device="cuda"):
        """Per-node mean and sample standard deviation over the runs of one
        centrality ("closeness", "harmonic", "lin", "reachable") or of the
        discounted accumulator ("discounted")."""
        names = ("closeness", "harmonic", "lin", "reachable", "discounted")
        w = names.index(which) if isinstance(which, str) else int(which)
        mean = self._out(self.n, torch.float64, device)
        sd = self._out(self.n, torch.float64, device)
        _check(load().hb_get_run_stats(self._h, w, _ptr(mean), _ptr(sd)))
        return mean, sd

    def step(self) -> int:
        return hb_step(self._h)

    def run(self) -> int:
        return hb_run_to_fixpoint(self._h)

    def info(self) -> dict:
        return hb_get_info(self._h)

    def reset(self, seed: int):
        hb_reset(self._h, seed)

    def tune(self) -> int:
        return hb_tune(self._h)

    def set_class_sizing(self, arcs_per_slot: int):
        _check(load().hb_set_class_sizing(self._h, int(arcs_per_slot)))

    def set_hot_nodes(self, hot_nodes: int, passes: int = 1):
        """Hot range of the gather (0: none): one pass with L2 priorities
        (passes=1) or the two-phase gather (passes=2); results do not
        depend on it."""
        _check(load().hb_set_hot_nodes(self._h, int(hot_nodes), int(passes)))

    def set_frontier_switch(self, push_frac: float):
        """HB_FRONTIER_AUTO pushes when the arcs to push are at most
        push_frac * m; results do not depend on it."""
        _check(load().hb_set_frontier_switch(self._h, float(push_frac)))

    def set_weights(self, weights=None):
        """Node weights by replicas (Sec. 6); restarts the computation."""
        if weights is not None and not isinstance(weights, torch.Tensor):
            weights = np.ascontiguousarray(weights, dtype=np.int64)
        hb_set_weights(self._h, weights)

    def set_discount(self, f=None):
        """Discount table f(1), f(2), ... (Sec. 7); restarts the computation."""
        if f is not None and not isinstance(f, torch.Tensor):
            f = np.ascontiguousarray(f, dtype=np.float64)
        hb_set_discount(self._h, f)

    def neighbourhood(self) -> np.ndarray:
        """The neighbourhood function N(0), ..., N(t) of the run so far."""
        return hb_get_neighbourhood(self._h)

    def discounted(self, device="cuda") -> torch.Tensor:
        out = self._out(self.n, torch.float64, device)
        hb_get_discounted(self._h, out)
        return out

    def _out(self, shape, dtype, device):
        return torch.empty(shape, dtype=dtype, device=device)

    def centralities(self, device="cuda") -> dict:
        out = {k: self._out(self.n, torch.float64, device)
               for k in ("closeness", "harmonic", "lin", "reachable")}
        hb_get_centralities(self._h, out["closeness"], out["harmonic"], out["lin"], out["reachable"])
        return out

    def accumulators(self, device="cuda"):
        sumd = self._out(self.n, torch.float64, device)
        harm = self._out(self.n, torch.float64, device)
        hb_get_accumulators(self._h, sumd, harm)
        return sumd, harm

    def registers(self, device="cuda") -> torch.Tensor:
        out = self._out((self.n, self.p), torch.uint8, device)
        hb_get_registers(self._h, out)
        return out

    def frontier(self, device="cuda"):
        ch = self._out(self.n, torch.uint8, device)
        mk = self._out(self.n, torch.uint8, device)
        hb_get_frontier(self._h, ch, mk)
        return ch, mk

    def save(self, path: str):
        hb_save(self._h, path)

    def close(self):
        if getattr(self, "_h", None):
            hb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
