"""ctypes binding of the C ABI in include/osp.h (argument marshalling only).

Every function here forwards to the same-named entry point of the in-tree
library ``_build/libosp_gb300.so``; all arithmetic runs in its CUDA kernels.
Loading fails loudly if the library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# OSP_LIBRARY selects another build of the same ABI (e.g. the bounds-checked one).
LIB_PATH = os.environ.get("OSP_LIBRARY") or os.path.join(HERE, "_build", "libosp_gb300.so")

OSP_OK, OSP_EINVAL, OSP_ENOMEM, OSP_ECUDA, OSP_ETIMEOUT, OSP_ENOCONV, OSP_ESTATE, OSP_ENOTSUP = (
    0, -1, -2, -3, -4, -5, -6, -7)
OSP_PREC_FP64, OSP_PREC_FP32_ACC64, OSP_PREC_BF16_ACC64 = 0, 1, 2
SEED_GATHER_REGISTERS, SEED_GATHER_BULK = 1, 2  # osp_options.seed_gather
UPDATE_DTYPE = np.dtype([("u", "<i4"), ("v", "<i4"), ("op", "<i4")])

TOPK_NOALLOC_MAX_N = 33554431  # OSP_TOPK_NOALLOC_MAX_N
MAX_APPLY_OPS = 1 << 22        # ops one apply call accepts (in sub-batches of osp_max_batch())

EXPORTED = [
    "osp_default_options", "osp_create", "osp_destroy", "osp_load_graph", "osp_set_seeds",
    "osp_init_scores", "osp_apply_updates", "osp_apply_updates_device", "osp_max_batch",
    "osp_query", "osp_query_device", "osp_topk", "osp_export_graph", "osp_get_size",
    "osp_get_l1_history", "osp_get_step_times", "osp_set_fixed_iterations", "osp_last_error",
    "osp_status_string", "osp_topk_noalloc", "osp_get_seed_stats",
    "osp_set_seed_iterations", "osp_get_schedule", "osp_query_slots", "osp_topk_async",
    "osp_topk_async_many", "osp_topk_wait", "osp_selftest_wait", "osp_num_nodes", "osp_get_residual_bounds",
    "osp_device_bytes",
]


class osp_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("stream", C.c_void_p),
                ("max_nodes", C.c_int64), ("push_alpha", C.c_double), ("push_beta", C.c_double),
                ("max_iter", C.c_int32), ("node_order", C.c_int32), ("use_graphs", C.c_int32),
                ("autotune", C.c_int32), ("seed_gather", C.c_int32),
                ("seed_group", C.c_int32), ("deterministic", C.c_int32),
                ("l2_hot_bytes", C.c_int64), ("hbm_budget_bytes", C.c_int64)]


class osp_batch_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("push_iterations", C.c_int32),
                ("qoff_l1", C.c_double), ("last_x_l1", C.c_double),
                ("visited_edges", C.c_int64), ("n_nodes", C.c_int64), ("m_edges", C.c_int64),
                ("net_inserts", C.c_int64), ("net_deletes", C.c_int64),
                ("changed_rows", C.c_int64), ("bad_op", C.c_int64),
                ("push_frontier", C.c_int64), ("push_reached", C.c_int64),
                ("ms_update", C.c_float), ("ms_propagate", C.c_float),
                ("kernel_launches", C.c_int32), ("reserved", C.c_int32),
                ("pull_dst_nodes", C.c_int64), ("pull_src_nodes", C.c_int64),
                ("residual_bound", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OspError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status_name(status), msg))
        self.status = status


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load the engine library. Raises if it is missing (build it first)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError("CUDA engine library not built: %s (run __graft_entry__.build())" % path)
        L = C.CDLL(path)
        P, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "osp_default_options": (None, [P]),
            "osp_create": (C.c_int, [P, P]),
            "osp_destroy": (None, [P]),
            "osp_load_graph": (C.c_int, [P, i64, i64, P, P, C.c_int]),
            "osp_set_seeds": (C.c_int, [P, P, i32, dbl]),
            "osp_init_scores": (C.c_int, [P, dbl, P]),
            "osp_apply_updates": (C.c_int, [P, P, i64, dbl, P]),
            "osp_apply_updates_device": (C.c_int, [P, P, i64, dbl, P]),
            "osp_max_batch": (i64, []),
            "osp_query": (C.c_int, [P, i32, C.c_int, P]),
            "osp_query_device": (C.c_int, [P, i32, C.c_int, P]),
            "osp_topk": (C.c_int, [P, i32, i32, C.c_int, P, P, P]),
            "osp_export_graph": (C.c_int, [P, C.c_int, P, P]),
            "osp_get_size": (C.c_int, [P, P, P]),
            "osp_get_l1_history": (C.c_int, [P, P, i32, P]),
            "osp_get_step_times": (C.c_int, [P, P, i32, P]),
            "osp_set_fixed_iterations": (C.c_int, [P, i32]),
            "osp_last_error": (C.c_char_p, [P]),
            "osp_status_string": (C.c_char_p, [C.c_int]),
            "osp_topk_noalloc": (C.c_int, [P, i64, i32, C.c_int, P, P, P, P]),
            "osp_get_seed_stats": (C.c_int, [P, P, P, P, i32, P]),
            "osp_set_seed_iterations": (C.c_int, [P, P, i32]),
            "osp_get_schedule": (C.c_int, [P, P]),
            "osp_query_slots": (C.c_int, [P, i32]),
            "osp_topk_async": (C.c_int, [P, i32, i32, i32, C.c_int]),
            "osp_topk_async_many": (C.c_int, [P, P, P, i32, i32, C.c_int]),
            "osp_topk_wait": (C.c_int, [P, i32, P, P, P]),
            "osp_selftest_wait": (C.c_int, [i32, i32, i32]),
            "osp_num_nodes": (i64, [P]),
            "osp_get_residual_bounds": (C.c_int, [P, P, i32, P]),
            "osp_device_bytes": (i64, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def status_name(s: int) -> str:
    names = {0: "OSP_OK", -1: "OSP_EINVAL", -2: "OSP_ENOMEM", -3: "OSP_ECUDA", -4: "OSP_ETIMEOUT",
             -5: "OSP_ENOCONV", -6: "OSP_ESTATE", -7: "OSP_ENOTSUP"}
    return names.get(s, "OSP_%d" % s)


def _ptr(a) -> C.c_void_p:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        return C.c_void_p(a.data_ptr())
    if isinstance(a, int):
        return C.c_void_p(a)
    return a.ctypes.data_as(C.c_void_p)


def selftest_wait(which, lose, device=0):
    """osp_selftest_wait: run one bounded wait of the persistent kernels
    (which 0 = grid barrier, 1 = staged-row mbarrier), made to run out when
    lose is true. Returns the status code (OSP_OK or OSP_ETIMEOUT)."""
    return load_library().osp_selftest_wait(int(device), int(which), int(bool(lose)))


def topk_noalloc(scores_device, n, k, ids_device, out_scores_device, k_out_device,
                 normalize=False, stream=None):
    """osp_topk_noalloc on device buffers (tensors or raw pointers) of the
    current device; asynchronous on `stream` (a raw cudaStream_t or None)."""
    L = load_library()
    s = L.osp_topk_noalloc(_ptr(scores_device), int(n), int(k), int(bool(normalize)),
                           _ptr(ids_device), _ptr(out_scores_device), _ptr(k_out_device),
                           _ptr(stream) if stream is not None else None)
    if s == OSP_EINVAL:
        raise OspError(s, "osp_topk_noalloc: n must lie in [0, %d], k in [1, 4096], every "
                          "pointer non-null, device ordinal <= 63" % TOPK_NOALLOC_MAX_N)
    if s != 0:
        raise OspError(s, "osp_topk_noalloc: CUDA call or launch failed")


class Engine:
    """One engine context (osp_ctx). Methods mirror the C ABI one to one."""

    def __init__(self, precision=OSP_PREC_FP32_ACC64, device=0, stream=None, max_nodes=0,
                 push_alpha=0.0, push_beta=0.0, max_iter=0, node_order=0, use_graphs=False,
                 autotune=False, seed_gather=0, seed_group=0, deterministic=False,
                 l2_hot_bytes=0, hbm_budget_bytes=0):
        L = load_library()
        opt = osp_options()
        L.osp_default_options(C.byref(opt))
        opt.precision = precision
        opt.device = device
        opt.stream = stream
        opt.max_nodes = max_nodes
        opt.push_alpha = push_alpha
        opt.push_beta = push_beta
        opt.max_iter = max_iter
        opt.node_order = node_order
        opt.use_graphs = int(bool(use_graphs))
        opt.autotune = int(bool(autotune))
        opt.seed_gather = int(seed_gather)
        opt.seed_group = int(seed_group)
        opt.deterministic = int(bool(deterministic))
        opt.l2_hot_bytes = int(l2_hot_bytes)
        opt.hbm_budget_bytes = int(hbm_budget_bytes)
        h = C.c_void_p()
        s = L.osp_create(C.byref(h), C.byref(opt))
        if s != OSP_OK:
            raise OspError(s, "osp_create failed")
        self._h = h
        self._L = L
        self.last_status = OSP_OK

    def close(self):
        if getattr(self, "_h", None):
            self._L.osp_destroy(self._h)
            self._h = None

    __del__ = close

    def _check(self, s, allow=()):
        self.last_status = s
        if s != OSP_OK and s not in allow:
            raise OspError(s, self.last_error())
        return s

    def last_error(self) -> str:
        return self._L.osp_last_error(self._h).decode()

    def load_graph(self, n, src, dst, undirected=False):
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        return self._check(self._L.osp_load_graph(self._h, int(n), int(src.size), _ptr(src),
                                                  _ptr(dst), int(bool(undirected))))

    def set_seeds(self, seeds, c):
        seeds = np.ascontiguousarray(np.atleast_1d(seeds), np.int32)
        return self._check(self._L.osp_set_seeds(self._h, _ptr(seeds), int(seeds.size), float(c)))

    def init_scores(self, eps, allow=()):
        st = osp_batch_stats()
        self._check(self._L.osp_init_scores(self._h, float(eps), C.byref(st)), allow)
        return st.as_dict()

    def apply_updates(self, ops, eps, allow=()):
        ops = np.ascontiguousarray(ops, UPDATE_DTYPE)
        st = osp_batch_stats()
        self._check(self._L.osp_apply_updates(self._h, _ptr(ops), int(ops.size), float(eps),
                                              C.byref(st)), allow)
        return st.as_dict()

    def apply_updates_device(self, ops_device, count, eps, stats=True, allow=()):
        """ops_device: a CUDA tensor (or raw device pointer) holding ``count`` updates."""
        st = osp_batch_stats() if stats else None
        self._check(self._L.osp_apply_updates_device(self._h, _ptr(ops_device), int(count),
                                                     float(eps),
                                                     C.byref(st) if st is not None else None),
                    allow)
        return st.as_dict() if st is not None else None

    def query(self, seed_idx=0, normalize=False, out=None):
        """Scores in caller order. out: a float64 host array of at least n
        entries to write them to (page-locked memory copies fastest); the
        first n entries are returned."""
        n, _ = self.get_size()
        if out is None:
            out = np.empty(n, np.float64)
        elif (not isinstance(out, np.ndarray) or out.dtype != np.float64 or out.ndim != 1
              or not out.flags.c_contiguous or out.size < n):
            raise ValueError("out must be a contiguous float64 array of at least %d entries" % n)
        self._check(self._L.osp_query(self._h, int(seed_idx), int(bool(normalize)), _ptr(out)))
        return out[:n]

    def query_device(self, out_device, seed_idx=0, normalize=False):
        return self._check(self._L.osp_query_device(self._h, int(seed_idx), int(bool(normalize)),
                                                    _ptr(out_device)))

    def topk(self, k, seed_idx=0, normalize=False):
        ids = np.empty(k, np.int32)
        sc = np.empty(k, np.float64)
        got = C.c_int32(0)
        self._check(self._L.osp_topk(self._h, int(seed_idx), int(k), int(bool(normalize)),
                                     _ptr(ids), _ptr(sc), C.byref(got)))
        return ids[: got.value], sc[: got.value]

    def export_graph(self, direction=0):
        n, m = self.get_size()
        ptr = np.empty(n + 1, np.int64)
        idx = np.empty(max(m, 1), np.int32)
        self._check(self._L.osp_export_graph(self._h, int(direction), _ptr(ptr), _ptr(idx)))
        return ptr, idx[:m]

    def get_size(self):
        n = C.c_int64()
        m = C.c_int64()
        self._check(self._L.osp_get_size(self._h, C.byref(n), C.byref(m)))
        return int(n.value), int(m.value)

    def get_l1_history(self, cap=4096):
        out = np.empty(cap, np.float64)
        cnt = C.c_int32(0)
        self._check(self._L.osp_get_l1_history(self._h, _ptr(out), int(cap), C.byref(cnt)))
        return out[: cnt.value]

    def set_seed_iterations(self, k=None):
        """Per-seed step counts for the following calls (None clears)."""
        if k is None:
            return self._check(self._L.osp_set_seed_iterations(self._h, None, 0))
        k = np.ascontiguousarray(k, np.int32)
        return self._check(self._L.osp_set_seed_iterations(self._h, _ptr(k), int(k.size)))

    def query_slots(self, nslots):
        return self._check(self._L.osp_query_slots(self._h, int(nslots)))

    def topk_async(self, slot, k, seed_idx=0, normalize=False):
        return self._check(self._L.osp_topk_async(self._h, int(slot), int(seed_idx), int(k),
                                                  int(bool(normalize))))

    def topk_async_many(self, slots, seed_idx, k, normalize=False):
        """One launch sequence for the top-k of several seeds, seed_idx[i] in
        slots[i] (at most 32); collect each slot with topk_wait."""
        sl = np.ascontiguousarray(slots, np.int32)
        sd = np.ascontiguousarray(seed_idx, np.int32)
        if sl.size != sd.size:
            raise ValueError("one slot per seed")
        return self._check(self._L.osp_topk_async_many(self._h, _ptr(sl), _ptr(sd), int(sl.size),
                                                       int(k), int(bool(normalize))))

    def topk_wait(self, slot, k_max=4096):
        ids = np.empty(k_max, np.int32)
        sc = np.empty(k_max, np.float64)
        got = C.c_int32(0)
        self._check(self._L.osp_topk_wait(self._h, int(slot), _ptr(ids), _ptr(sc), C.byref(got)))
        return ids[: got.value], sc[: got.value]

    def get_schedule(self):
        """(task items, long-list threshold, piece length, node items) in force."""
        out = np.zeros(4, np.int32)
        self._check(self._L.osp_get_schedule(self._h, _ptr(out)))
        return tuple(int(x) for x in out)

    def get_seed_stats(self, cap=256):
        """Per seed of the last call: (steps run, ||x(0)||_1, ||x(k)||_1 at its stop)."""
        it = np.empty(cap, np.int32)
        q = np.empty(cap, np.float64)
        last = np.empty(cap, np.float64)
        cnt = C.c_int32(0)
        self._check(self._L.osp_get_seed_stats(self._h, _ptr(it), _ptr(q), _ptr(last), int(cap),
                                               C.byref(cnt)))
        k = cnt.value
        return it[:k], q[:k], last[:k]

    def num_nodes(self):
        return int(self._L.osp_num_nodes(self._h))

    def device_bytes(self):
        return int(self._L.osp_device_bytes(self._h))

    def get_residual_bounds(self, cap=256):
        """Per seed: the bound on ||rho||_1 of the stored scores (see osp_batch_stats)."""
        out = np.empty(cap, np.float64)
        cnt = C.c_int32(0)
        self._check(self._L.osp_get_residual_bounds(self._h, _ptr(out), int(cap), C.byref(cnt)))
        return out[: cnt.value]

    def get_step_times(self, cap=4096):
        """Microseconds of the x(0) pass and of each propagation step of the last call."""
        out = np.empty(cap, np.float64)
        cnt = C.c_int32(0)
        self._check(self._L.osp_get_step_times(self._h, _ptr(out), int(cap), C.byref(cnt)))
        return out[: cnt.value]

    def set_fixed_iterations(self, k):
        return self._check(self._L.osp_set_fixed_iterations(self._h, int(k)))

    @staticmethod
    def max_batch():
        return int(load_library().osp_max_batch())
