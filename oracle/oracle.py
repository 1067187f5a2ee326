"""Python access to the FP64 CPU oracle (osp_oracle.c) plus the dense closed form.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the product path never imports it. It shares
nothing with the CUDA engine.

Functions follow the paper (Yoon, Jin, Kang, WWW 2018):
  * ``dense_rwr``      Eq. 1 solved directly, r = c (I - (1-c) A~^T)^-1 e_s.
  * ``cpi``            Sec. 2.2, cumulative power iteration.
  * ``offset``         Sec. 3.1 / Algorithm 1, q_offset = (1-c)(B~^T - A~^T) r_old.
  * ``osp``            Algorithm 1 (OSP; OSP-T is the same call with a larger eps).
  * ``normalize``      Sec. 3.4.2 / Theorem 5, dead-end handling r / ||r||_1.
  * ``topk``           ranking by (score descending, id ascending).
  * ``residual_l1``    ||c e_s - (I - (1-c) B~^T) r||_1, an a-posteriori bound
                       on ||r - r*||_1 times c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "osp_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE arithmetic: no FMA contraction)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("q_l1", C.c_double), ("last_l1", C.c_double),
                ("visited_edges", C.c_int64)]

    def as_dict(self):
        return {"iterations": self.iterations, "q_l1": self.q_l1, "last_l1": self.last_l1,
                "visited_edges": self.visited_edges}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            i64, i32, dbl = C.c_int64, C.c_int32, C.c_double
            L.orc_graph_new.restype = P
            L.orc_graph_new.argtypes = [i64, i64, P, P, C.c_int]
            L.orc_graph_free.argtypes = [P]
            L.orc_graph_n.restype = i64
            L.orc_graph_n.argtypes = [P]
            L.orc_graph_m.restype = i64
            L.orc_graph_m.argtypes = [P]
            L.orc_graph_validate.restype = i64
            L.orc_graph_validate.argtypes = [P, P, i64, P, i32]
            L.orc_graph_apply.restype = i64
            L.orc_graph_apply.argtypes = [P, P, i64, P, i32]
            L.orc_graph_csr.argtypes = [P, P, P]
            L.orc_graph_csc.argtypes = [P, P, P]
            L.orc_graph_dead.argtypes = [P, P]
            L.orc_propagate.restype = C.c_int
            L.orc_propagate.argtypes = [i64, P, P, P, dbl, dbl, i32, i32, P, P, P]
            L.orc_cpi.restype = C.c_int
            L.orc_cpi.argtypes = [i64, P, P, i32, dbl, dbl, i32, i32, P, P, P]
            L.orc_offset.argtypes = [i64, P, P, i64, P, P, P, dbl, P]
            L.orc_osp.restype = C.c_int
            L.orc_osp.argtypes = [i64, P, P, i64, P, P, P, dbl, dbl, i32, i32, P, P, P, P]
            L.orc_residual_l1.restype = dbl
            L.orc_residual_l1.argtypes = [i64, P, P, i32, dbl, P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _csr(row_ptr, col):
    return (np.ascontiguousarray(row_ptr, np.int64), np.ascontiguousarray(col, np.int32))


class Graph:
    """The edge set of a simple directed graph, updated by batches applied in order."""

    def __init__(self, n, src, dst, undirected=False):
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        self._h = lib().orc_graph_new(int(n), int(src.size), _p(src), _p(dst), int(undirected))
        if not self._h:
            raise ValueError("bad edge list")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_graph_free(h)
            self._h = None

    @property
    def n(self):
        return int(lib().orc_graph_n(self._h))

    @property
    def m(self):
        return int(lib().orc_graph_m(self._h))

    def validate(self, ops, protect=()):
        ops = np.ascontiguousarray(ops)
        pr = np.ascontiguousarray(np.asarray(protect, np.int32))
        return int(lib().orc_graph_validate(self._h, _p(ops), int(ops.size), _p(pr), int(pr.size)))

    def apply(self, ops, protect=()):
        """Returns -1 on success, else the index of the first invalid op (graph unchanged)."""
        ops = np.ascontiguousarray(ops)
        pr = np.ascontiguousarray(np.asarray(protect, np.int32))
        bad = int(lib().orc_graph_apply(self._h, _p(ops), int(ops.size), _p(pr), int(pr.size)))
        if bad == -2:
            raise MemoryError("oracle out of memory")
        return bad

    def csr(self):
        rp = np.empty(self.n + 1, np.int64)
        col = np.empty(max(self.m, 1), np.int32)
        lib().orc_graph_csr(self._h, _p(rp), _p(col))
        return rp, col[: self.m]

    def csc(self):
        cp = np.empty(self.n + 1, np.int64)
        row = np.empty(max(self.m, 1), np.int32)
        lib().orc_graph_csc(self._h, _p(cp), _p(row))
        return cp, row[: self.m]

    def dead(self):
        out = np.empty(self.n, np.uint8)
        lib().orc_graph_dead(self._h, _p(out))
        return out


def propagate(row_ptr, col, x0, c, eps, force_iters=0, max_iter=100000):
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.size - 1
    x0 = np.ascontiguousarray(x0, np.float64)
    r = np.empty(n, np.float64)
    hist = np.zeros(max_iter + 1, np.float64)
    st = _Stats()
    rc = lib().orc_propagate(n, _p(row_ptr), _p(col), _p(x0), float(c), float(eps),
                             int(force_iters), int(max_iter), _p(r), _p(hist), C.byref(st))
    if rc < 0:
        raise MemoryError
    d = st.as_dict()
    d["converged"] = rc == 0
    return r, d, hist[: st.iterations + 1]


def cpi(row_ptr, col, seed, c, eps, force_iters=0, max_iter=100000):
    """CPI from seed (Sec. 2.2). Returns (r, stats, ||x(i)||_1 history)."""
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.size - 1
    r = np.empty(n, np.float64)
    hist = np.zeros(max_iter + 1, np.float64)
    st = _Stats()
    rc = lib().orc_cpi(n, _p(row_ptr), _p(col), int(seed), float(c), float(eps), int(force_iters),
                       int(max_iter), _p(r), _p(hist), C.byref(st))
    if rc < 0:
        raise MemoryError
    d = st.as_dict()
    d["converged"] = rc == 0
    return r, d, hist[: st.iterations + 1]


def offset(old_csr, new_csr, r_old, c):
    rpo, co = _csr(*old_csr)
    rpn, cn = _csr(*new_csr)
    r_old = np.ascontiguousarray(r_old, np.float64)
    q = np.empty(rpn.size - 1, np.float64)
    lib().orc_offset(rpo.size - 1, _p(rpo), _p(co), rpn.size - 1, _p(rpn), _p(cn), _p(r_old),
                     float(c), _p(q))
    return q


def osp(old_csr, new_csr, r_old, c, eps, force_iters=0, max_iter=100000):
    """Algorithm 1. Returns (r_new, q_offset, stats, ||x(i)||_1 history)."""
    rpo, co = _csr(*old_csr)
    rpn, cn = _csr(*new_csr)
    r_old = np.ascontiguousarray(r_old, np.float64)
    nn = rpn.size - 1
    r_new = np.empty(nn, np.float64)
    q = np.empty(nn, np.float64)
    hist = np.zeros(max_iter + 1, np.float64)
    st = _Stats()
    rc = lib().orc_osp(rpo.size - 1, _p(rpo), _p(co), nn, _p(rpn), _p(cn), _p(r_old), float(c),
                       float(eps), int(force_iters), int(max_iter), _p(r_new), _p(q), _p(hist),
                       C.byref(st))
    if rc < 0:
        raise MemoryError
    d = st.as_dict()
    d["converged"] = rc == 0
    return r_new, q, d, hist[: st.iterations + 1]


def residual_l1(row_ptr, col, seed, c, r):
    row_ptr, col = _csr(row_ptr, col)
    r = np.ascontiguousarray(r, np.float64)
    return float(lib().orc_residual_l1(row_ptr.size - 1, _p(row_ptr), _p(col), int(seed), float(c),
                                       _p(r)))


def normalize(r):
    """Dead-end handling (Sec. 3.4.2, Theorem 5): r_final = r_temp / ||r_temp||_1."""
    r = np.asarray(r, np.float64)
    return r / np.abs(r).sum()


def topk(r, k):
    """The k largest scores, ordered by (score descending, id ascending)."""
    r = np.asarray(r, np.float64)
    order = np.lexsort((np.arange(r.size), -r))[:k]
    return order.astype(np.int32), r[order]


def dense_matrix(n, src, dst):
    """Row-normalised adjacency A~ (Eq. 1) as a dense n x n array; dead-end rows are zero.
    Duplicate pairs count once."""
    A = np.zeros((n, n), np.float64)
    A[np.asarray(src), np.asarray(dst)] = 1.0
    d = A.sum(axis=1)
    nz = d > 0
    A[nz] /= d[nz][:, None]
    return A


def dense_rwr_q(n, src, dst, q, c):
    """Eq. 1 with a general restart vector q: r = c (I - (1-c) A~^T)^-1 q (dense LU)."""
    A = dense_matrix(n, src, dst)
    return np.linalg.solve(np.eye(n) - (1.0 - c) * A.T, c * np.asarray(q, np.float64))


def dense_rwr(n, src, dst, seed, c):
    """Eq. 1 solved directly: r = c (I - (1-c) A~^T)^-1 e_s, by LU with partial pivoting."""
    A = dense_matrix(n, src, dst)
    q = np.zeros(n)
    q[seed] = 1.0
    return np.linalg.solve(np.eye(n) - (1.0 - c) * A.T, c * q)
