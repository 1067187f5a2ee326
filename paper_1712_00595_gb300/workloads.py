"""Seeded synthetic workloads: graphs, update streams and seed choice.

This module only draws inputs. It holds none of the RWR / OSP arithmetic, so
both the CUDA path and the CPU oracle can consume what it produces without
sharing any of the method's code.

The paper measures on SNAP graphs (WikiLink, Orkut, LiveJournal, Berkstan,
DBLP, Slashdot; Table 3). Those datasets are not available here; the
generators below produce power-law directed graphs of the same shape
(R-MAT, Chung-Lu) and uniform Erdos-Renyi graphs for small cases. Update
streams follow Section 4.2/4.3: uniformly random edge insertions and
deletions of existing edges.

Every generator takes an integer ``seed`` and uses numpy's counter-based
Philox bit generator, so a (generator, seed) pair always yields the same
input.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

# One update operation, laid out exactly as ``osp_update`` in include/osp.h.
UPDATE_DTYPE = np.dtype([("u", "<i4"), ("v", "<i4"), ("op", "<i4")])
OP_INSERT_EDGE = 0
OP_DELETE_EDGE = 1
OP_ADD_NODE = 2
OP_DELETE_NODE = 3
OP_ZERO_ROW = 4

BASE_SEED = 20180423


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def edge_keys(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    return (src.astype(np.uint64) << np.uint64(32)) | dst.astype(np.uint64)


def split_keys(keys: np.ndarray):
    src = (keys >> np.uint64(32)).astype(np.int32)
    dst = (keys & np.uint64(0xFFFFFFFF)).astype(np.int32)
    return src, dst


def _first_unique(keys: np.ndarray) -> np.ndarray:
    """Unique keys, kept in order of first appearance."""
    _, idx = np.unique(keys, return_index=True)
    return keys[np.sort(idx)]


def _fill_unique(draw, m: int, chunk: int) -> np.ndarray:
    """Draw candidate edge keys until ``m`` distinct ones exist (redraw duplicates)."""
    have = np.empty(0, np.uint64)
    while have.size < m:
        need = m - have.size
        cand = draw(max(int(need * 1.05) + 64, min(chunk, 4 * need + 64)))
        have = _first_unique(np.concatenate([have, cand]))
    return np.sort(have[:m])


# --------------------------------------------------------------------------
# Native sampler (gen.c): counter-based draws, sort and de-duplication of
# edge keys, multi-threaded; it draws inputs only.
# --------------------------------------------------------------------------
_GEN_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gen.c")
_GEN_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libgen.so")
_gen_lock = threading.Lock()
_gen_lib = None


def build_gen(force: bool = False) -> str:
    """Compile gen.c with gcc into the package's _build folder."""
    os.makedirs(os.path.dirname(_GEN_LIB), exist_ok=True)
    if force or not os.path.exists(_GEN_LIB) or os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", tmp,
                               _GEN_SRC])
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _gen():
    global _gen_lib
    with _gen_lock:
        if _gen_lib is None:
            L = C.CDLL(build_gen())
            P, i64, i32, u64, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_double
            L.gen_rmat.argtypes = [u64, i32, dbl, dbl, dbl, i64, i64, P, P, i32, i32]
            L.gen_chunglu.argtypes = [u64, P, i64, i64, i64, P, P, i32, i32]
            L.keys_sort_unique.restype = i64
            L.keys_sort_unique.argtypes = [P, i64, i32, i32]
            L.keys_merge_unique.restype = i64
            L.keys_merge_unique.argtypes = [P, i64, P, i64, P]
            L.keys_apply.restype = i64
            L.keys_apply.argtypes = [P, i64, P, i64, P, i64, P]
            _gen_lib = L
    return _gen_lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


THREADS = 0  # native sampler threads (0: one per core, at most 32); results do not depend on it


def _nthreads() -> int:
    return THREADS if THREADS > 0 else max(1, min(32, os.cpu_count() or 1))


def _key_bits(n: int) -> int:
    return 32 + max(1, int(n - 1).bit_length())


def sort_unique_keys(keys: np.ndarray, n: int) -> np.ndarray:
    """Distinct keys of ``keys`` ascending (rejected draws dropped); ids below n."""
    keys = np.ascontiguousarray(keys, np.uint64).copy()
    k = _gen().keys_sort_unique(_ptr(keys), keys.size, _key_bits(n), _nthreads())
    if k < 0:
        raise MemoryError("key sort")
    return keys[:k]


def _unique_draws(draw, m: int, n: int) -> np.ndarray:
    """The first ``m`` distinct keys of a counter-based sampler, ascending.

    draw(start, count) returns draws start .. start + count - 1 as keys
    (rejections as all-ones keys). Rounds draw the missing count (plus a
    margin) until m distinct keys exist; a surplus from the last round is
    thinned at evenly spaced positions of the sorted set."""
    have = np.empty(0, np.uint64)
    start, k = 0, m + m // 16 + 1024
    while True:
        cand = sort_unique_keys(draw(start, k), n)
        start += k
        if have.size == 0:
            have = cand
        else:
            out = np.empty(have.size + cand.size, np.uint64)
            got = _gen().keys_merge_unique(_ptr(have), have.size, _ptr(cand), cand.size, _ptr(out))
            have = out[:got]
        if have.size >= m:
            break
        k = 2 * (m - have.size) + 1024
    extra = have.size - m
    if extra > 0:
        pos = ((np.arange(extra, dtype=np.float64) + 0.5) * (have.size / extra)).astype(np.int64)
        have = np.delete(have, pos)
    return have


# --------------------------------------------------------------------------
# Graphs
# --------------------------------------------------------------------------
def er_graph(n: int, m: int, seed: int):
    """Directed Erdos-Renyi graph: ``m`` distinct uniform (u, v) pairs, u != v."""
    rng = rng_for(seed)

    def draw(k):
        u = rng.integers(0, n, k, dtype=np.int64)
        v = rng.integers(0, n, k, dtype=np.int64)
        ok = u != v
        return edge_keys(u[ok], v[ok])

    keys = _fill_unique(draw, m, 1 << 22)
    return split_keys(keys)


class RMat:
    """R-MAT sampler (a, b, c, d quadrant probabilities) over 2**scale nodes.

    Vertex ids are relabelled by a seeded random permutation so that hubs are
    not clustered at small ids; the same permutation is used for the edges of
    the initial graph and for later insertions drawn from the same sampler.
    Draws come from the counter-based native sampler (gen.c): the graph's
    candidates and the stream samples use two streams keyed from ``seed``.
    """

    def __init__(self, scale: int, a=0.57, b=0.19, c=0.19, d=0.05, seed: int = BASE_SEED,
                 permute: bool = True):
        self.scale = scale
        self.n = 1 << scale
        self.p = (a, b, c, d)
        self.rng = rng_for(seed)
        self.perm = self.rng.permutation(self.n).astype(np.int64) if permute else None
        self.key_graph, self.key_sample = (int(x) for x in self.rng.integers(0, 1 << 63, 2))
        self.drawn = 0

    def _draw(self, key, start, k, keep_loops):
        a, b, c, _ = self.p
        out = np.empty(k, np.uint64)
        _gen().gen_rmat(key, self.scale, a, b, c, start, k, _ptr(self.perm), _ptr(out),
                        int(keep_loops), _nthreads())
        return out

    def sample(self, k: int):
        """The next k draws of the sample stream as (u, v), self-loops included."""
        keys = self._draw(self.key_sample, self.drawn, int(k), True)
        self.drawn += int(k)
        return ((keys >> np.uint64(32)).astype(np.int64),
                (keys & np.uint64(0xFFFFFFFF)).astype(np.int64))

    def graph(self, m: int):
        """m distinct directed edges without self-loops, sorted by (u, v)."""
        keys = _unique_draws(lambda s, k: self._draw(self.key_graph, s, k, False), m, self.n)
        return split_keys(keys)


class ChungLu:
    """Chung-Lu power-law sampler over n nodes (undirected pairs).

    Node i (before relabelling) has weight w_i proportional to
    (i + 1) ** (-1 / (beta - 1)), scaled so that the weights sum to
    mean_degree * n and capped at sqrt(sum w); an edge's endpoints are drawn
    independently with probability proportional to w. Ids are relabelled by a
    seeded permutation, as for R-MAT; draws come from the native sampler.
    """

    def __init__(self, n: int, mean_degree: float = 16.0, beta: float = 2.1,
                 seed: int = BASE_SEED):
        self.n = n
        self.rng = rng_for(seed)
        w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (beta - 1.0))
        w *= mean_degree * n / w.sum()
        w = np.minimum(w, np.sqrt(w.sum()))
        self.cdf = np.cumsum(w)
        self.cdf /= self.cdf[-1]
        self.perm = self.rng.permutation(n).astype(np.int64)
        self.key_graph, self.key_sample = (int(x) for x in self.rng.integers(0, 1 << 63, 2))
        self.drawn = 0

    def _draw(self, key, start, k, keep_loops):
        out = np.empty(k, np.uint64)
        _gen().gen_chunglu(key, _ptr(self.cdf), self.n, start, k, _ptr(self.perm), _ptr(out),
                           int(keep_loops), _nthreads())
        return out

    def sample(self, k: int):
        """The next k draws of the sample stream as (u, v), self-loops included."""
        keys = self._draw(self.key_sample, self.drawn, int(k), True)
        self.drawn += int(k)
        return ((keys >> np.uint64(32)).astype(np.int64),
                (keys & np.uint64(0xFFFFFFFF)).astype(np.int64))

    def graph(self, m_undirected: int):
        """m_undirected distinct unordered pairs {u, v}, u != v, returned as
        (lo, hi) arrays (the caller stores both directions)."""
        keys = _unique_draws(lambda s, k: self._draw(self.key_graph, s, k, False), m_undirected,
                             self.n)
        return split_keys(keys)


def chung_lu_graph(n: int, m_undirected: int, seed: int = BASE_SEED, **kw):
    g = ChungLu(n, seed=seed, **kw)
    lo, hi = g.graph(m_undirected)
    return g, lo, hi


def rmat_graph(scale: int, m: int, seed: int = BASE_SEED, **kw):
    g = RMat(scale, seed=seed, **kw)
    src, dst = g.graph(m)
    return g, src, dst


def out_degrees(n: int, src: np.ndarray) -> np.ndarray:
    return np.bincount(src, minlength=n).astype(np.int64)


def max_out_degree_seed(n: int, src: np.ndarray) -> int:
    """Node of highest out-degree, ties broken by the smaller id."""
    deg = out_degrees(n, src)
    return int(np.argmax(deg))  # argmax returns the first (smallest id) maximum


# --------------------------------------------------------------------------
# Update streams
# --------------------------------------------------------------------------
class EdgeSet:
    """A set of directed edge keys, used to draw valid updates.

    ``keys`` is the sorted array; batches applied with ``apply`` are kept as
    small pending insert / delete sets and merged into the array (one linear
    pass) only when ``keys`` is read or the pending sets grow large."""

    _PENDING_MAX = 1 << 20

    def __init__(self, src, dst):
        keys = edge_keys(np.asarray(src), np.asarray(dst))
        if keys.size > 1 and not bool(np.all(keys[1:] > keys[:-1])):
            # distinct keys, ascending (the native radix sort over the bits in use)
            bits = max(1, int(keys.max()).bit_length())
            keys = np.ascontiguousarray(keys)
            k = _gen().keys_sort_unique(_ptr(keys), keys.size, bits, _nthreads())
            keys = keys[:k]
        self._base = keys
        self._ins = np.empty(0, np.uint64)  # present, not in _base
        self._del = np.empty(0, np.uint64)  # in _base, not present

    @property
    def keys(self) -> np.ndarray:
        if self._ins.size or self._del.size:
            out = np.empty(self._base.size + self._ins.size, np.uint64)
            k = _gen().keys_apply(_ptr(self._base), self._base.size, _ptr(self._ins), self._ins.size,
                                  _ptr(self._del), self._del.size, _ptr(out))
            self._base = out[:k]
            self._ins = np.empty(0, np.uint64)
            self._del = np.empty(0, np.uint64)
        return self._base

    @keys.setter
    def keys(self, value):
        self._base = np.asarray(value, np.uint64)
        self._ins = np.empty(0, np.uint64)
        self._del = np.empty(0, np.uint64)

    @property
    def size(self) -> int:
        return int(self._base.size + self._ins.size - self._del.size)

    def _in_base(self, keys):
        if self._base.size == 0:
            return np.zeros(np.shape(keys), bool)
        pos = np.minimum(np.searchsorted(self._base, keys), self._base.size - 1)
        return self._base[pos] == keys

    def contains(self, keys: np.ndarray) -> np.ndarray:
        keys = np.asarray(keys, np.uint64)
        got = self._in_base(keys)
        if self._del.size:
            got &= ~np.isin(keys, self._del)
        if self._ins.size:
            got |= np.isin(keys, self._ins)
        return got

    def apply(self, ins_keys: np.ndarray, del_keys: np.ndarray):
        """Remove del_keys (present), then add ins_keys (absent)."""
        ins = np.unique(np.asarray(ins_keys, np.uint64))
        dels = np.unique(np.asarray(del_keys, np.uint64))
        if dels.size:
            self._ins = np.setdiff1d(self._ins, dels, assume_unique=True)
            self._del = np.union1d(self._del, dels[self._in_base(dels)])
        if ins.size:
            base = self._in_base(ins)
            self._del = np.setdiff1d(self._del, ins[base], assume_unique=True)
            self._ins = np.union1d(self._ins, ins[~base])
        if self._ins.size + self._del.size > self._PENDING_MAX:
            _ = self.keys

    def draw_present(self, rng, count: int) -> np.ndarray:
        """``count`` keys drawn uniformly (with replacement) from the present keys."""
        nb, ni = self._base.size, self._ins.size
        out = np.empty(0, np.uint64)
        while out.size < count:
            i = rng.integers(0, nb + ni, 2 * (count - out.size) + 8)
            cand = np.where(i < nb, self._base[np.minimum(i, max(nb - 1, 0))],
                            self._ins[np.maximum(i - nb, 0)] if ni else np.uint64(0))
            ok = i >= nb
            if self._del.size:
                ok |= ~np.isin(cand, self._del)
            else:
                ok |= True
            out = np.concatenate([out, cand[ok]])
        return out[:count]


def _pack(ins_keys, del_keys, rng) -> np.ndarray:
    ops = np.empty(ins_keys.size + del_keys.size, UPDATE_DTYPE)
    iu, iv = split_keys(ins_keys)
    du, dv = split_keys(del_keys)
    ops["u"] = np.concatenate([iu, du])
    ops["v"] = np.concatenate([iv, dv])
    ops["op"] = np.concatenate([np.full(ins_keys.size, OP_INSERT_EDGE, np.int32),
                                np.full(del_keys.size, OP_DELETE_EDGE, np.int32)])
    return ops[rng.permutation(ops.size)]


def _draw_absent(es: EdgeSet, k: int, sampler, rng) -> np.ndarray:
    got = np.empty(0, np.uint64)
    while got.size < k:
        u, v = sampler(max(2 * (k - got.size), 16))
        ok = u != v
        cand = edge_keys(u[ok], v[ok])
        cand = cand[~es.contains(cand)]
        got = _first_unique(np.concatenate([got, cand]))
    return got[:k]


def _draw_present(es: EdgeSet, k: int, rng) -> np.ndarray:
    idx = rng.choice(es.keys.size, size=k, replace=False)
    return es.keys[idx]


def edge_update_stream(src, dst, n: int, batches: int, n_ins: int, n_del: int, seed: int,
                       sampler=None):
    """``batches`` batches of ``n_ins`` insertions of absent edges and ``n_del``
    deletions of existing edges, drawn against the graph as updated by the
    previous batches. Insert endpoints come from ``sampler(k) -> (u, v)``
    (uniform over node pairs if None). The ops of a batch are shuffled.
    """
    rng = rng_for(seed)
    es = EdgeSet(src, dst)
    if sampler is None:
        def sampler(k):
            return (rng.integers(0, n, k, dtype=np.int64), rng.integers(0, n, k, dtype=np.int64))
    out = []
    for _ in range(batches):
        ins = _draw_absent(es, n_ins, sampler, rng)
        dels = _draw_present(es, n_del, rng)
        out.append(_pack(ins, dels, rng))
        es.apply(ins, dels)
    return out


def random_mixed_batch(rng, n: int, es: EdgeSet, dead: np.ndarray, n_ops: int,
                       p_add=0.05, p_delnode=0.03, protect=(), p_zero_row=0.0):
    """A small batch mixing the op kinds, valid in sequence (used by tests).

    Node deletions never hit ``protect`` (the seeds) and later ops never name
    a node deleted earlier. ``p_zero_row`` > 0 adds row zeroings (any live
    node, seeds included). ``dead`` is updated in place; the returned n is the
    node count after the batch.
    """
    ops = []
    live = [i for i in range(n) if not dead[i]]
    cur_keys = set(es.keys.tolist())
    dead_now = set()
    nn = n
    for _ in range(n_ops):
        r = rng.random()
        if r < p_add:
            ops.append((0, 0, OP_ADD_NODE))
            live.append(nn)
            nn += 1
        elif r < p_add + p_delnode and len(live) > 2:
            cands = [x for x in live if x not in protect]
            if not cands:
                continue
            w = int(cands[rng.integers(len(cands))])
            ops.append((w, 0, OP_DELETE_NODE))
            live.remove(w)
            dead_now.add(w)
            cur_keys = {k for k in cur_keys if (k >> 32) != w and (k & 0xFFFFFFFF) != w}
        elif p_zero_row > 0 and r < p_add + p_delnode + p_zero_row:
            w = int(live[rng.integers(len(live))])
            ops.append((w, 0, OP_ZERO_ROW))
            cur_keys = {k for k in cur_keys if (k >> 32) != w}
        else:
            u = int(live[rng.integers(len(live))])
            v = int(live[rng.integers(len(live))])
            key = (u << 32) | v
            if rng.random() < 0.5:
                ops.append((u, v, OP_INSERT_EDGE))
                cur_keys.add(key)
            else:
                # Prefer deleting an existing out-edge of u, else a no-op delete.
                outs = [k for k in cur_keys if (k >> 32) == u]
                if outs and rng.random() < 0.8:
                    key = outs[rng.integers(len(outs))]
                    v = key & 0xFFFFFFFF
                ops.append((u, int(v), OP_DELETE_EDGE))
                cur_keys.discard((u << 32) | int(v))
    for w in dead_now:
        dead[w] = 1
    arr = np.array(ops, dtype=np.int64).reshape(-1, 3)
    out = np.empty(arr.shape[0], UPDATE_DTYPE)
    out["u"], out["v"], out["op"] = arr[:, 0], arr[:, 1], arr[:, 2]
    keys = np.array(sorted(cur_keys), dtype=np.uint64)
    es.keys = keys
    return out, nn


def undirected_update_stream(lo, hi, n: int, sizes, seed: int, sampler):
    """One batch per entry of ``sizes``: that many undirected pairs, half
    insertions of absent pairs drawn from ``sampler`` and half deletions of
    present pairs (uniform), each pair as its two directed ops."""
    rng = rng_for(seed)
    es = EdgeSet(lo, hi)  # canonical (min, max) keys
    out = []
    for k in sizes:
        n_ins = int(k) // 2
        n_del = int(k) - n_ins

        def canon(kk):
            u, v = sampler(kk)
            return np.minimum(u, v), np.maximum(u, v)

        ins = _draw_absent(es, n_ins, canon, rng)
        dels = _draw_present(es, n_del, rng)
        iu, iv = split_keys(ins)
        du, dv = split_keys(dels)
        ops = np.empty(2 * (ins.size + dels.size), UPDATE_DTYPE)
        ops["u"] = np.concatenate([iu, iv, du, dv])
        ops["v"] = np.concatenate([iv, iu, dv, du])
        ops["op"] = np.concatenate([np.full(2 * ins.size, OP_INSERT_EDGE, np.int32),
                                    np.full(2 * dels.size, OP_DELETE_EDGE, np.int32)])
        out.append(ops[rng.permutation(ops.size)])
        es.apply(ins, dels)
    return out


def log_uniform_sizes(batches: int, lo: float, hi: float, seed: int):
    """floor(10 ** U(log10 lo, log10 hi)) per batch."""
    rng = rng_for(seed)
    return np.floor(10.0 ** rng.uniform(np.log10(lo), np.log10(hi), batches)).astype(np.int64)


def node_op_stream(src, dst, n: int, batches: int, n_new: int, new_degree: int, n_del_nodes: int,
                   n_edge_ops: int, seed: int, protect=()):
    """Batches mixing node and edge operations, valid in sequence:
    ``n_edge_ops`` edge ops (half insertions of absent edges between live
    nodes, half deletions of present edges), then ``n_new`` node additions each
    followed by ``new_degree`` out-edges to distinct live targets (uniform),
    then ``n_del_nodes`` deletions of nodes that existed before the batch
    (uniform over live nodes, never one in ``protect``)."""
    rng = rng_for(seed)
    es = EdgeSet(src, dst)
    cap = n + batches * n_new + 8
    dead = np.zeros(cap, bool)
    guard = np.zeros(cap, bool)
    guard[list(protect)] = True
    nn = n
    out = []
    for _ in range(batches):
        parts = []
        # edge ops between live nodes
        k_ins = n_edge_ops // 2
        k_del = n_edge_ops - k_ins

        def live_pairs(k):
            u = rng.integers(0, nn, k, dtype=np.int64)
            v = rng.integers(0, nn, k, dtype=np.int64)
            ok = ~dead[u] & ~dead[v]
            return u[ok], v[ok]

        ins = _draw_absent(es, k_ins, live_pairs, rng)
        dels = np.empty(0, np.uint64)
        while dels.size < k_del:
            cand = es.draw_present(rng, 2 * (k_del - dels.size) + 16)
            cu, cv = split_keys(cand)
            cand = cand[~dead[cu] & ~dead[cv]]
            dels = _first_unique(np.concatenate([dels, cand]))
            dels = dels[~np.isin(dels, ins)]
        dels = dels[:k_del]
        parts.append(_pack(ins, dels, rng))
        es.apply(ins, dels)
        # new nodes with their out-edges
        new_keys = []
        for i in range(n_new):
            w = nn + i
            add = np.zeros(1, UPDATE_DTYPE)
            add["op"] = OP_ADD_NODE
            parts.append(add)
            tg = np.empty(0, np.int64)
            while tg.size < new_degree:
                c = rng.integers(0, nn, 2 * new_degree, dtype=np.int64)
                c = c[~dead[c]]
                tg = np.unique(np.concatenate([tg, c]))
            tg = rng.permutation(tg)[:new_degree]
            e = np.zeros(new_degree, UPDATE_DTYPE)
            e["u"], e["v"], e["op"] = w, tg, OP_INSERT_EDGE
            parts.append(e)
            new_keys.append(edge_keys(np.full(new_degree, w), tg))
        nn += n_new
        es.apply(np.concatenate(new_keys) if new_keys else np.empty(0, np.uint64),
                 np.empty(0, np.uint64))
        # node deletions among the nodes that existed before the batch
        cand = np.flatnonzero(~dead[: nn - n_new] & ~guard[: nn - n_new])
        victims = rng.choice(cand, n_del_nodes, replace=False)
        dn = np.zeros(n_del_nodes, UPDATE_DTYPE)
        dn["u"], dn["op"] = victims, OP_DELETE_NODE
        parts.append(dn)
        dead[victims] = True
        out.append(np.concatenate(parts))
    return out


def sized_update_stream(src, dst, n: int, sizes, seed: int, sampler):
    """One batch per entry of ``sizes``: half insertions of absent edges drawn
    from ``sampler``, half deletions of edges of the initial graph (uniform),
    valid in sequence. Absence and presence are checked against the initial
    edge set and the keys inserted or deleted so far, so no batch rewrites the
    whole edge set (inserted edges are never deleted again)."""
    rng = rng_for(seed)
    es = EdgeSet(src, dst)
    inserted, deleted = set(), set()
    out = []
    for k in sizes:
        k = int(k)
        n_ins, n_del = k // 2, k - k // 2
        ins = []
        while len(ins) < n_ins:
            u, v = sampler(2 * (n_ins - len(ins)) + 8)
            ok = u != v
            cand = edge_keys(u[ok], v[ok])
            cand = cand[~es.contains(cand)]
            for c in cand.tolist():
                if c not in inserted:
                    inserted.add(c)
                    ins.append(c)
                    if len(ins) == n_ins:
                        break
        dels = []
        while len(dels) < n_del:
            for c in es.keys[rng.integers(0, es.keys.size, 2 * (n_del - len(dels)) + 8)].tolist():
                if c not in deleted:
                    deleted.add(c)
                    dels.append(c)
                    if len(dels) == n_del:
                        break
        out.append(_pack(np.array(ins, np.uint64), np.array(dels, np.uint64), rng))
    return out
