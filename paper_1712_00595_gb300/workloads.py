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

import numpy as np

# One update operation, laid out exactly as ``osp_update`` in include/osp.h.
UPDATE_DTYPE = np.dtype([("u", "<i4"), ("v", "<i4"), ("op", "<i4")])
OP_INSERT_EDGE = 0
OP_DELETE_EDGE = 1
OP_ADD_NODE = 2
OP_DELETE_NODE = 3

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
    """

    def __init__(self, scale: int, a=0.57, b=0.19, c=0.19, d=0.05, seed: int = BASE_SEED,
                 permute: bool = True):
        self.scale = scale
        self.n = 1 << scale
        self.p = (a, b, c, d)
        self.rng = rng_for(seed)
        self.perm = self.rng.permutation(self.n).astype(np.int64) if permute else None

    def sample(self, k: int):
        a, b, c, _ = self.p
        u = np.zeros(k, np.int64)
        v = np.zeros(k, np.int64)
        for _lvl in range(self.scale):
            r = self.rng.random(k)
            ubit = r >= (a + b)
            vbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
            u = (u << 1) | ubit
            v = (v << 1) | vbit
        if self.perm is not None:
            u = self.perm[u]
            v = self.perm[v]
        return u, v

    def graph(self, m: int):
        def draw(k):
            out = []
            for s in range(0, k, 1 << 24):
                u, v = self.sample(min(1 << 24, k - s))
                ok = u != v
                out.append(edge_keys(u[ok], v[ok]))
            return np.concatenate(out)

        return split_keys(_fill_unique(draw, m, 1 << 24))


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
    """Sorted array of directed edge keys, used to draw valid updates."""

    def __init__(self, src, dst):
        self.keys = np.sort(edge_keys(np.asarray(src), np.asarray(dst)))

    def contains(self, keys: np.ndarray) -> np.ndarray:
        pos = np.searchsorted(self.keys, keys)
        pos = np.minimum(pos, self.keys.size - 1)
        return self.keys[pos] == keys

    def apply(self, ins_keys: np.ndarray, del_keys: np.ndarray):
        if del_keys.size:
            pos = np.searchsorted(self.keys, np.sort(del_keys))
            self.keys = np.delete(self.keys, pos)
        if ins_keys.size:
            ins = np.sort(ins_keys)
            pos = np.searchsorted(self.keys, ins)
            self.keys = np.insert(self.keys, pos, ins)


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
                       p_add=0.05, p_delnode=0.03, protect=()):
    """A small batch mixing all four op kinds, valid in sequence (used by tests).

    Node deletions never hit ``protect`` (the seeds) and later ops never name
    a node deleted earlier. ``dead`` is updated in place; the returned n is the
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
