"""Serving loop: a stream of update and query requests over one engine.

Requests carry arrival times. The server walks them in arrival order:

* consecutive update requests that have arrived are merged into one engine
  batch (up to the engine's batch limit), so one propagation serves all of
  them;
* a query (top-k for one or more tracked seeds) takes free query slots, one
  per seed, and is enqueued on the engine's query stream. It reads the scores
  after exactly the updates that arrived before it, because a query is never
  merged past: the next batch is applied only after the query is enqueued,
  and that batch's propagation waits for it on the device. Its ingest, merge
  and offset kernels run while the query does.

The seeds of one query are ranked by one launch sequence (osp_topk_async_many).
A ranking is kept per seed with the number of engine batches applied before
it (the score version): a later query for that seed, at the same version and
for no more entries, takes it instead of ranking again; the same holds for a
ranking still in flight.

Results are therefore the same as serving the requests one at a time, up to
the truncation of OSP-T (merging update requests changes where the series of
Algorithm 1 is cut, within its error bound). The number of slots is the HBM
budget for queries divided by the bytes of one slot.

With policy "latest" the server instead merges every arrived update request
(in batches up to the engine limit) before the queries that arrived with them,
and answers those queries on the newest scores; each query records how many
engine batches it saw, so its result equals the top-k after those batches
applied one by one. This trades arrival-order reads for far fewer batches.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import native as N


@dataclass
class Update:
    t: float          # arrival time (s from the start of the run)
    ops: np.ndarray   # UPDATE_DTYPE


@dataclass
class Query:
    t: float
    seeds: tuple      # seed indices (columns of the engine's seed block)
    k: int = 100


@dataclass
class Result:
    request: object
    done: float = 0.0                             # completion time (s from the start)
    batch: int = -1                               # updates: the engine batch that applied them
    seen: int = -1                                # queries: engine batches applied before them
    topk: list = field(default_factory=list)      # queries: (ids, scores) per seed

    @property
    def latency(self):
        return self.done - self.request.t


def slot_bytes(n_slots_nodes: int) -> int:
    """Device bytes of one query slot for an engine of n node slots (an upper
    bound: the column buffer, chunk counts and the select and sort scratch)."""
    return 8 * n_slots_nodes + 160 * 1024


class Server:
    def __init__(self, engine: N.Engine, slots: int, eps: float, max_ops: int = 0,
                 policy: str = "ordered"):
        if policy not in ("ordered", "latest"):
            raise ValueError("policy is 'ordered' or 'latest'")
        self.policy = policy
        self.eng = engine
        self.slots = int(slots)
        self.eps = eps
        self.max_ops = int(max_ops) or N.MAX_APPLY_OPS
        engine.query_slots(self.slots)
        self.batches = []      # sizes (ops) of the engine batches formed
        self.batch_requests = []  # request indices (of the last run) merged into each batch
        # top-k results by seed: (score version = batches applied, k, ids, scores);
        # a query for a seed whose scores have not changed since takes them
        self.cache = {}
        self.topk_computed = 0  # seeds ranked on the device
        self.topk_reused = 0    # seeds answered from a result of the same score version

    def run(self, requests, realtime=True):
        """Serve ``requests`` (sorted by arrival). realtime: a request is taken
        only once the wall clock reaches its arrival time; otherwise all are
        available at once (closed loop)."""
        reqs = list(requests)
        res = [Result(r) for r in reqs]
        free = list(range(self.slots))
        # slot -> [seed, score version, k, [(result index, position, k wanted), ...]]
        inflight = {}
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: float("inf"))
        self._now = lambda: time.perf_counter() - t0

        def collect_all():
            for slot, (seed, ver, k, waiters) in inflight.items():
                ids, sc = self.eng.topk_wait(slot)
                old = self.cache.get(seed)
                if old is None or old[0] < ver or (old[0] == ver and old[1] < k):
                    self.cache[seed] = (ver, k, ids, sc)
                now = time.perf_counter() - t0
                for ri, pos, kw in waiters:
                    res[ri].topk[pos] = (ids[:kw], sc[:kw])
                    res[ri].done = max(res[ri].done, now)
                free.append(slot)
            inflight.clear()

        if self.policy == "latest":
            return self._run_latest(reqs, res, free, inflight, t0, clock, collect_all)
        i = 0
        while i < len(reqs):
            if reqs[i].t > clock():
                if inflight:
                    collect_all()
                    continue
                time.sleep(max(0.0, reqs[i].t - clock()))
                continue
            r = reqs[i]
            if isinstance(r, Query):
                res[i].seen = len(self.batches)
                self._enqueue_query(r, i, res, free, inflight, collect_all)
                i += 1
                continue
            # merge the consecutive arrived updates that fit in one batch
            j, ops = i, 0
            while (j < len(reqs) and isinstance(reqs[j], Update) and reqs[j].t <= clock()
                   and ops + reqs[j].ops.size <= self.max_ops):
                ops += reqs[j].ops.size
                j += 1
            if j == i:  # a single request larger than the limit is an error of the caller
                raise ValueError("update request of %d ops exceeds the batch limit %d"
                                 % (reqs[i].ops.size, self.max_ops))
            self._apply(reqs, res, list(range(i, j)), t0)
            collect_all()   # the queries enqueued before this batch have finished
            i = j
        collect_all()
        return res

    def _enqueue_query(self, r, ri, res, free, inflight, collect_all):
        # A seed whose top-k is known for the current score version (with at
        # least r.k entries), or already in flight for it, costs nothing more;
        # the other seeds go out as one launch sequence, up to 32 (and up to
        # the free slots) at a time.
        ver = len(self.batches)
        res[ri].topk = [None] * len(r.seeds)
        todo = []
        for pos, s in enumerate(r.seeds):
            s = int(s)
            c = self.cache.get(s)
            if c is not None and c[0] == ver and c[1] >= r.k:
                res[ri].topk[pos] = (c[2][:r.k], c[3][:r.k])
                self.topk_reused += 1
                continue
            hit = next((e for e in inflight.values() if e[0] == s and e[1] == ver and e[2] >= r.k),
                       None)
            if hit is not None:
                hit[3].append((ri, pos, r.k))
                self.topk_reused += 1
                continue
            todo.append((pos, s))
        if not todo and all(t is not None for t in res[ri].topk):
            res[ri].done = max(res[ri].done, self._now())
        at = 0
        while at < len(todo):
            if not free:
                collect_all()
            take = min(len(todo) - at, len(free), 32)
            slots = [free.pop() for _ in range(take)]
            part = todo[at:at + take]
            self.eng.topk_async_many(slots, [s for _, s in part], r.k)
            for sl, (pos, s) in zip(slots, part):
                inflight[sl] = [s, ver, r.k, [(ri, pos, r.k)]]
            self.topk_computed += take
            at += take

    def _apply(self, reqs, res, idx, t0):
        batch = np.concatenate([reqs[q].ops for q in idx])
        self.eng.apply_updates(batch, self.eps)
        now = time.perf_counter() - t0
        for q in idx:
            res[q].done = now
            res[q].batch = len(self.batches)
        self.batches.append(int(batch.size))
        self.batch_requests.append(list(idx))

    def _run_latest(self, reqs, res, free, inflight, t0, clock, collect_all):
        i = 0
        while i < len(reqs):
            if reqs[i].t > clock():
                if inflight:
                    collect_all()
                    continue
                time.sleep(max(0.0, reqs[i].t - clock()))
                continue
            j = i
            while j < len(reqs) and reqs[j].t <= clock():
                j += 1
            ups = [q for q in range(i, j) if isinstance(reqs[q], Update)]
            qs = [q for q in range(i, j) if isinstance(reqs[q], Query)]
            cur, ops = [], 0
            for q in ups:  # every arrived update, in batches up to the engine limit
                if reqs[q].ops.size > self.max_ops:
                    raise ValueError("update request of %d ops exceeds the batch limit %d"
                                     % (reqs[q].ops.size, self.max_ops))
                if ops + reqs[q].ops.size > self.max_ops:
                    self._apply(reqs, res, cur, t0)
                    collect_all()
                    cur, ops = [], 0
                cur.append(q)
                ops += reqs[q].ops.size
            if cur:
                self._apply(reqs, res, cur, t0)
                collect_all()
            for q in qs:  # on the newest scores; they overlap the next batch
                res[q].seen = len(self.batches)
                self._enqueue_query(reqs[q], q, res, free, inflight, collect_all)
            i = j
        collect_all()
        return res


def latency_summary(results, kind):
    lat = np.array([r.latency for r in results if isinstance(r.request, kind)])
    if lat.size == 0:
        return None
    return {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}


def poisson_requests(rate, count, n_seeds, update_stream, query_frac, seed, k=100,
                     max_query_seeds=32):
    """``count`` requests with exponential inter-arrival times at ``rate`` per
    second: a fraction ``query_frac`` are top-k queries for 1..max_query_seeds
    distinct tracked seeds, the rest take the next batch of ``update_stream``."""
    from .workloads import rng_for
    rng = rng_for(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    out = []
    it = iter(update_stream)
    for a in t:
        if rng.random() < query_frac:
            m = int(rng.integers(1, max_query_seeds + 1))
            out.append(Query(float(a), tuple(int(x) for x in rng.choice(n_seeds, m, replace=False)), k))
        else:
            nxt = next(it, None)
            if nxt is None:
                break
            out.append(Update(float(a), nxt))
    return out
