"""Host logic of the serving loop (paper_1712_00595_gb300/serve.py) against a
fake engine: which updates each batch merges, what each query sees, the batch
limit and the reuse of query slots. No GPU is involved; the GPU tests check
the same loop's answers against serving each request alone."""
import numpy as np
import pytest

from paper_1712_00595_gb300 import serve as SV
from paper_1712_00595_gb300 import workloads as W


class FakeEngine:
    """Records the calls the server makes. A top-k answer holds k entries,
    each id encoding the number of batches applied when the ranking was
    enqueued and the seed it ranks (version * 1000 + seed)."""

    def __init__(self):
        self.batches = []      # op counts of the applied batches
        self.slots = 0
        self.busy = {}         # slot -> (version, seed, k)
        self.ranked = 0        # seeds ranked

    def query_slots(self, k):
        self.slots = k

    def apply_updates(self, ops, eps):
        assert ops.dtype == W.UPDATE_DTYPE and ops.size > 0
        self.batches.append(ops.copy())
        return {}

    def topk_async(self, slot, k, seed_idx=0):
        assert 0 <= slot < self.slots and slot not in self.busy, "slot in use"
        self.busy[slot] = (len(self.batches), seed_idx, k)
        self.ranked += 1

    def topk_async_many(self, slots, seeds, k):
        assert 1 <= len(slots) <= 32 and len(slots) == len(seeds)
        assert len(set(slots)) == len(slots), "a slot named twice"
        for sl, sd in zip(slots, seeds):
            self.topk_async(sl, k, seed_idx=sd)

    def topk_wait(self, slot):
        version, seed, k = self.busy.pop(slot)
        return np.full(k, version * 1000 + seed, np.int32), np.full(k, float(version))


def _update(t, tag, size=1):
    ops = np.zeros(size, W.UPDATE_DTYPE)
    ops["u"] = tag  # identifies the request inside merged batches
    ops["op"] = W.OP_INSERT_EDGE
    return SV.Update(t, ops)


def _mixed(rng, count, max_size=5, n_seeds=8):
    reqs = []
    for i in range(count):
        if rng.random() < 0.4:
            m = int(rng.integers(1, 4))
            reqs.append(SV.Query(float(i), tuple(int(x) for x in rng.choice(n_seeds, m, replace=False)),
                                 int(rng.integers(1, 50))))
        else:
            reqs.append(_update(float(i), i, int(rng.integers(1, max_size + 1))))
    return reqs


@pytest.mark.parametrize("seed", range(4))
def test_ordered_policy_never_merges_past_a_query(seed):
    rng = np.random.default_rng(seed)
    reqs = _mixed(rng, 60)
    eng = FakeEngine()
    srv = SV.Server(eng, slots=3, eps=1e-6, max_ops=7, policy="ordered")
    res = srv.run(reqs, realtime=False)
    # every batch holds consecutive update requests, within the limit
    for idx, b in zip(srv.batch_requests, eng.batches):
        assert idx == list(range(idx[0], idx[-1] + 1))
        assert all(isinstance(reqs[i], SV.Update) for i in idx)
        assert b.size == sum(reqs[i].ops.size for i in idx) <= 7
        assert np.array_equal(b["u"], np.concatenate([reqs[i].ops["u"] for i in idx]))
    applied = [i for idx in srv.batch_requests for i in idx]
    assert applied == [i for i, r in enumerate(reqs) if isinstance(r, SV.Update)]
    for i, (r, out) in enumerate(zip(reqs, res)):
        if isinstance(r, SV.Query):
            # it saw exactly the updates that arrived before it
            before = sum(1 for idx in srv.batch_requests[:out.seen] for _ in idx)
            assert before == sum(1 for q in reqs[:i] if isinstance(q, SV.Update))
            assert [int(ids[0]) % 1000 for ids, _ in out.topk] == list(r.seeds)
            assert all(int(ids[0]) // 1000 == out.seen for ids, _ in out.topk)
            assert all(ids.size == sc.size == r.k for ids, sc in out.topk)
        else:
            assert 0 <= out.batch < len(eng.batches) and i in srv.batch_requests[out.batch]
    assert not eng.busy  # every slot was collected


def test_latest_policy_merges_every_arrived_update_first():
    rng = np.random.default_rng(9)
    reqs = _mixed(rng, 50)
    eng = FakeEngine()
    srv = SV.Server(eng, slots=2, eps=1e-6, max_ops=9, policy="latest")
    res = srv.run(reqs, realtime=False)  # everything has arrived: one round
    n_upd = sum(1 for r in reqs if isinstance(r, SV.Update))
    assert sum(len(idx) for idx in srv.batch_requests) == n_upd
    assert all(b.size <= 9 for b in eng.batches)
    for r, out in zip(reqs, res):
        if isinstance(r, SV.Query):
            assert out.seen == len(eng.batches)
            assert all(int(ids[0]) // 1000 == len(eng.batches) for ids, _ in out.topk)


def test_batch_limit_and_oversized_requests():
    eng = FakeEngine()
    srv = SV.Server(eng, slots=1, eps=1e-6, max_ops=4, policy="ordered")
    with pytest.raises(ValueError):
        srv.run([_update(0.0, 1, 5)], realtime=False)
    with pytest.raises(ValueError):
        SV.Server(FakeEngine(), slots=1, eps=1e-6, policy="newest")
    eng = FakeEngine()
    srv = SV.Server(eng, slots=1, eps=1e-6, max_ops=4, policy="ordered")
    srv.run([_update(0.0, k, 2) for k in range(5)], realtime=False)
    assert [b.size for b in eng.batches] == [4, 4, 2]


def test_slots_are_reused_when_a_query_asks_for_more_seeds_than_slots():
    eng = FakeEngine()
    srv = SV.Server(eng, slots=2, eps=1e-6, policy="ordered")
    q = SV.Query(0.0, (0, 1, 2, 3, 4), 10)
    res = srv.run([_update(0.0, 1), q, _update(0.0, 2), q], realtime=False)
    assert [int(ids[0]) % 1000 for ids, _ in res[1].topk] == [0, 1, 2, 3, 4]
    assert [int(ids[0]) // 1000 for ids, _ in res[1].topk] == [1] * 5
    assert [int(ids[0]) // 1000 for ids, _ in res[3].topk] == [2] * 5
    assert not eng.busy


def test_poisson_requests_and_latency_summary():
    stream = [np.zeros(3, W.UPDATE_DTYPE) for _ in range(100)]
    reqs = SV.poisson_requests(1000.0, 80, 16, stream, 0.5, seed=3, max_query_seeds=4)
    ts = [r.t for r in reqs]
    assert ts == sorted(ts) and len(reqs) == 80
    qs = [r for r in reqs if isinstance(r, SV.Query)]
    assert qs and all(1 <= len(q.seeds) <= 4 and len(set(q.seeds)) == len(q.seeds) for q in qs)
    res = [SV.Result(r, done=r.t + 0.001) for r in reqs]
    summ = SV.latency_summary(res, SV.Query)
    assert summ["count"] == len(qs) and abs(summ["p50_ms"] - 1.0) < 1e-6
    assert SV.latency_summary([], SV.Query) is None


@pytest.mark.parametrize("policy", ["ordered", "latest"])
def test_rankings_reused_within_a_score_version(policy):
    """Queries for a seed at the same score version (no batch in between) and
    for no more entries take the ranking already made (or in flight); a larger
    k or a new version ranks again. Every answer has the requested k entries
    of the right version and seed."""
    reqs = [SV.Query(0.0, (0, 1), 10), SV.Query(1.0, (1, 2), 5), SV.Query(2.0, (1,), 20),
            _update(3.0, 3), SV.Query(4.0, (0, 1), 10), SV.Query(5.0, (0,), 3)]
    eng = FakeEngine()
    srv = SV.Server(eng, slots=4, eps=1e-6, policy=policy)
    res = srv.run(reqs, realtime=False)
    if policy == "ordered":  # queries see the updates that arrived before them
        v = [0, 0, 0, None, 1, 1]
        ranked, reused = 6, 2   # 0, 1, 2, 1 (k = 20) at version 0; 0, 1 at version 1
    else:  # closed loop: the update is merged first, every query sees version 1
        v = [1, 1, 1, None, 1, 1]
        ranked, reused = 4, 4   # 0, 1, 2, 1 (k = 20); the rest reused
    for i, r in enumerate(reqs):
        if isinstance(r, SV.Query):
            got = [(int(ids[0]) % 1000, int(ids[0]) // 1000) for ids, _ in res[i].topk]
            assert got == [(s, v[i]) for s in r.seeds], (i, got)
            assert all(ids.size == r.k for ids, _ in res[i].topk)
    assert eng.ranked == srv.topk_computed == ranked
    assert srv.topk_reused == reused
