"""The serving loop: results in the mix (merged update batches, queries in
slots overlapping the next batch) equal those of serving each request alone."""
import numpy as np
import pytest

from paper_1712_00595_gb300 import native as N
from paper_1712_00595_gb300 import serve as SV
from paper_1712_00595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C_RESTART = 0.15


def _graph(rng, n):
    src = list(rng.integers(0, n, 12 * n))
    dst = list(rng.integers(0, n, 12 * n))
    h = min(1500, n - 1)
    src += list(rng.choice(n, h, replace=False))
    dst += [1] * h
    s, d = np.array(src, np.int32), np.array(dst, np.int32)
    keep = s != d
    return s[keep], d[keep]


def _requests(rng, n, src, dst, seeds, count):
    es = W.EdgeSet(src, dst)
    dead = np.zeros(n + count * 64, np.uint8)
    nn = n
    out, t = [], 0.0
    for _ in range(count):
        t += float(rng.exponential(1e-4))
        if rng.random() < 0.4:
            m = int(rng.integers(1, len(seeds) + 1))
            out.append(SV.Query(t, tuple(int(x) for x in rng.choice(len(seeds), m, replace=False)),
                                int(rng.integers(1, 60))))
        else:
            ops, nn = W.random_mixed_batch(rng, nn, es, dead, int(rng.integers(1, 60)),
                                           protect=tuple(int(s) for s in seeds))
            out.append(SV.Update(t, ops))
    return out


def _engine(n, src, dst, seeds):
    e = N.Engine(precision=N.OSP_PREC_FP64, device=0, max_nodes=n + 8192, use_graphs=True)
    e.load_graph(n, src, dst)
    e.set_seeds(np.array(seeds, np.int32), C_RESTART)
    e.init_scores(1e-13)
    return e


def _same_topk(a, b, tol=1e-10):
    (ia, sa), (ib, sb) = a, b
    assert ia.size == ib.size
    assert np.allclose(sa, sb, rtol=0, atol=tol)
    for x, y, s in zip(ia, ib, sa):
        if x != y:  # only a tie (equal scores within tol) may change places
            assert np.sum(np.abs(sa - s) <= tol) > 1


@pytest.mark.parametrize("realtime", [False, True])
def test_served_results_equal_requests_served_alone(realtime):
    rng = np.random.default_rng(31)
    n = 3000
    src, dst = _graph(rng, n)
    seeds = [0, 1, 7, 100, 2000]
    reqs = _requests(rng, n, src, dst, seeds, 60)
    eng = _engine(n, src, dst, seeds)
    srv = SV.Server(eng, slots=3, eps=1e-12)
    got = srv.run(reqs, realtime=realtime)
    n_upd = sum(isinstance(r, SV.Update) for r in reqs)
    if not realtime:
        assert len(srv.batches) < n_upd  # consecutive updates were merged
    final = [eng.query(j) for j in range(len(seeds))]
    eng.close()
    # each request alone, in arrival order, on a fresh engine
    ref = _engine(n, src, dst, seeds)
    for r, g in zip(reqs, got):
        if isinstance(r, SV.Update):
            ref.apply_updates(r.ops, 1e-12)
            assert g.batch >= 0
        else:
            for pos, s in enumerate(r.seeds):
                _same_topk(g.topk[pos], ref.topk(r.k, seed_idx=s))
    for j in range(len(seeds)):
        assert np.abs(ref.query(j) - final[j]).sum() <= 1e-10
    ref.close()
    assert all(g.done >= g.request.t for g in got)


def test_latest_policy_matches_its_batches_applied_alone():
    rng = np.random.default_rng(32)
    n = 3000
    src, dst = _graph(rng, n)
    seeds = [0, 1, 7, 100, 2000]
    reqs = _requests(rng, n, src, dst, seeds, 60)
    eng = _engine(n, src, dst, seeds)
    srv = SV.Server(eng, slots=3, eps=1e-12, policy="latest")
    got = srv.run(reqs, realtime=False)
    eng.close()
    n_upd = sum(isinstance(r, SV.Update) for r in reqs)
    assert len(srv.batches) < n_upd
    # replay: the server's merged batches one by one; each query after the
    # number of batches it saw
    ref = _engine(n, src, dst, seeds)
    applied = 0
    order = sorted((g.seen, k) for k, g in enumerate(got) if isinstance(g.request, SV.Query))
    for seen, k in order:
        while applied < seen:
            ref.apply_updates(np.concatenate([reqs[q].ops for q in srv.batch_requests[applied]]),
                              1e-12)
            applied += 1
        r = reqs[k]
        for pos, s in enumerate(r.seeds):
            _same_topk(got[k].topk[pos], ref.topk(r.k, seed_idx=s))
    ref.close()


def test_query_slots_api():
    rng = np.random.default_rng(2)
    n = 500
    src, dst = _graph(rng, n)
    e = _engine(n, src, dst, [0, 3])
    with pytest.raises(N.OspError):
        e.topk_async(0, 10)  # no slots yet
    e.query_slots(2)
    e.topk_async(0, 10, seed_idx=1)
    with pytest.raises(N.OspError) as err:
        e.topk_async(0, 10, seed_idx=0)  # slot busy
    assert err.value.status == N.OSP_ESTATE
    ids, sc = e.topk_wait(0)
    want_ids, want_sc = e.topk(10, seed_idx=1)
    assert np.array_equal(ids, want_ids) and np.array_equal(sc, want_sc)
    with pytest.raises(N.OspError):
        e.topk_wait(0)  # nothing enqueued
    e.query_slots(0)
    e.close()


@pytest.mark.parametrize("k", [1, 100, 4096])
@pytest.mark.parametrize("normalize", [False, True])
def test_topk_async_many_matches_topk_per_seed(k, normalize):
    """One launch sequence for many seeds (live seeds, and dead-end seeds whose
    vector is c e_s, so that the k-th score is a tie among zeros broken by id)
    gives, slot by slot, the same ids and scores as osp_topk seed by seed."""
    rng = np.random.default_rng(11)
    n = 6000
    src, dst = _graph(rng, n)
    dead = [7, 8, 9]
    keep = ~np.isin(src, dead)  # three dead-end nodes
    src, dst = src[keep], dst[keep]
    outdeg = np.bincount(src, minlength=n)
    live = [int(x) for x in rng.choice(np.flatnonzero(outdeg > 0), 37, replace=False)]
    seeds = live + dead
    e = _engine(n, src, dst, seeds)
    e.query_slots(40)
    order = rng.permutation(len(seeds))
    for a in range(0, len(seeds), 32):
        part = [int(x) for x in order[a:a + 32]]
        slots = list(range(len(part)))
        e.topk_async_many(slots, part, k, normalize=normalize)
        for sl, sd in zip(slots, part):
            ids, sc = e.topk_wait(sl)
            want_ids, want_sc = e.topk(k, seed_idx=sd, normalize=normalize)
            assert np.array_equal(ids, want_ids) and np.array_equal(sc, want_sc)
            r = e.query(sd, normalize=normalize)
            # the ranking: the k largest scores in order, ties by smaller id
            ref = np.lexsort((np.arange(n), -r))[:k]
            assert np.array_equal(ids, ref)
    with pytest.raises(N.OspError) as err:
        e.topk_async_many([0, 0], [1, 2], 10)
    assert err.value.status == N.OSP_EINVAL
    e.close()
