"""Input generators: seeded, thread-count independent, and the edge-set
bookkeeping that keeps update streams valid."""
import numpy as np

from paper_1712_00595_gb300 import workloads as W


def test_native_samplers_do_not_depend_on_thread_count():
    outs = []
    for th in (1, 3, 0):
        W.THREADS = th
        try:
            _, s, d = W.rmat_graph(14, 200000, seed=41)
            g, lo, hi = W.chung_lu_graph(1 << 14, 80000, seed=42)
            u, v = g.sample(1000)
            outs.append((s, d, lo, hi, u, v))
        finally:
            W.THREADS = 0
    for o in outs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(outs[0], o))
    s, d = outs[0][:2]
    keys = W.edge_keys(s, d)
    assert keys.size == 200000 and np.all(keys[1:] > keys[:-1]) and np.all(s != d)


def test_rmat_quadrant_frequencies():
    # one level of R-MAT picks (src bit, dst bit) = (0,0), (0,1), (1,0), (1,1)
    # with probabilities a, b, c, d; with scale 1 that is the whole draw
    g = W.RMat(1, permute=False, seed=5)
    u, v = g.sample(400000)
    f = np.bincount(2 * u + v, minlength=4) / u.size
    assert np.allclose(f, [0.57, 0.19, 0.19, 0.05], atol=4e-3)


def test_sort_unique_keys_matches_numpy():
    rng = np.random.default_rng(3)
    keys = W.edge_keys(rng.integers(0, 5000, 300000), rng.integers(0, 5000, 300000))
    got = W.sort_unique_keys(keys, 5000)
    assert np.array_equal(got, np.unique(keys))


def test_edge_set_pending_updates_match_a_python_set():
    rng = np.random.default_rng(9)
    src, dst = rng.integers(0, 300, 4000), rng.integers(0, 300, 4000)
    es = W.EdgeSet(src, dst)
    model = set(W.edge_keys(src, dst).tolist())
    for _ in range(30):
        present = np.array(sorted(model), np.uint64)
        dels = rng.choice(present, 40, replace=False)
        cand = W.edge_keys(rng.integers(0, 300, 200), rng.integers(0, 300, 200))
        ins = np.unique(cand[~np.isin(cand, present)])[:40]
        if rng.random() < 0.3:  # re-insert some of the deleted keys in the same call
            ins = np.union1d(ins, dels[:5])
        es.apply(ins, dels)
        model -= set(dels.tolist())
        model |= set(ins.tolist())
        probe = np.concatenate([cand, dels, ins])
        assert np.array_equal(es.contains(probe), np.isin(probe, np.array(sorted(model), np.uint64)))
        assert es.size == len(model)
        drawn = es.draw_present(rng, 500)
        assert np.isin(drawn, np.array(sorted(model), np.uint64)).all()
    assert es.keys.tolist() == sorted(model)
