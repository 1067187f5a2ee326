"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances: FP64 path L1 <= 1e-10; FP32-products / FP64-accumulation path
L1 <= 1e-5 against the oracle replaying the same iteration counts (lock-step).
The graph store is compared bit for bit.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_00595_gb300 import native as N
from paper_1712_00595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C_RESTART = 0.15
TOL = {N.OSP_PREC_FP64: 1e-10, N.OSP_PREC_FP32_ACC64: 1e-5}
PRECS = [N.OSP_PREC_FP64, N.OSP_PREC_FP32_ACC64]


def l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).sum())


def engine(prec, n, src, dst, seed=0, c=C_RESTART, eps_init=1e-13, **kw):
    eng = N.Engine(precision=prec, device=0, **kw)
    eng.load_graph(n, src, dst)
    eng.set_seeds([seed], c)
    st = eng.init_scores(eps_init)
    return eng, st


def hub_graph(rng, n=6000, m=40000, hub_in=5000, hub_out=3000, mids=40):
    """Uniform edges plus one column of in-degree > 2048 (pull hub pieces), one
    row of out-degree > 32 x 32 (heavy push row) and mid-size lists."""
    src = list(rng.integers(0, n, m))
    dst = list(rng.integers(0, n, m))
    src += list(rng.choice(n, hub_in, replace=False))
    dst += [1] * hub_in
    src += [2] * hub_out
    dst += list(rng.choice(n, hub_out, replace=False))
    for k in range(mids):
        v = int(rng.integers(3, n))
        cnt = min(int(rng.integers(33, 1500)), n - 1)
        src += list(rng.choice(n, cnt, replace=False))
        dst += [v] * cnt
    s = np.array(src, np.int32)
    d = np.array(dst, np.int32)
    keep = s != d
    return s[keep], d[keep]


def check_graph(eng, g):
    ptr, idx = eng.export_graph(0)
    rp, col = g.csr()
    assert np.array_equal(ptr, rp) and np.array_equal(idx, col), "out-lists differ"
    ptr, idx = eng.export_graph(1)
    cp, row = g.csc()
    assert np.array_equal(ptr, cp) and np.array_equal(idx, row), "in-lists differ"
    assert eng.get_size() == (g.n, g.m)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PRECS)
def test_cpi_matches_oracle(prec):
    rng = np.random.default_rng(1)
    for src, dst, n in [(*W.er_graph(2000, 16000, 11), 2000), (*hub_graph(rng), 6000)]:
        eng, st = engine(prec, n, src, dst, seed=5, eps_init=1e-12)
        rp, col = O.Graph(n, src, dst).csr()
        r_o, ost, hist = O.cpi(rp, col, 5, C_RESTART, 1e-12)
        assert abs(st["iterations"] - ost["iterations"]) <= 1
        if st["iterations"] != ost["iterations"]:
            r_o, ost, hist = O.cpi(rp, col, 5, C_RESTART, 1e-12, force_iters=st["iterations"])
        assert l1(eng.query(), r_o) <= TOL[prec]
        h = eng.get_l1_history()
        assert h.size == st["iterations"] + 1
        # CPI vectors are nonnegative, so relative errors compose step by step.
        # A GPU step rounds the stored gather value, the scale and its product
        # once each and sums an in-list with a per-lane depth of at most
        # 1024 / 32 terms plus a 5-level warp reduction: at most 40 u per entry
        # (u = 2^-24 for FP32, 2^-53 for FP64). The oracle's step adds each
        # in-edge into its target in turn: at most (d_in + 2) 2^-53 per entry.
        # After i steps ||x(i)||_1 differs by at most (1 + delta)^i - 1 relative,
        # plus the rounding of the two FP64 norm sums over n entries, 2 n 2^-53.
        u = 2.0 ** -24 if prec else 2.0 ** -53
        d_in = int(np.bincount(col, minlength=n).max())
        delta = 40 * u + (d_in + 2) * 2.0 ** -53
        rtol = (1.0 + delta) ** np.arange(h.size) - 1.0 + 2 * n * 2.0 ** -53
        assert np.all(np.abs(h - hist) <= rtol * hist), (np.abs(h - hist) / hist).max()
        eng.close()


def test_cpi_iteration_count_116_on_gpu():
    # Table 2: CPI with c = 0.15, eps = 1e-9 runs 116 iterations on any dead-end free graph.
    rng = np.random.default_rng(7)
    n = 5000
    src = np.concatenate([np.arange(n), rng.integers(0, n, 40000)]).astype(np.int32)
    dst = np.concatenate([(np.arange(n) + 1) % n, rng.integers(0, n, 40000)]).astype(np.int32)
    for prec in PRECS:
        eng, st = engine(prec, n, src, dst, seed=3, eps_init=1e-9)
        assert st["iterations"] == 116
        eng.close()


def test_cpi_matches_dense_closed_form():
    rng = np.random.default_rng(2)
    for trial in range(4):
        n = int(rng.integers(5, 60))
        A = rng.random((n, n)) < 0.08
        src, dst = [a.astype(np.int32) for a in np.nonzero(A)]
        eng, _ = engine(N.OSP_PREC_FP64, n, src, dst, seed=0, eps_init=1e-15)
        want = O.dense_rwr(n, src, dst, 0, C_RESTART)
        assert l1(eng.query(), want) < 1e-12
        assert l1(eng.query(normalize=True), O.normalize(want)) < 1e-12
        eng.close()


# ---------------------------------------------------------------------------
def mixed_sequence(rng, n, src, dst, batches, n_ops, seed=0, p_zero_row=0.0):
    es = W.EdgeSet(src, dst)
    dead = np.zeros(n + batches * n_ops + 8, np.uint8)
    nn = n
    out = []
    for _ in range(batches):
        ops, nn = W.random_mixed_batch(rng, nn, es, dead, n_ops, protect=(seed,),
                                       p_zero_row=p_zero_row)
        out.append(ops)
    return out


@pytest.mark.parametrize("zero_rows", [False, True])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
def test_osp_sequence_with_all_op_kinds(prec, order, zero_rows):
    # zero_rows: batches also hold OSP_OP_ZERO_ROW (the literal node deletion of
    # Sec. 3.4.1), on the seed too, with edges re-inserted after it
    rng = np.random.default_rng(40 + prec + 100 * zero_rows)
    n = 400
    src, dst = hub_graph(rng, n=n, m=3000, hub_in=300, hub_out=200, mids=5)
    batches = mixed_sequence(rng, n, src, dst, 6, 150, p_zero_row=0.04 if zero_rows else 0.0)
    eps = 1e-12
    eng, _ = engine(prec, n, src, dst, eps_init=eps, max_nodes=n + 4096, node_order=order)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r_o, _, _ = O.cpi(*cur, 0, C_RESTART, eps)
    for ops in batches:
        st = eng.apply_updates(ops, eps)
        assert g.apply(ops, protect=(0,)) == -1
        new = g.csr()
        check_graph(eng, g)
        # net counts: edges the batch added and removed, from the edge sets
        old_set = set(zip(np.repeat(np.arange(cur[0].size - 1), np.diff(cur[0])).tolist(),
                          cur[1].tolist()))
        new_set = set(zip(np.repeat(np.arange(new[0].size - 1), np.diff(new[0])).tolist(),
                          new[1].tolist()))
        assert st["net_inserts"] == len(new_set - old_set)
        assert st["net_deletes"] == len(old_set - new_set)
        force = st["iterations"] if prec == N.OSP_PREC_FP32_ACC64 else 0
        r_o, q, ost, _ = O.osp(cur, new, r_o, C_RESTART, eps, force_iters=force)
        cur = new
        if prec == N.OSP_PREC_FP64:
            assert abs(st["iterations"] - ost["iterations"]) <= 1
        assert st["qoff_l1"] == pytest.approx(np.abs(q).sum(), rel=1e-6, abs=1e-15)
        assert l1(eng.query(), r_o) <= TOL[prec]
    # Theorem 2: the tracked scores equal a recompute on the final graph
    r_cpi, _, _ = O.cpi(*cur, 0, C_RESTART, 1e-14)
    assert l1(eng.query(), r_cpi) <= TOL[prec] + 1e-9
    eng.close()


@pytest.mark.parametrize("prec", PRECS)
def test_dense_offset_scan_then_push_steps(prec):
    """A batch whose changed rows could reach more than n/beta nodes makes the
    merge skip the frontier queue and x(0) is found by a dense scan; when the
    offset is in fact small (the long row belongs to a node with zero score) the
    scan's queue must drive push steps."""
    rng = np.random.default_rng(77)
    n = 5000
    src = rng.integers(0, 3000, 9000)
    dst = rng.integers(0, 3000, 9000)
    src = np.concatenate([src, [0, 0], np.full(1000, 4000)])  # 4000: unreachable, long row
    dst = np.concatenate([dst, [1, 2], rng.choice(3000, 1000, replace=False)])
    keep = src != dst
    src, dst = src[keep].astype(np.int32), dst[keep].astype(np.int32)
    eps = 1e-12
    eng, _ = engine(prec, n, src, dst, eps_init=eps)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r_o, _, _ = O.cpi(*cur, 0, C_RESTART, eps)
    assert r_o[4000] == 0.0
    nbr = int(dst[src == 0][0])
    for rows in ([(4000, 4500, 0), (0, 4999, 0)], [(4000, 4501, 0), (0, nbr, 1)]):
        arr = np.empty(len(rows), W.UPDATE_DTYPE)
        arr["u"], arr["v"], arr["op"] = np.array(rows).T
        st = eng.apply_updates(arr, 1e-9)
        assert g.apply(arr, protect=(0,)) == -1
        new = g.csr()
        force = st["iterations"]
        r_o, q, ost, _ = O.osp(cur, new, r_o, C_RESTART, 1e-9, force_iters=force)
        cur = new
        assert st["push_iterations"] >= 1
        assert st["qoff_l1"] == pytest.approx(np.abs(q).sum(), rel=1e-6, abs=1e-15)
        assert l1(eng.query(), r_o) <= TOL[prec]
    eng.close()


@pytest.mark.parametrize("seeds", [[0], [0, 17, 99, 250]])
def test_graph_replay_matches_eager_launches(seeds):
    """The same batches through CUDA-graph replays (several batch-size buckets,
    a change of eps, a fixed step count) and through eager launches agree with
    each other and with the oracle."""
    rng = np.random.default_rng(55)
    n = 400
    src, dst = hub_graph(rng, n=n, m=3000, hub_in=300, hub_out=200, mids=5)
    es = W.EdgeSet(src, dst)
    dead = np.zeros(n + 10 * 400 + 8, np.uint8)
    nn = n
    batches = []
    for k in (5, 150, 300, 17, 150, 1):
        ops, nn = W.random_mixed_batch(rng, nn, es, dead, k, protect=tuple(seeds), p_zero_row=0.03)
        batches.append(ops)
    engs = []
    for graphs in (False, True):
        e = N.Engine(precision=N.OSP_PREC_FP64, device=0, max_nodes=n + 4096, use_graphs=graphs)
        e.load_graph(n, src, dst)
        e.set_seeds(np.array(seeds, np.int32), C_RESTART)
        e.init_scores(1e-12)
        engs.append(e)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r_o = [O.cpi(*cur, s, C_RESTART, 1e-13)[0] for s in seeds]
    for b, ops in enumerate(batches):
        eps = 1e-12 if b != 3 else 1e-9
        if b == 4:
            for e in engs:
                e.set_fixed_iterations(6)
        sts = [e.apply_updates(ops, eps) for e in engs]
        if b == 4:
            for e in engs:
                e.set_fixed_iterations(0)
        assert sts[0]["iterations"] == sts[1]["iterations"]
        assert sts[0]["kernel_launches"] == sts[1]["kernel_launches"]
        assert g.apply(ops, protect=tuple(seeds)) == -1
        new = g.csr()
        for j, s in enumerate(seeds):
            a, c = engs[0].query(j), engs[1].query(j)
            assert l1(a, c) <= 1e-13
            if b < 3:  # exact mode until the eps change (later batches keep its truncation)
                r_o[j], _, _, _ = O.osp(cur, new, r_o[j], C_RESTART, 1e-13)
                assert l1(c, r_o[j]) <= 1e-10
        cur = new
    check_graph(engs[1], g)
    for e in engs:
        e.close()


@pytest.mark.parametrize("seeds", [[0], [0, 17, 99]])
def test_autotuned_schedule_gives_the_same_scores(seeds):
    rng = np.random.default_rng(66)
    n = 3000
    src, dst = hub_graph(rng, n=n, m=30000, hub_in=2500, hub_out=900, mids=12)
    stream = W.edge_update_stream(src, dst, n, 3, 60, 40, seed=9)
    out = []
    for tune in (False, True):
        e = N.Engine(precision=N.OSP_PREC_FP64, device=0, autotune=tune, use_graphs=tune)
        e.load_graph(n, src, dst)
        e.set_seeds(np.array(seeds, np.int32), C_RESTART)
        e.init_scores(1e-12)
        for ops in stream:
            e.apply_updates(ops, 1e-12)
        out.append(([e.query(j) for j in range(len(seeds))], e.get_schedule()))
        e.close()
    ti, thr, piece, nw = out[1][1]
    assert ti in (512, 1024, 2048) and thr == piece
    assert thr in ((256, 512, 1024) if len(seeds) > 1 else (512, 1024, 4096))
    assert nw in ((2, 4, 8) if len(seeds) > 1 else (1,))
    for a, b in zip(out[0][0], out[1][0]):
        assert l1(a, b) <= 1e-12


@pytest.mark.parametrize("seeds", [[0], [0, 5, 77, 310]])
def test_large_edge_batch_grouped_by_source_row(seeds):
    """A host batch of edge ops above osp_max_batch() is cut by source row: one
    row with more ops than a sub-batch holds (cut across sub-batches, order
    kept), re-insertions and deletions of the same edge in one batch, and
    random edits elsewhere. The graph equals the oracle's after the batch in
    the caller's order and the scores equal the oracle's OSP."""
    rng = np.random.default_rng(72)
    n = 30000
    src, dst = W.er_graph(n, 240000, 9)
    ops = []
    # row 3: 20,000 insertions, then half of them deleted again, then some re-inserted
    tgt = rng.choice(np.arange(4, n), 20000, replace=False)
    ops += [(3, int(v), W.OP_INSERT_EDGE) for v in tgt]
    ops += [(3, int(v), W.OP_DELETE_EDGE) for v in tgt[::2]]
    ops += [(3, int(v), W.OP_INSERT_EDGE) for v in tgt[::8]]
    es = set(zip(src.tolist(), dst.tolist()))
    for _ in range(30000):
        u, v = int(rng.integers(0, n)), int(rng.integers(0, n))
        if u == 3 or u == v:
            continue
        ops.append((u, v, W.OP_DELETE_EDGE if (u, v) in es and rng.random() < 0.7
                    else W.OP_INSERT_EDGE))
    order = rng.permutation(len(ops))
    batch = np.zeros(len(ops), W.UPDATE_DTYPE)
    for i, k in enumerate(order):  # interleave the rows, keeping row 3's own order
        batch[i] = ops[k]
    r3 = np.flatnonzero(batch["u"] == 3)
    batch[r3] = np.array([o for o in ops if o[0] == 3], dtype=W.UPDATE_DTYPE)
    assert batch.size > 3 * 16384
    prec = N.OSP_PREC_FP64
    eng = N.Engine(precision=prec, device=0)
    eng.load_graph(n, src, dst)
    eng.set_seeds(np.array(seeds, np.int32), C_RESTART)
    eng.init_scores(1e-13)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    st = eng.apply_updates(batch, 1e-13)
    assert g.apply(batch, protect=tuple(seeds)) == -1
    new = g.csr()
    check_graph(eng, g)
    for j, s in enumerate(seeds):
        r_o, _, _ = O.cpi(*cur, s, C_RESTART, 1e-13)
        r_o, _, _, _ = O.osp(cur, new, r_o, C_RESTART, 1e-13)
        assert l1(eng.query(j), r_o) <= 1e-10
    eng.close()


def test_large_batch_in_sub_batches():
    """A batch above osp_max_batch() is merged in sub-batches against the same
    r_old with one propagation: exact OSP of the whole batch. An invalid op in a
    later sub-batch leaves the earlier sub-batches applied and propagated."""
    rng = np.random.default_rng(71)
    n = 3000
    src, dst = hub_graph(rng, n=n, m=60000, hub_in=2500, hub_out=900, mids=12)
    gen = np.random.default_rng(5)
    sampler = lambda k: (gen.integers(0, n, k), gen.integers(0, n, k))  # noqa: E731
    big = W.sized_update_stream(src, dst, n, [40000, 40000], 3, sampler)
    eng, _ = engine(N.OSP_PREC_FP64, n, src, dst, eps_init=1e-13)
    assert eng._L.osp_max_batch() == 16384
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r_o, _, _ = O.cpi(*cur, 0, C_RESTART, 1e-13)
    st = eng.apply_updates(big[0], 1e-13)
    assert g.apply(big[0], protect=(0,)) == -1
    new = g.csr()
    r_o, q, _, _ = O.osp(cur, new, r_o, C_RESTART, 1e-13)
    assert st["qoff_l1"] == pytest.approx(np.abs(q).sum(), rel=1e-9, abs=1e-15)
    check_graph(eng, g)
    assert l1(eng.query(), r_o) <= 1e-10
    cur = new
    bad = big[1].copy()
    bad[35000] = (0, n + 100, 0)  # insert to a node that does not exist
    st = eng.apply_updates(bad, 1e-13, allow=(N.OSP_EINVAL,))
    assert eng.last_status == N.OSP_EINVAL and st["bad_op"] == 35000
    done = 2 * 16384  # the two sub-batches before the one holding op 35000
    assert g.apply(bad[:done], protect=(0,)) == -1
    new = g.csr()
    r_o, _, _, _ = O.osp(cur, new, r_o, C_RESTART, 1e-13)
    check_graph(eng, g)
    assert l1(eng.query(), r_o) <= 1e-10
    eng.close()


@pytest.mark.parametrize("prec", PRECS)
def test_pagerank_mode_uniform_restart(prec):
    """seed = OSP_PAGERANK: q uniform over the nodes at osp_set_seeds, fixed
    afterwards. CPI and OSP through all op kinds match the oracle run from
    x(0) = c q; at the end, a recompute on the final graph with the same q."""
    rng = np.random.default_rng(90 + prec)
    n = 500
    src, dst = hub_graph(rng, n=n, m=4000, hub_in=400, hub_out=250, mids=5)
    batches = mixed_sequence(rng, n, src, dst, 4, 120)
    eps = 1e-12
    eng = N.Engine(precision=prec, device=0, max_nodes=n + 4096)
    eng.load_graph(n, src, dst)
    eng.set_seeds([-1], C_RESTART)
    st = eng.init_scores(eps)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    force = st["iterations"] if prec == N.OSP_PREC_FP32_ACC64 else 0
    r_o, _, _ = O.propagate(*cur, np.full(n, C_RESTART / n), C_RESTART, eps, force_iters=force)
    assert l1(eng.query(), r_o) <= TOL[prec]
    for ops in batches:
        st = eng.apply_updates(ops, eps)
        assert g.apply(ops) == -1
        new = g.csr()
        force = st["iterations"] if prec == N.OSP_PREC_FP32_ACC64 else 0
        r_o, _, _, _ = O.osp(cur, new, r_o, C_RESTART, eps, force_iters=force)
        cur = new
        assert l1(eng.query(), r_o) <= TOL[prec]
    q = np.zeros(g.n)
    q[:n] = 1.0 / n
    r_cpi, _, _ = O.propagate(*cur, C_RESTART * q, C_RESTART, 1e-14)
    assert l1(eng.query(), r_cpi) <= TOL[prec] + 1e-9
    eng.close()


def test_invalid_batches_rejected_state_unchanged():
    rng = np.random.default_rng(9)
    n = 50
    src, dst = W.er_graph(n, 300, 5)
    eng, _ = engine(N.OSP_PREC_FP64, n, src, dst)
    r0 = eng.query()
    g0 = eng.export_graph(0)
    g = O.Graph(n, src, dst)
    cases = [
        [(0, 99, 0)],
        [(0, 0, 2), (0, 50, 0), (0, 51, 0)],
        [(7, 0, 3), (1, 7, 0)],
        [(7, 0, 3), (7, 0, 3)],
        [(0, 0, 3)],
        [(0, 1, 9)],
        [(3, 4, 0), (-1, 2, 1)],
    ]
    for rows in cases:
        ops = np.array(rows, dtype=np.int64)
        arr = np.empty(len(rows), W.UPDATE_DTYPE)
        arr["u"], arr["v"], arr["op"] = ops[:, 0], ops[:, 1], ops[:, 2]
        want = g.validate(arr, protect=(0,))
        assert want >= 0
        st = eng.apply_updates(arr, 1e-12, allow=(N.OSP_EINVAL,))
        assert eng.last_status == N.OSP_EINVAL and st["bad_op"] == want
        assert eng.get_size() == (n, g.m)
        p, i = eng.export_graph(0)
        assert np.array_equal(p, g0[0]) and np.array_equal(i, g0[1])
        assert np.array_equal(eng.query(), r0)
    # the context still works afterwards
    ok = np.zeros(1, W.UPDATE_DTYPE)
    ok[0] = (3, 4, 0)
    eng.apply_updates(ok, 1e-12)
    eng.close()


def test_invalid_bad_op_index_reported():
    src, dst = W.er_graph(30, 100, 3)
    eng, _ = engine(N.OSP_PREC_FP64, 30, src, dst)
    arr = np.zeros(5, W.UPDATE_DTYPE)
    arr[:] = [(1, 2, 0), (2, 3, 0), (4, 5, 1), (40, 1, 0), (1, 3, 0)]
    st = eng.apply_updates(arr, 1e-12, allow=(N.OSP_EINVAL,))
    assert eng.last_status == N.OSP_EINVAL and st["bad_op"] == 3
    eng.close()


def test_config1_er_exact_osp():
    # ER 10,000 nodes / 100,000 edges, seed 0, c = 0.15, eps = 1e-12, one batch
    # of 50 insertions of absent edges and 50 deletions of existing edges.
    n, m, eps = 10000, 100000, 1e-12
    src, dst = W.er_graph(n, m, W.BASE_SEED + 1)
    ops = W.edge_update_stream(src, dst, n, 1, 50, 50, seed=W.BASE_SEED + 101)[0]
    eng, _ = engine(N.OSP_PREC_FP64, n, src, dst, eps_init=eps)
    st = eng.apply_updates(ops, eps)
    g = O.Graph(n, src, dst)
    old = g.csr()
    assert g.apply(ops) == -1
    check_graph(eng, g)
    r0, _, _ = O.cpi(*old, 0, C_RESTART, eps)
    r1, q, ost, _ = O.osp(old, g.csr(), r0, C_RESTART, eps)
    assert st["net_inserts"] == 50 and st["net_deletes"] == 50
    assert abs(st["iterations"] - ost["iterations"]) <= 1
    assert l1(eng.query(), r1) <= 1e-10
    r_cpi, _, _ = O.cpi(*g.csr(), 0, C_RESTART, 1e-15)
    assert l1(eng.query(), r_cpi) <= 1e-10
    eng.close()


@pytest.mark.parametrize("prec", PRECS)
def test_hub_lists_and_ospt_bounds(prec):
    rng = np.random.default_rng(77)
    n = 6000
    src, dst = hub_graph(rng, n=n)
    eps_init = 1e-13
    eng, _ = engine(prec, n, src, dst, seed=2, eps_init=eps_init)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r_o, _, _ = O.cpi(*cur, 2, C_RESTART, eps_init)
    es = W.EdgeSet(src, dst)
    for b, eps in enumerate([1e-4, 1e-8, 1e-12, 1e-6]):
        # touch the hub column, the heavy row and random rows
        ins = np.array([(int(rng.integers(n)) << 32) | 1 for _ in range(30)]
                       + [(2 << 32) | int(rng.integers(n)) for _ in range(30)], np.uint64)
        ins = np.unique(ins[~es.contains(ins)])
        ins = ins[(ins >> np.uint64(32)) != (ins & np.uint64(0xFFFFFFFF))]
        dels = es.keys[rng.choice(es.keys.size, 200, replace=False)]
        ops = W._pack(ins, dels, rng)
        es.apply(ins, dels)
        st = eng.apply_updates(ops, eps)
        assert g.apply(ops) == -1
        new = g.csr()
        r_o, q, ost, _ = O.osp(cur, new, r_o, C_RESTART, eps, force_iters=st["iterations"])
        cur = new
        check_graph(eng, g)
        assert l1(eng.query(), r_o) <= TOL[prec]
        ql1 = float(np.abs(q).sum())
        bound = 1 if ql1 <= eps else max(1, math.ceil(math.log(eps / ql1) / math.log(1 - C_RESTART)))
        assert 1 <= st["iterations"] <= bound + 1
    eng.close()


def test_empty_and_noop_batches_leave_scores():
    src, dst = W.er_graph(500, 4000, 21)
    eng, _ = engine(N.OSP_PREC_FP64, 500, src, dst)
    r0 = eng.query()
    st = eng.apply_updates(np.zeros(0, W.UPDATE_DTYPE), 1e-12)
    assert st["iterations"] == 1 and st["qoff_l1"] == 0.0
    assert np.array_equal(eng.query(), r0)
    ops = np.zeros(3, W.UPDATE_DTYPE)
    ops[0] = (int(src[0]), int(dst[0]), 0)  # insert existing
    have = set(zip(src.tolist(), dst.tolist()))
    absent = [(u, v) for u in range(5) for v in range(5, 60) if (u, v) not in have][:2]
    ops[1] = (absent[0][0], absent[0][1], 1)  # delete absent
    ops[2] = (absent[1][0], absent[1][1], 1)
    st = eng.apply_updates(ops, 1e-12)
    assert st["net_inserts"] == 0 and st["net_deletes"] == 0 and st["changed_rows"] == 0
    assert np.array_equal(eng.query(), r0)
    eng.close()


def test_dead_end_seed_and_new_nodes():
    src = np.array([1, 2, 3], np.int32)
    dst = np.array([0, 0, 1], np.int32)
    eng, st = engine(N.OSP_PREC_FP64, 4, src, dst, seed=0, max_nodes=64)
    r = eng.query()
    assert r[0] == C_RESTART and np.all(r[1:] == 0)
    ops = np.zeros(4, W.UPDATE_DTYPE)
    ops[:] = [(0, 0, 2), (4, 0, 0), (0, 4, 0), (0, 2, 0)]
    eng.apply_updates(ops, 1e-14)
    g = O.Graph(4, src, dst)
    assert g.apply(ops) == -1
    check_graph(eng, g)
    rp, col = g.csr()
    r_cpi, _, _ = O.cpi(rp, col, 0, C_RESTART, 1e-15)
    assert l1(eng.query(), r_cpi) < 1e-12
    eng.close()


def test_max_size_batch():
    n = 20000
    src, dst = W.er_graph(n, 120000, 33)
    U = N.Engine.max_batch()
    ops = W.edge_update_stream(src, dst, n, 1, U // 2, U - U // 2, seed=34)[0]
    assert ops.size == U
    eng, _ = engine(N.OSP_PREC_FP32_ACC64, n, src, dst, eps_init=1e-10)
    st = eng.apply_updates(ops, 1e-6)
    g = O.Graph(n, src, dst)
    old = g.csr()
    assert g.apply(ops) == -1
    check_graph(eng, g)
    r0, _, _ = O.cpi(*old, 0, C_RESTART, 1e-10)
    r1, _, _, _ = O.osp(old, g.csr(), r0, C_RESTART, 1e-6, force_iters=st["iterations"])
    assert l1(eng.query(), r1) <= 1e-5
    with pytest.raises(N.OspError):  # above what one call accepts (sub-batches included)
        eng.apply_updates(np.zeros(N.MAX_APPLY_OPS + 1, W.UPDATE_DTYPE), 1e-6)
    eng.close()


def test_pool_compaction_keeps_graph_exact():
    rng = np.random.default_rng(5)
    n = 3000
    src, dst = hub_graph(rng, n=n, m=15000, hub_in=2500, hub_out=2500, mids=4)
    eng, _ = engine(N.OSP_PREC_FP64, n, src, dst, seed=7, eps_init=1e-12)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r_o, _, _ = O.cpi(*cur, 7, C_RESTART, 1e-12)
    es = W.EdgeSet(src, dst)
    for b in range(60):  # the hub lists are rewritten every batch: the pool fills and compacts
        ins = np.array([(2 << 32) | int(x) for x in rng.integers(0, n, 20)]
                       + [(int(x) << 32) | 1 for x in rng.integers(0, n, 20)], np.uint64)
        ins = np.unique(ins[~es.contains(ins)])
        ins = ins[(ins >> np.uint64(32)) != (ins & np.uint64(0xFFFFFFFF))]
        dels = es.keys[rng.choice(es.keys.size, 40, replace=False)]
        ops = W._pack(ins, dels, rng)
        es.apply(ins, dels)
        eng.apply_updates(ops, 1e-12)
        assert g.apply(ops) == -1
        new = g.csr()
        r_o, _, _, _ = O.osp(cur, new, r_o, C_RESTART, 1e-12)
        cur = new
    check_graph(eng, g)
    assert l1(eng.query(), r_o) <= 1e-10
    eng.close()


def test_rmat20_bench_configuration_sampled():
    """The benchmark's workload at full size (R-MAT scale 20, 16.8M edges, seed of
    highest out-degree, batches of 600 insertions + 400 deletions), a few batches,
    both precisions against the oracle."""
    gen, src, dst = W.rmat_graph(20, 1 << 24, seed=W.BASE_SEED + 2)
    n = gen.n
    seed = W.max_out_degree_seed(n, src)
    stream = W.edge_update_stream(src, dst, n, 3, 600, 400, seed=W.BASE_SEED + 202,
                                  sampler=gen.sample)
    eps_init, eps = 1e-10, 1e-6
    g = O.Graph(n, src, dst)
    cur = g.csr()
    engs, chains = {}, {}
    for prec in PRECS:
        engs[prec], st0 = engine(prec, n, src, dst, seed=seed, eps_init=eps_init)
        chains[prec], _, _ = O.cpi(*cur, seed, C_RESTART, eps_init, force_iters=st0["iterations"])
        assert l1(engs[prec].query(), chains[prec]) <= TOL[prec]
    for ops in stream:
        assert g.apply(ops) == -1
        new = g.csr()
        for prec in PRECS:
            st = engs[prec].apply_updates(ops, eps)
            r_new, _, ost, _ = O.osp(cur, new, chains[prec], C_RESTART, eps,
                                     force_iters=st["iterations"])
            chains[prec] = r_new
            assert l1(engs[prec].query(), r_new) <= TOL[prec]
        cur = new
    ptr, idx = engs[N.OSP_PREC_FP32_ACC64].export_graph(1)
    cp, row = g.csc()
    assert np.array_equal(ptr, cp) and np.array_equal(idx, row)
    for e in engs.values():
        e.close()


@pytest.mark.parametrize("order", [0, 1])
def test_topk_matches_ranking_of_the_score_vector(order):
    rng = np.random.default_rng(8)
    # star with 700 equal-score leaves (ties), unreachable nodes (zero scores), random part
    n = 3000
    src = [0] * 700 + list(rng.integers(701, n, 8000))
    dst = list(range(1, 701)) + list(rng.integers(701, n, 8000))
    src += [5, 9]
    dst += [801, 802]
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    for seed in (0, 5):
        eng, _ = engine(N.OSP_PREC_FP64, n, src, dst, seed=seed, eps_init=1e-13, node_order=order)
        r = eng.query()
        for k in (1, 10, 100, 701, 1000, 4096):
            ids, sc = eng.topk(k)
            want_ids, want_sc = O.topk(r, k)
            assert np.array_equal(ids, want_ids), (seed, k)
            assert np.array_equal(sc, want_sc)
            ids_n, sc_n = eng.topk(k, normalize=True)
            assert np.array_equal(ids_n, want_ids)
            assert np.allclose(sc_n, want_sc / np.abs(r).sum(), rtol=1e-14, atol=0)
        eng.close()
    # fewer nodes than k
    eng, _ = engine(N.OSP_PREC_FP64, 7, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    ids, sc = eng.topk(20)
    want_ids, want_sc = O.topk(eng.query(), 20)
    assert ids.size == 7 and np.array_equal(ids, want_ids) and np.array_equal(sc, want_sc)
    eng.close()


def test_zero_rows_across_sub_batches():
    """Row zeroings (OSP_OP_ZERO_ROW) at and around the sub-batch boundaries of
    a large batch, with edge ops on the same rows before and after them: the
    graph and the scores equal the oracle's (exact mode)."""
    rng = np.random.default_rng(73)
    n = 3000
    src, dst = hub_graph(rng, n=n, m=60000, hub_in=2500, hub_out=900, mids=12)
    gen = np.random.default_rng(6)
    sampler = lambda k: (gen.integers(0, n, k), gen.integers(0, n, k))  # noqa: E731
    big = W.sized_update_stream(src, dst, n, [40000], 3, sampler)[0].copy()
    for p in (100, 16383, 16384, 20000, 32767, 32768, 39998):
        u = int(big["u"][p + 1]) if p + 1 < big.size else int(big["u"][p - 1])
        big[p] = (u, 0, W.OP_ZERO_ROW)
    big[16390] = (int(src[0]), 0, W.OP_ZERO_ROW)
    big[16391] = (int(src[0]), int(dst[0]), W.OP_INSERT_EDGE)  # re-inserted after the zeroing
    eng, _ = engine(N.OSP_PREC_FP64, n, src, dst, eps_init=1e-13)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r_o, _, _ = O.cpi(*cur, 0, C_RESTART, 1e-13)
    m0 = g.m
    st = eng.apply_updates(big, 1e-13)
    assert g.apply(big, protect=(0,)) == -1
    new = g.csr()
    check_graph(eng, g)
    old_set = set(zip(np.repeat(np.arange(n), np.diff(cur[0])).tolist(), cur[1].tolist()))
    new_set = set(zip(np.repeat(np.arange(n), np.diff(new[0])).tolist(), new[1].tolist()))
    # counted per sub-batch: an edge added by one sub-batch and removed by a
    # later one counts in both columns
    assert st["net_inserts"] - st["net_deletes"] == g.m - m0 and st["m_edges"] == g.m
    assert st["net_inserts"] >= len(new_set - old_set)
    assert st["net_deletes"] >= len(old_set - new_set)
    r_o, q, _, _ = O.osp(cur, new, r_o, C_RESTART, 1e-13)
    assert st["qoff_l1"] == pytest.approx(np.abs(q).sum(), rel=1e-9, abs=1e-15)
    assert l1(eng.query(), r_o) <= 1e-10
    eng.close()


@pytest.mark.parametrize("prec", PRECS)
def test_residual_bound_covers_the_oracle_residual(prec):
    """osp_batch_stats.residual_bound (Theorem 4, reading c5) bounds the FP64
    residual rho = c e_s - (I - (1-c) B~^T) r that the oracle computes on its own
    graph after the same batches, up to rounding (1e-10 for FP64, c 1e-5 for
    FP32); and it grows by (1-c) ||x(k)||_1 per call."""
    n = 3000
    src, dst = W.er_graph(n, 24000, 5)
    eng, st0 = engine(prec, n, src, dst, seed=9, eps_init=1e-6)
    assert st0["residual_bound"] == pytest.approx((1 - C_RESTART) * st0["last_x_l1"], rel=1e-12)
    g = O.Graph(n, src, dst)
    slack = 1e-10 if prec == N.OSP_PREC_FP64 else C_RESTART * 1e-5
    prev = st0["residual_bound"]
    for ops in W.edge_update_stream(src, dst, n, 4, 60, 40, seed=6):
        st = eng.apply_updates(ops, 1e-4)
        assert g.apply(ops, protect=(9,)) == -1
        assert st["residual_bound"] == pytest.approx(prev + (1 - C_RESTART) * st["last_x_l1"],
                                                     rel=1e-12)
        prev = st["residual_bound"]
        rho = O.residual_l1(*g.csr(), 9, C_RESTART, eng.query())
        assert rho <= st["residual_bound"] + slack, (rho, st["residual_bound"])
        assert np.allclose(eng.get_residual_bounds(), [st["residual_bound"]], rtol=0, atol=0)
    eng.close()


def test_hbm_budget_option():
    """osp_options.hbm_budget_bytes: a budget below what the graph store needs
    fails the load with OSP_ENOMEM and leaves nothing allocated; with a budget
    just above what load, seeds and scores take, query slots are admitted only
    while they fit, and the context's device bytes never exceed the budget."""
    n = 2000
    src, dst = W.er_graph(n, 16000, 4)
    seeds = np.arange(40, dtype=np.int32)

    def setup(budget):
        e = N.Engine(precision=N.OSP_PREC_FP32_ACC64, device=0, hbm_budget_bytes=budget)
        e.load_graph(n, src, dst)
        e.set_seeds(seeds, C_RESTART)
        e.init_scores(1e-8)
        return e

    e = N.Engine(precision=N.OSP_PREC_FP32_ACC64, device=0, hbm_budget_bytes=1 << 20)
    with pytest.raises(N.OspError) as err:
        e.load_graph(n, src, dst)
    assert err.value.status == N.OSP_ENOMEM
    assert e.device_bytes() == 0
    e.close()
    e = setup(0)  # no limit: what this setup takes
    used = e.device_bytes()
    e.query_slots(1)
    slot = e.device_bytes() - used
    e.close()
    budget = used + 2 * slot + slot // 2
    e = setup(budget)
    assert e.device_bytes() == used
    with pytest.raises(N.OspError) as err:
        e.query_slots(3)
    assert err.value.status == N.OSP_ENOMEM
    assert e.device_bytes() <= budget
    e.query_slots(2)
    assert e.device_bytes() == used + 2 * slot <= budget
    ids, _ = e.topk(10)
    assert ids.size == 10
    assert e.num_nodes() == n
    e.close()


@pytest.mark.parametrize("prec", PRECS)
def test_deterministic_mode_gives_the_same_bits(prec):
    """osp_options.deterministic: two contexts fed the same calls (a batch
    merged in three sub-batches, then mixed batches with node additions and
    deletions) agree bit for bit in the scores, the normalised scores, the
    per-step norms and the statistics; every step pulls; autotune is ignored;
    and the scores still match the oracle at the path's tolerance."""
    rng = np.random.default_rng(90 + prec)
    n = 3000
    src, dst = hub_graph(rng, n=n, m=60000, hub_in=2500, hub_out=900, mids=12)
    gen = np.random.default_rng(6)
    sampler = lambda k: (gen.integers(0, n, k), gen.integers(0, n, k))  # noqa: E731
    big = W.sized_update_stream(src, dst, n, [40000], 4, sampler)[0]
    g = O.Graph(n, src, dst)
    cur = g.csr()
    assert g.apply(big, protect=(0,)) == -1
    rp, col = g.csr()
    src2 = np.repeat(np.arange(rp.size - 1), np.diff(rp)).astype(np.int32)
    batches = [big] + mixed_sequence(rng, n, src2, col.astype(np.int32), 4, 150)
    g = O.Graph(n, src, dst)
    eps = 1e-12
    runs = []
    for _ in range(2):
        eng, st = engine(prec, n, src, dst, eps_init=eps, max_nodes=n + 4096,
                         deterministic=True, autotune=True)
        rec = []
        for ops in [None] + batches:
            if ops is not None:
                st = eng.apply_updates(ops, eps)
            st = {k: v for k, v in st.items() if not k.startswith("ms_")}
            assert st["push_iterations"] == 0
            rec.append((st, eng.query(), eng.query(normalize=True), eng.get_l1_history(),
                        eng.topk(50, normalize=True)))
        runs.append(rec)
        eng.close()
    for a, b in zip(*runs):
        assert a[0] == b[0]
        for x, y in zip(a[1:4], b[1:4]):
            assert x.shape == y.shape and np.array_equal(x.view(np.uint64), y.view(np.uint64))
        assert np.array_equal(a[4][0], b[4][0])
        assert np.array_equal(a[4][1].view(np.uint64), b[4][1].view(np.uint64))
    # parity of the first run with the oracle, batch by batch
    r_o, _, _ = O.cpi(*cur, 0, C_RESTART, eps)
    assert l1(runs[0][0][1], r_o) <= TOL[prec]
    for ops, (st, r, *_rest) in zip(batches, runs[0][1:]):
        assert g.apply(ops, protect=(0,)) == -1
        new = g.csr()
        force = st["iterations"] if prec == N.OSP_PREC_FP32_ACC64 else 0
        r_o, q, _, _ = O.osp(cur, new, r_o, C_RESTART, eps, force_iters=force)
        cur = new
        assert st["qoff_l1"] == pytest.approx(np.abs(q).sum(), rel=1e-6, abs=1e-15)
        assert l1(r, r_o) <= TOL[prec]


def test_deterministic_mode_is_for_one_seed():
    src, dst = W.er_graph(500, 4000, 2)
    eng = N.Engine(precision=N.OSP_PREC_FP64, device=0, deterministic=True)
    eng.load_graph(500, src, dst)
    with pytest.raises(N.OspError) as err:
        eng.set_seeds([0, 1], C_RESTART)
    assert err.value.status == N.OSP_ENOTSUP
    eng.close()
