"""Several seeds (the n x Sp seed block) against the FP64 CPU oracle, one oracle
run per seed, in lock-step: the oracle replays each seed's own step count.

Tolerances: FP64 L1 <= 1e-10, FP32_ACC64 and BF16_ACC64 L1 <= 1e-5 per seed.
bf16 gather rows reach the float tolerance because of error feedback: if z_i
is the stored row and e_i = (x_i s + e_(i-1)) - z_i the residual carried to
the next step, the stored values sum to the exact ones minus e_k, so after k
steps the scores miss only sum_(j<=k) M^(k+1-j) e_j (M the propagation
operator, ||M||_1 <= 1-c): each residual is damped by the steps after it
instead of piling up, at most 2^-9 (k+1) (1-c)^(k+1) ||q_offset||_1 when
||x_j||_1 <= (1-c)^j ||q_offset||_1. Without the feedback the bound is
2^-9 (1-c) ||q_offset||_1 / c^2, far above 1e-5 for these batches.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_00595_gb300 import native as N
from paper_1712_00595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C_RESTART = 0.15
TOL = {N.OSP_PREC_FP64: 1e-10, N.OSP_PREC_FP32_ACC64: 1e-5, N.OSP_PREC_BF16_ACC64: 1e-5}


def l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).sum())


def hub_graph(rng, n, m, hub_in, hub_out, mids):
    """Uniform edges, one in-list longer than 1024 (summed in pieces), one long
    out-list and some mid-size in-lists."""
    src = list(rng.integers(0, n, m))
    dst = list(rng.integers(0, n, m))
    src += list(rng.choice(n, hub_in, replace=False))
    dst += [1] * hub_in
    src += [2] * hub_out
    dst += list(rng.choice(n, hub_out, replace=False))
    for _ in range(mids):
        v = int(rng.integers(3, n))
        cnt = min(int(rng.integers(33, 600)), n - 1)
        src += list(rng.choice(n, cnt, replace=False))
        dst += [v] * cnt
    s = np.array(src, np.int32)
    d = np.array(dst, np.int32)
    keep = s != d
    return s[keep], d[keep]


def make_engine(prec, n, src, dst, seeds, eps, **kw):
    eng = N.Engine(precision=prec, device=0, **kw)
    eng.load_graph(n, src, dst)
    eng.set_seeds(np.asarray(seeds, np.int32), C_RESTART)
    eng.init_scores(eps)
    return eng


def check_graph(eng, g):
    ptr, idx = eng.export_graph(0)
    rp, col = g.csr()
    assert np.array_equal(ptr, rp) and np.array_equal(idx, col)
    ptr, idx = eng.export_graph(1)
    cp, row = g.csc()
    assert np.array_equal(ptr, cp) and np.array_equal(idx, row)


GATHERS = [N.SEED_GATHER_REGISTERS, N.SEED_GATHER_BULK]


@pytest.mark.parametrize("gather", GATHERS)
@pytest.mark.parametrize("S", [5, 40, 100, 256])
@pytest.mark.parametrize("prec", [N.OSP_PREC_FP64, N.OSP_PREC_FP32_ACC64])
def test_multi_cpi_lockstep(prec, S, gather):
    rng = np.random.default_rng(100 + S)
    n = 1200
    src, dst = hub_graph(rng, n, 9000, 1100, 500, 6)
    seeds = rng.permutation(n)[:S].astype(np.int32)
    eps = 1e-10
    eng = make_engine(prec, n, src, dst, seeds, eps, seed_gather=gather)
    iters, q, last = eng.get_seed_stats()
    assert iters.size == S and np.all(iters >= 1)
    assert np.allclose(q, C_RESTART, rtol=1e-12)  # ||x(0)||_1 = c for CPI
    csr = O.Graph(n, src, dst).csr()
    for j, s in enumerate(seeds):
        r_o, st, _ = O.cpi(*csr, int(s), C_RESTART, eps, force_iters=int(iters[j]))
        assert l1(eng.query(j), r_o) <= TOL[prec], (j, s)
        if prec == N.OSP_PREC_FP64:
            _, st_free, _ = O.cpi(*csr, int(s), C_RESTART, eps)
            assert abs(st_free["iterations"] - int(iters[j])) <= 1
    eng.close()


@pytest.mark.parametrize("gather", GATHERS)
@pytest.mark.parametrize("prec", [N.OSP_PREC_FP64, N.OSP_PREC_FP32_ACC64, N.OSP_PREC_BF16_ACC64])
def test_multi_osp_sequence_all_op_kinds(prec, gather):
    rng = np.random.default_rng(7 + prec)
    n = 1200
    src, dst = hub_graph(rng, n, 8000, 1100, 300, 5)
    S = 40
    seeds = rng.permutation(n)[:S].astype(np.int32)
    es = W.EdgeSet(src, dst)
    dead = np.zeros(n + 6 * 120 + 8, np.uint8)
    nn = n
    batches = []
    for _ in range(6):
        # row zeroings (Sec. 3.4.1 read literally) too, seeds included
        ops, nn = W.random_mixed_batch(rng, nn, es, dead, 120, protect=tuple(int(s) for s in seeds),
                                       p_zero_row=0.03)
        batches.append(ops)
    eps = 1e-12 if prec == N.OSP_PREC_FP64 else 1e-9
    eng = make_engine(prec, n, src, dst, seeds, 1e-12, max_nodes=n + 4096, seed_gather=gather)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    it0, _, _ = eng.get_seed_stats()
    r_o = [O.cpi(*cur, int(s), C_RESTART, 1e-12, force_iters=int(it0[j]))[0]
           for j, s in enumerate(seeds)]
    tol = TOL[prec]
    for j in range(S):
        assert l1(eng.query(j), r_o[j]) <= tol
    for ops in batches:
        st = eng.apply_updates(ops, eps)
        assert g.apply(ops, protect=tuple(int(s) for s in seeds)) == -1
        new = g.csr()
        iters, q, _ = eng.get_seed_stats()
        assert st["iterations"] == int(iters.max())
        for j in range(S):
            r_o[j], qv, _, _ = O.osp(cur, new, r_o[j], C_RESTART, eps, force_iters=int(iters[j]))
            # ||q||_1 differs by at most ||(1-c)(B~^T - A~^T) dr||_1 <= 2 (1-c) ||dr||_1
            # (dr = the error r_old already carries) plus rounding
            qn = np.abs(qv).sum()
            assert abs(q[j] - qn) <= 2 * (1 - C_RESTART) * tol + 1e-6 * qn + 1e-15
            assert l1(eng.query(j), r_o[j]) <= tol, (j, l1(eng.query(j), r_o[j]))
        cur = new
    check_graph(eng, g)
    eng.close()


def test_multi_seed_iterations_fixed_per_seed():
    rng = np.random.default_rng(11)
    n = 800
    src, dst = hub_graph(rng, n, 6000, 0, 200, 3)
    seeds = np.array([0, 10, 20, 30, 40], np.int32)
    eng = make_engine(N.OSP_PREC_FP32_ACC64, n, src, dst, seeds, 1e-10)
    want = np.array([1, 3, 7, 2, 5], np.int32)
    eng.set_seed_iterations(want)
    stream = W.edge_update_stream(src, dst, n, 2, 30, 20, seed=5)
    st = eng.apply_updates(stream[0], 1e-3)
    iters, _, _ = eng.get_seed_stats()
    assert np.array_equal(iters, want) and st["iterations"] == 7
    eng.set_seed_iterations(None)  # back to each seed's eps rule
    eng.apply_updates(stream[1], 1e-3)
    iters, _, last = eng.get_seed_stats()
    assert np.all(iters >= 1) and np.all(last <= 1e-3)
    eng.close()


def test_multi_query_topk_columns():
    rng = np.random.default_rng(8)
    n = 3000
    src = [0] * 700 + list(rng.integers(701, n, 8000)) + [5, 9]
    dst = list(range(1, 701)) + list(rng.integers(701, n, 8000)) + [801, 802]
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    seeds = np.array([0, 5, 1234], np.int32)
    for order in (0, 1):
        eng = make_engine(N.OSP_PREC_FP64, n, src, dst, seeds, 1e-13, node_order=order)
        csr = O.Graph(n, src, dst).csr()
        for j, s in enumerate(seeds):
            r = eng.query(j)
            r_o, _, _ = O.cpi(*csr, int(s), C_RESTART, 1e-13)
            assert l1(r, r_o) <= 1e-10
            assert np.allclose(eng.query(j, normalize=True), O.normalize(r), rtol=1e-12, atol=0)
            for k in (1, 100, 701, 4096):
                ids, sc = eng.topk(k, seed_idx=j)
                want_ids, want_sc = O.topk(r, k)
                assert np.array_equal(ids, want_ids) and np.array_equal(sc, want_sc)
        eng.close()


def test_multi_rejects_bad_seed_sets_and_seed_deletion():
    rng = np.random.default_rng(3)
    n = 200
    src, dst = W.er_graph(n, 1500, 3)
    eng = N.Engine(precision=N.OSP_PREC_FP64, device=0)
    eng.load_graph(n, src, dst)
    for bad in ([1, 2, 1], list(range(257)), [5, n]):
        with pytest.raises(N.OspError) as e:
            eng.set_seeds(np.array(bad, np.int32), C_RESTART)
        assert e.value.status == N.OSP_EINVAL
    eng.set_seeds(np.array([3, 7, 11], np.int32), C_RESTART)
    eng.init_scores(1e-12)
    r0 = [eng.query(j) for j in range(3)]
    ops = np.empty(2, W.UPDATE_DTYPE)
    ops["u"], ops["v"], ops["op"] = [4, 7], [5, 0], [0, 3]  # second op deletes seed 7
    st = eng.apply_updates(ops, 1e-12, allow=(N.OSP_EINVAL,))
    assert eng.last_status == N.OSP_EINVAL and st["bad_op"] == 1
    for j in range(3):
        assert np.array_equal(eng.query(j), r0[j])
    with pytest.raises(N.OspError):
        eng.query(3)
    eng.close()
    e16 = N.Engine(precision=N.OSP_PREC_BF16_ACC64, device=0)
    e16.load_graph(n, src, dst)
    with pytest.raises(N.OspError) as e:
        e16.set_seeds(np.array([3], np.int32), C_RESTART)
    assert e.value.status == N.OSP_ENOTSUP
    e16.close()


@pytest.mark.parametrize("workload,log2n", [("chunglu22_s64", 22), ("rmat24_s256", 21)])
def test_seed_block_workloads_residual_certificate(workload, log2n):
    """The seed-block workloads of the benchmark (generators and precisions as
    bench.py runs them; Chung-Lu at full size, R-MAT at 2^21 nodes) through
    every batch, with the oracle's graph updated by the same batches. For
    sampled seeds the FP64 residual rho = c e_s - (I - (1-c) B~^T) r of the
    engine's final scores, computed by the oracle on its own graph, bounds
    ||r - r*||_1 <= ||rho||_1 / c. In exact arithmetic the initial CPI leaves
    a residual of at most (1-c) eps_init and each batch adds at most
    (1-c) eps (its untaken tail x(k+1), reading c5); rounding may add at most
    c 1e-5, so that the rounding part of ||r - r*||_1 stays within 1e-5."""
    import bench

    cfg, n, src, dst, seeds, stream, _ = bench.make_multi_workload(workload, log2n)
    prec = {"fp32": N.OSP_PREC_FP32_ACC64, "bf16": N.OSP_PREC_BF16_ACC64}[cfg["precision"]]
    eps, eps_init = cfg["eps"], 1e-8
    eng = make_engine(prec, n, src, dst, seeds, eps_init, use_graphs=True, node_order=1)
    g = O.Graph(n, src, dst)
    protect = tuple(int(x) for x in seeds)
    for ops in stream:
        eng.apply_updates(ops, eps)
        assert g.apply(ops, protect=protect) == -1
    rp, col = g.csr()
    bound = (1 - C_RESTART) * (eps_init + len(stream) * eps) + C_RESTART * 1e-5
    got = eng.get_residual_bounds()
    for j in np.linspace(0, len(seeds) - 1, 6).astype(int):
        rho = O.residual_l1(rp, col, int(seeds[j]), C_RESTART, eng.query(int(j)))
        assert rho <= bound, (j, rho, bound)
        # the engine's own bound (exact-arithmetic part) covers the residual too
        assert rho <= got[j] + C_RESTART * 1e-5, (j, rho, got[j])
    eng.close()


def test_bf16_seed_block_lockstep_on_the_benchmark_workload():
    """The R-MAT 256-seed workload at 2^17 nodes, every batch (node insertions
    with out-edges, node deletions, edge edits) in bf16, against the oracle
    replaying each sampled seed's step counts: L1 <= 1e-5 per seed after every
    batch."""
    import bench

    cfg, n, src, dst, seeds, stream, _ = bench.make_multi_workload("rmat24_s256", 17)
    eps, eps_init = cfg["eps"], 1e-8
    eng = make_engine(N.OSP_PREC_BF16_ACC64, n, src, dst, seeds, eps_init, node_order=1)
    it0, _, _ = eng.get_seed_stats()
    g = O.Graph(n, src, dst)
    cur = g.csr()
    outdeg = np.diff(cur[0])
    live = [j for j in range(len(seeds)) if outdeg[seeds[j]] > 0]
    # eight live seeds spread over the column order (several column groups;
    # bf16 batches pack their columns into groups by offset size)
    sample = [live[i] for i in np.linspace(0, len(live) - 1, 8).astype(int)]
    r_o = {j: O.cpi(*cur, int(seeds[j]), C_RESTART, eps_init, force_iters=int(it0[j]))[0]
           for j in sample}
    protect = tuple(int(x) for x in seeds)
    worst = 0.0
    for ops in stream:
        eng.apply_updates(ops, eps)
        assert g.apply(ops, protect=protect) == -1
        new = g.csr()
        iters, _, _ = eng.get_seed_stats()
        for j in sample:
            r_o[j], _, _, _ = O.osp(cur, new, r_o[j], C_RESTART, eps, force_iters=int(iters[j]))
            err = l1(eng.query(j), r_o[j])
            worst = max(worst, err)
            assert err <= 1e-5, (j, err)
        cur = new
    eng.close()
