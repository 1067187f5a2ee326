"""Pins for the FP64 CPU oracle, checked against what the paper and the
mathematics fix (closed forms, exact rationals, the paper's printed iteration
count, Theorems 2-5) rather than against the oracle itself."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_00595_gb300 import workloads as W

C_RESTART = 0.15
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = [s.strip() for s in line.split("=", 1)]
            parts = v.split()
            vals[k] = [float(p) for p in parts] if len(parts) > 1 else float(parts[0])
    return vals


def csr_from_edges(n, src, dst):
    g = O.Graph(n, np.asarray(src, np.int32), np.asarray(dst, np.int32))
    return g.csr()


def random_graph(rng, n, p, self_loops=True):
    A = rng.random((n, n)) < p
    if not self_loops:
        np.fill_diagonal(A, False)
    src, dst = np.nonzero(A)
    return src.astype(np.int32), dst.astype(np.int32)


def iter_bound(eps, q_l1, c):
    """Theorem 3: k <= ceil(log_{1-c}(eps / ||q||_1)), and the loop runs at least once."""
    if q_l1 <= eps:
        return 1
    return max(1, math.ceil(math.log(eps / q_l1) / math.log(1.0 - c)))


# ---------------------------------------------------------------------------
# The dense closed form itself (Eq. 1), pinned by hand-solved graphs
# ---------------------------------------------------------------------------
def exact_rwr_fraction(n, edges, seed, c):
    """Eq. 1 over the rationals (Gauss-Jordan with Fractions), independent of numpy."""
    c = Fraction(c).limit_denominator(10**6)
    deg = [0] * n
    for u, _ in edges:
        deg[u] += 1
    # M = I - (1-c) A~^T ;  M r = c e_s
    M = [[Fraction(int(i == j)) for j in range(n)] + [c if i == seed else Fraction(0)]
         for i in range(n)]
    for u, v in edges:
        M[v][u] -= (1 - c) / deg[u]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [x / pv for x in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    return [M[i][n] for i in range(n)]


def test_dense_directed_cycle_closed_form():
    # Directed cycle 0->1->...->L-1->0, seed 0: r_k = c (1-c)^k / (1 - (1-c)^L).
    L, c = 7, C_RESTART
    src = np.arange(L)
    dst = (src + 1) % L
    r = O.dense_rwr(L, src, dst, 0, c)
    want = np.array([c * (1 - c) ** k / (1 - (1 - c) ** L) for k in range(L)])
    assert np.abs(r - want).max() < 1e-15


def test_dense_complete_graph_closed_form():
    # K_n without self-loops, seed s: r_o = (1-c) r_s / (1 + c(n-2)), r_s = c + (1-c) r_o.
    n, c = 9, C_RESTART
    src, dst = np.nonzero(~np.eye(n, dtype=bool))
    r = O.dense_rwr(n, src, dst, 3, c)
    rs = c * (1 + c * (n - 2)) / (1 + c * (n - 2) - (1 - c) ** 2)
    ro = (1 - c) * rs / (1 + c * (n - 2))
    assert abs(r[3] - rs) < 1e-15
    assert np.abs(np.delete(r, 3) - ro).max() < 1e-15
    assert abs(r.sum() - 1.0) < 1e-14


def test_dense_star_dead_ends_leak():
    # seed -> k leaves, leaves are dead ends: r_seed = c, r_leaf = c (1-c) / k (mass leaks).
    k, c = 5, C_RESTART
    r = O.dense_rwr(k + 1, np.zeros(k, np.int32), np.arange(1, k + 1), 0, c)
    assert abs(r[0] - c) < 1e-16
    assert np.abs(r[1:] - c * (1 - c) / k).max() < 1e-16


def test_dense_matches_exact_rationals_asymmetric():
    # A small directed graph where a transposed A~ gives a different answer.
    edges = [(0, 1), (0, 2), (1, 2), (2, 0), (2, 3), (3, 3), (4, 0)]
    n = 5
    src = np.array([e[0] for e in edges])
    dst = np.array([e[1] for e in edges])
    exact = exact_rwr_fraction(n, edges, 0, 0.15)
    r = O.dense_rwr(n, src, dst, 0, 0.15)
    assert np.abs(r - np.array([float(x) for x in exact])).max() < 1e-15
    # transposing A~ gives a visibly different vector
    A = O.dense_matrix(n, src, dst)
    wrong = np.linalg.solve(np.eye(n) - 0.85 * A, 0.15 * np.eye(n)[0])
    assert np.abs(wrong - r).sum() > 1e-2


# ---------------------------------------------------------------------------
# CPI (Sec. 2.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("trial", range(6))
def test_cpi_matches_dense_solve(trial):
    rng = np.random.default_rng(100 + trial)
    n = int(rng.integers(3, 80))
    src, dst = random_graph(rng, n, float(rng.uniform(0.02, 0.3)))
    rp, col = csr_from_edges(n, src, dst)
    seed = int(rng.integers(n))
    r, st, hist = O.cpi(rp, col, seed, C_RESTART, 1e-15)
    want = O.dense_rwr(n, src, dst, seed, C_RESTART)
    assert np.abs(r - want).sum() <= 1e-15 * (1 - C_RESTART) / C_RESTART + 1e-13
    assert st["converged"]


def test_cpi_iteration_count_matches_paper_table2():
    # Table 2: CPI at c = 0.15, eps = 1e-9 runs 116 iterations. With no dead-ends
    # ||x(i)||_1 = c (1-c)^i exactly, whatever the graph.
    g = golden("paper_table2.txt")
    rng = np.random.default_rng(7)
    n = 300
    # dead-end free: every node has out-edge to its successor plus random edges
    src = np.concatenate([np.arange(n), rng.integers(0, n, 2000)]).astype(np.int32)
    dst = np.concatenate([(np.arange(n) + 1) % n, rng.integers(0, n, 2000)]).astype(np.int32)
    rp, col = csr_from_edges(n, src, dst)
    r, st, hist = O.cpi(rp, col, 5, g["cpi_c"], g["cpi_eps"])
    assert st["iterations"] == int(g["cpi_iterations"])
    i = np.arange(hist.size)
    assert np.allclose(hist, g["cpi_c"] * (1 - g["cpi_c"]) ** i, rtol=1e-12, atol=0)
    assert abs(r.sum() - 1.0) < 1e-8  # all mass kept, up to the truncated tail


def test_cpi_dead_end_seed():
    # A seed with no out-edges keeps exactly c.
    rp, col = csr_from_edges(4, [1, 2], [0, 0])
    r, st, _ = O.cpi(rp, col, 0, C_RESTART, 1e-12)
    assert r[0] == C_RESTART and np.all(r[1:] == 0) and st["iterations"] == 1


def test_cpi_force_iters_replays_exact_count():
    rng = np.random.default_rng(3)
    src, dst = random_graph(rng, 30, 0.1)
    rp, col = csr_from_edges(30, src, dst)
    r5, st5, h5 = O.cpi(rp, col, 0, C_RESTART, 1.0, force_iters=5)
    assert st5["iterations"] == 5 and h5.size == 6


# ---------------------------------------------------------------------------
# Graph updates (sequential semantics), pinned by a Python set implementation
# ---------------------------------------------------------------------------
def apply_python(n, edges, dead, ops, protect=()):
    edges, dead = set(edges), set(dead)
    for p, (u, v, op) in enumerate(ops.tolist()):
        if op in (0, 1):
            if not (0 <= u < n and 0 <= v < n) or u in dead or v in dead:
                return p
            if op == 0:
                edges.add((u, v))
            else:
                edges.discard((u, v))
        elif op == 2:
            n += 1
        elif op == 3:
            if not (0 <= u < n) or u in dead or u in protect:
                return p
            edges = {(a, b) for (a, b) in edges if a != u and b != u}
            dead.add(u)
        elif op == 4:
            if not (0 <= u < n) or u in dead:
                return p
            edges = {(a, b) for (a, b) in edges if a != u}
        else:
            return p
    return n, edges, dead


def edges_of(g):
    rp, col = g.csr()
    src = np.repeat(np.arange(g.n), np.diff(rp))
    return set(zip(src.tolist(), col.tolist()))


@pytest.mark.parametrize("trial", range(12))
def test_graph_apply_matches_python_sets(trial):
    rng = np.random.default_rng(500 + trial)
    p_zero = 0.0 if trial < 8 else 0.06  # the last trials also zero rows
    n = int(rng.integers(5, 40))
    src, dst = random_graph(rng, n, 0.15)
    g = O.Graph(n, src, dst)
    edges = set(zip(src.tolist(), dst.tolist()))
    dead = set()
    for _ in range(4):
        es = W.EdgeSet(*zip(*edges)) if edges else W.EdgeSet([], [])
        deadarr = np.zeros(g.n + 64, np.uint8)
        for d in dead:
            deadarr[d] = 1
        ops, _ = W.random_mixed_batch(rng, g.n, es, deadarr, 25, protect=(0,), p_zero_row=p_zero)
        want = apply_python(g.n, edges, dead, ops, protect=(0,))
        bad = g.apply(ops, protect=(0,))
        assert bad == -1 and not isinstance(want, int)
        n2, edges, dead = want
        assert g.n == n2 and edges_of(g) == edges
        rp, col = g.csr()
        assert np.all(np.diff(rp) >= 0)
        for u in range(g.n):  # rows sorted ascending, no duplicates
            row = col[rp[u]:rp[u + 1]]
            assert np.all(np.diff(row) > 0)
        cp, rows = g.csc()
        src2 = np.repeat(np.arange(g.n), np.diff(cp))
        assert set(zip(rows.tolist(), src2.tolist())) == edges
        assert set(np.nonzero(g.dead())[0].tolist()) == dead


def test_graph_invalid_batches_leave_graph_unchanged():
    g = O.Graph(4, [0, 1, 2], [1, 2, 3])
    before = edges_of(g)
    mk = lambda rows: np.array(rows, dtype=np.int64)
    cases = [
        ([(0, 9, 0)], 0),                 # id out of range
        ([(0, 0, 2), (0, 4, 0), (0, 5, 0)], 2),  # node 4 exists after the add, 5 does not
        ([(2, 0, 3), (1, 2, 0)], 1),      # use after delete
        ([(2, 0, 3), (2, 0, 3)], 1),      # double delete
        ([(0, 0, 3)], 0),                 # protected seed
        ([(0, 1, 7)], 0),                 # bad op code
        ([(2, 0, 3), (2, 0, 4)], 1),      # zero the row of a deleted node
        ([(0, 0, 4), (9, 0, 4)], 1),      # zero the row of an absent node
    ]
    for rows, bad_at in cases:
        arr = mk(rows)
        ops = np.empty(len(rows), W.UPDATE_DTYPE)
        ops["u"], ops["v"], ops["op"] = arr[:, 0], arr[:, 1], arr[:, 2]
        assert g.apply(ops, protect=(0,)) == bad_at
        assert apply_python(4, before, set(), ops, protect=(0,)) == bad_at
        assert edges_of(g) == before and g.n == 4


# ---------------------------------------------------------------------------
# Offset vector and OSP (Sec. 3.1, Algorithm 1, Theorems 2-4, Sec. 3.3)
# ---------------------------------------------------------------------------
def random_case(rng, n=None, n_ops=30, p=0.12, ops_kinds=True, p_zero_row=0.0):
    n = n or int(rng.integers(8, 70))
    src, dst = random_graph(rng, n, p)
    g = O.Graph(n, src, dst)
    seed = 0
    old = g.csr()
    es = W.EdgeSet(src, dst)
    dead = np.zeros(n + n_ops + 1, np.uint8)
    if ops_kinds:
        ops, _ = W.random_mixed_batch(rng, n, es, dead, n_ops, protect=(seed,),
                                      p_zero_row=p_zero_row)
    else:
        ops, _ = W.random_mixed_batch(rng, n, es, dead, n_ops, p_add=0, p_delnode=0,
                                      protect=(seed,))
    assert g.apply(ops, protect=(seed,)) == -1
    return g, old, g.csr(), seed, n


def dense_from_csr(rp, col):
    n = rp.size - 1
    return np.repeat(np.arange(n), np.diff(rp)), col


@pytest.mark.parametrize("trial", range(8))
def test_offset_matches_dense_definition(trial):
    rng = np.random.default_rng(900 + trial)
    g, old, new, seed, n_old = random_case(rng)
    r_old, _, _ = O.cpi(*old, seed, C_RESTART, 1e-14)
    q = O.offset(old, new, r_old, C_RESTART)
    n_new = new[0].size - 1
    A = np.zeros((n_new, n_new))
    A[:n_old, :n_old] = O.dense_matrix(n_old, *dense_from_csr(*old))
    B = O.dense_matrix(n_new, *dense_from_csr(*new))
    ro = np.zeros(n_new)
    ro[:n_old] = r_old
    want = (1 - C_RESTART) * (B.T - A.T) @ ro
    assert np.abs(q - want).max() < 1e-15
    # Sec. 3.3: ||q||_1 <= (1-c) ||D r_old||_1 with D_ii = sum_j |dA_ij|, and <= 2(1-c)||r_old||_1
    D = np.abs(B - A).sum(axis=1)
    assert np.abs(q).sum() <= (1 - C_RESTART) * np.abs(D * ro).sum() + 1e-15
    assert np.abs(q).sum() <= 2 * (1 - C_RESTART) * np.abs(ro).sum() + 1e-15


@pytest.mark.parametrize("trial", range(12))
def test_osp_exactness_theorem2(trial):
    # Theorem 2: r_old + r_offset equals the RWR vector of the updated graph
    # (the last trials also zero rows, the literal node deletion of Sec. 3.4.1).
    rng = np.random.default_rng(1300 + trial)
    g, old, new, seed, _ = random_case(rng, p_zero_row=0.0 if trial < 8 else 0.08)
    r_old = O.dense_rwr(old[0].size - 1, *dense_from_csr(*old), seed, C_RESTART)
    r_new, q, st, _ = O.osp(old, new, r_old, C_RESTART, 1e-16)
    want = O.dense_rwr(new[0].size - 1, *dense_from_csr(*new), seed, C_RESTART)
    assert np.abs(r_new - want).sum() < 1e-13
    # the literal "r_offset = 0" start of the listing misses q_offset itself
    if np.abs(q).sum() > 1e-6:
        assert np.abs((r_new - q) - want).sum() > 1e-3 * np.abs(q).sum()


def test_osp_equals_recompute_after_several_batches():
    rng = np.random.default_rng(77)
    n = 60
    src, dst = random_graph(rng, n, 0.08)
    g = O.Graph(n, src, dst)
    es = W.EdgeSet(src, dst)
    dead = np.zeros(n + 200, np.uint8)
    cur = g.csr()
    r, _, _ = O.cpi(*cur, 0, C_RESTART, 1e-15)
    for _ in range(5):
        ops, _ = W.random_mixed_batch(rng, g.n, es, dead, 20, protect=(0,))
        assert g.apply(ops, protect=(0,)) == -1
        new = g.csr()
        r, _, _, _ = O.osp(cur, new, r, C_RESTART, 1e-15)
        cur = new
    r_cpi, _, _ = O.cpi(*cur, 0, C_RESTART, 1e-15)
    assert np.abs(r - r_cpi).sum() < 1e-12


@pytest.mark.parametrize("eps", [1e-2, 1e-3, 1e-5])
def test_ospt_iteration_and_error_bounds(eps):
    # Theorem 3 (iterations) and Theorem 4 in its exact form for one batch from an
    # exact r_old: ||r_new - r*||_1 <= ||x(k)||_1 (1-c)/c <= eps (1-c)/c.
    rng = np.random.default_rng(int(-math.log10(eps)) * 17)
    for _ in range(5):
        g, old, new, seed, _ = random_case(rng, n_ops=40)
        r_old = O.dense_rwr(old[0].size - 1, *dense_from_csr(*old), seed, C_RESTART)
        r_new, q, st, hist = O.osp(old, new, r_old, C_RESTART, eps)
        want = O.dense_rwr(new[0].size - 1, *dense_from_csr(*new), seed, C_RESTART)
        ql1 = np.abs(q).sum()
        assert 1 <= st["iterations"] <= iter_bound(eps, ql1, C_RESTART)
        assert st["iterations"] < math.log(eps / 2) / math.log(1 - C_RESTART) or ql1 <= eps
        err = np.abs(r_new - want).sum()
        assert err <= st["last_l1"] * (1 - C_RESTART) / C_RESTART + 1e-14
        assert err <= eps * (1 - C_RESTART) / C_RESTART + 1e-14
        assert hist[0] == pytest.approx(ql1, rel=1e-15)


def test_ospt_runs_at_least_once_as_in_table2():
    # Table 2 first row: ||q_offset|| below eps still gives one iteration.
    gold = golden("paper_table2.txt")
    rng = np.random.default_rng(5)
    g, old, new, seed, _ = random_case(rng, n_ops=2, ops_kinds=False)
    r_old, _, _ = O.cpi(*old, seed, C_RESTART, 1e-14)
    _, q, st, _ = O.osp(old, new, r_old, C_RESTART, 1e6)
    assert st["iterations"] == int(gold["ospt_row1_iterations"])
    # the printed rows respect Theorem 3's bound
    for ql1, it in zip(gold["osp_qoff_l1_by_deleted"], gold["osp_iterations_by_deleted"]):
        assert it <= iter_bound(gold["osp_row1_eps"], ql1, gold["cpi_c"])
    assert int(gold["osp_row1_iterations"]) <= iter_bound(gold["osp_row1_eps"],
                                                           gold["osp_row1_qoff_l1"], 0.15)
    assert np.all(np.diff(gold["osp_qoff_l1_by_deleted"]) > 0)


def test_new_node_with_only_out_edges_leaves_scores_unchanged():
    # Sec. 3.4.1: r_old gets a zero entry for the new node, so its new row adds
    # nothing to q_offset; nothing else changes.
    rng = np.random.default_rng(11)
    src, dst = random_graph(rng, 20, 0.2)
    g = O.Graph(20, src, dst)
    old = g.csr()
    r_old, _, _ = O.cpi(*old, 0, C_RESTART, 1e-15)
    ops = np.zeros(4, W.UPDATE_DTYPE)
    ops[0] = (0, 0, W.OP_ADD_NODE)
    ops[1] = (20, 3, W.OP_INSERT_EDGE)
    ops[2] = (20, 5, W.OP_INSERT_EDGE)
    ops[3] = (20, 20, W.OP_INSERT_EDGE)
    assert g.apply(ops) == -1
    r_new, q, st, _ = O.osp(old, g.csr(), r_old, C_RESTART, 1e-15)
    assert np.all(q == 0)
    assert np.array_equal(r_new[:20], r_old) and r_new[20] == 0


# ---------------------------------------------------------------------------
# Dead-ends (Theorem 5) and the residual certificate
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("trial", range(5))
def test_dead_end_normalisation_theorem5(trial):
    # r_temp / ||r_temp||_1 equals RWR on the graph where every dead-end links to the seed.
    rng = np.random.default_rng(2100 + trial)
    n = int(rng.integers(5, 50))
    src, dst = random_graph(rng, n, 0.06)
    seed = int(rng.integers(n))
    rp, col = csr_from_edges(n, src, dst)
    r_temp, _, _ = O.cpi(rp, col, seed, C_RESTART, 1e-16)
    deg = np.diff(rp)
    de = np.nonzero(deg == 0)[0]
    src2 = np.concatenate([src, de]).astype(np.int32)
    dst2 = np.concatenate([dst, np.full(de.size, seed)]).astype(np.int32)
    want = O.dense_rwr(n, src2, dst2, seed, C_RESTART)
    assert np.abs(O.normalize(r_temp) - want).sum() < 1e-12


def test_residual_certificate_bounds_error():
    rng = np.random.default_rng(31)
    for _ in range(5):
        n = int(rng.integers(10, 60))
        src, dst = random_graph(rng, n, 0.1)
        rp, col = csr_from_edges(n, src, dst)
        want = O.dense_rwr(n, src, dst, 1, C_RESTART)
        r = want + rng.normal(0, 1e-4, n)
        rho = O.residual_l1(rp, col, 1, C_RESTART, r)
        err = np.abs(r - want).sum()
        assert err <= rho / C_RESTART + 1e-15
        assert O.residual_l1(rp, col, 1, C_RESTART, want) < 1e-14


def test_topk_order_and_ties():
    r = np.array([0.1, 0.3, 0.3, 0.05, 0.3, 0.2])
    ids, sc = O.topk(r, 4)
    assert ids.tolist() == [1, 2, 4, 5]
    assert sc.tolist() == [0.3, 0.3, 0.3, 0.2]


def test_generators_are_seeded_and_valid():
    s1, d1 = W.er_graph(1000, 5000, 1)
    s2, d2 = W.er_graph(1000, 5000, 1)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    keys = W.edge_keys(s1, d1)
    assert np.unique(keys).size == 5000 and np.all(s1 != d1)
    g, s, d = W.rmat_graph(12, 40000, seed=3)
    assert np.unique(W.edge_keys(s, d)).size == 40000 and np.all(s != d)
    deg = W.out_degrees(g.n, s)
    assert deg.max() > 20 * deg.mean()  # power-law hubs
    stream = W.edge_update_stream(s1, d1, 1000, 3, 50, 50, seed=9)
    es = W.EdgeSet(s1, d1)
    for ops in stream:
        ins = ops[ops["op"] == 0]
        dels = ops[ops["op"] == 1]
        assert not es.contains(W.edge_keys(ins["u"], ins["v"])).any()
        assert es.contains(W.edge_keys(dels["u"], dels["v"])).all()
        es.apply(W.edge_keys(ins["u"], ins["v"]), W.edge_keys(dels["u"], dels["v"]))


def test_uniform_restart_vector_pagerank_mode():
    """PageRank mode (uniform q): on a directed cycle every node keeps 1/n (A~ 1 =
    1 so r = c (1 - (1-c))^-1 q); on random graphs with dead-ends the CPI series
    from x(0) = c q matches the dense solve of Eq. 1 with that q."""
    n, c = 9, 0.15
    src = np.arange(n, dtype=np.int32)
    dst = ((src + 1) % n).astype(np.int32)
    g = O.Graph(n, src, dst)
    r, _, _ = O.propagate(*g.csr(), np.full(n, c / n), c, 1e-15)
    assert np.allclose(r, 1.0 / n, rtol=0, atol=1e-13)
    rng = np.random.default_rng(12)
    for _ in range(3):
        n = 60
        src = rng.integers(0, n, 200).astype(np.int32)
        dst = rng.integers(0, n, 200).astype(np.int32)
        src[src < 5] = 5  # nodes 0..4 keep no out-edges (dead-ends)
        g = O.Graph(n, src, dst)
        q = np.full(n, 1.0 / n)
        r, _, _ = O.propagate(*g.csr(), c * q, c, 1e-15)
        want = O.dense_rwr_q(n, *O_edges(g), q, c)
        assert np.abs(r - want).sum() <= 1e-12
        # the seed form is the special case q = e_s
        e = np.zeros(n)
        e[7] = 1.0
        assert np.abs(O.dense_rwr_q(n, *O_edges(g), e, c) - O.dense_rwr(n, *O_edges(g), 7, c)).sum() <= 1e-14


def O_edges(g):
    rp, col = g.csr()
    src = np.repeat(np.arange(rp.size - 1), np.diff(rp)).astype(np.int32)
    return src, np.asarray(col, np.int32)


def test_zero_row_is_the_literal_node_deletion():
    # Sec. 3.4.1 read literally: deleting node u sets u's row of B~ to zero. The
    # node keeps its in-edges, so it still collects score but passes none on
    # (it is a dead-end); with the seed's row zeroed, r = c e_s.
    n = 5
    src = [0, 0, 1, 2, 3, 3]
    dst = [1, 2, 2, 3, 0, 4]
    g = O.Graph(n, src, dst)
    ops = np.empty(1, W.UPDATE_DTYPE)
    ops[0] = (3, 0, W.OP_ZERO_ROW)
    old = g.csr()
    assert g.apply(ops, protect=(0,)) == -1
    assert edges_of(g) == {(0, 1), (0, 2), (1, 2), (2, 3)}
    new = g.csr()
    r_old = O.dense_rwr(n, *dense_from_csr(*old), 0, C_RESTART)
    r_new, _, _, _ = O.osp(old, new, r_old, C_RESTART, 1e-16)
    # closed form on the zeroed graph: 0 -> {1, 2}, 1 -> 2, 2 -> 3, 3 a dead-end
    a = 1 - C_RESTART
    r0 = C_RESTART
    r1 = a * r0 / 2
    r2 = a * (r0 / 2 + r1)
    r3 = a * r2
    want = np.array([r0, r1, r2, r3, 0.0])
    assert np.abs(r_new - want).sum() < 1e-14
    # the seed's own row
    g2 = O.Graph(n, src, dst)
    ops[0] = (0, 0, W.OP_ZERO_ROW)
    assert g2.apply(ops, protect=(0,)) == -1
    r_seed, _, _, _ = O.osp(old, g2.csr(), r_old, C_RESTART, 1e-16)
    assert np.abs(r_seed - C_RESTART * np.eye(n)[0]).sum() < 1e-14
    # edges re-inserted after the zeroing in the same batch are kept
    g3 = O.Graph(n, src, dst)
    ops3 = np.empty(3, W.UPDATE_DTYPE)
    ops3[0] = (3, 4, W.OP_INSERT_EDGE)
    ops3[1] = (3, 0, W.OP_ZERO_ROW)
    ops3[2] = (3, 0, W.OP_INSERT_EDGE)
    assert g3.apply(ops3, protect=(0,)) == -1
    assert edges_of(g3) == {(0, 1), (0, 2), (1, 2), (2, 3), (3, 0)}


def test_seed_block_input_generators():
    # Chung-Lu: distinct unordered pairs, exact count, heavy-tailed degrees
    # that follow the weights (the top-weight nodes carry the largest degrees)
    g, lo, hi = W.chung_lu_graph(4096, 4096 * 8, seed=11)
    assert lo.size == 4096 * 8 and np.all(lo < hi)
    assert np.unique(W.edge_keys(lo, hi)).size == lo.size
    deg = np.bincount(np.concatenate([lo, hi]), minlength=4096)
    assert deg.mean() == 16.0
    top = g.perm[:8]  # the largest weights, capped at sqrt(sum w) = 256
    assert deg[top].min() > 8 * deg.mean() and deg.max() < 2 * 256
    # undirected stream: both directions of every pair, insertions absent,
    # deletions present, sizes as asked
    sizes = W.log_uniform_sizes(6, 10, 1000, seed=4)
    assert np.all((sizes >= 10) & (sizes < 1000))
    stream = W.undirected_update_stream(lo, hi, 4096, sizes, 5, g.sample)
    es = W.EdgeSet(np.concatenate([lo, hi]), np.concatenate([hi, lo]))
    for k, ops in zip(sizes, stream):
        assert ops.size == 2 * k
        fwd = set(zip(ops["u"].tolist(), ops["v"].tolist(), ops["op"].tolist()))
        assert all((v, u, op) in fwd for (u, v, op) in fwd)
        ins = ops[ops["op"] == W.OP_INSERT_EDGE]
        dels = ops[ops["op"] == W.OP_DELETE_EDGE]
        assert not es.contains(W.edge_keys(ins["u"], ins["v"])).any()
        assert es.contains(W.edge_keys(dels["u"], dels["v"])).all()
        es.apply(W.edge_keys(ins["u"], ins["v"]), W.edge_keys(dels["u"], dels["v"]))
    # node operations: valid in sequence, seeds never deleted
    _, s, d = W.rmat_graph(10, 6000, seed=2)
    batches = W.node_op_stream(s, d, 1024, 3, 20, 8, 10, 40, seed=6, protect=(0, 5))
    gr = O.Graph(1024, s, d)
    for ops in batches:
        assert gr.apply(ops, protect=(0, 5)) == -1
        assert (ops["op"] == W.OP_ADD_NODE).sum() == 20
        assert (ops["op"] == W.OP_DELETE_NODE).sum() == 10


@pytest.mark.parametrize("trial", range(3))
def test_batch_equals_its_ops_applied_one_at_a_time(trial):
    # Several ops on one row in one batch (reading c12): Delta A is the rows
    # after the whole batch minus the rows before it, so in exact mode one OSP
    # call over the batch equals one OSP call per op, and both equal the dense
    # solve on the final graph (Theorem 2).
    rng = np.random.default_rng(2100 + trial)
    n = 40
    src, dst = random_graph(rng, n, 0.1)
    es = W.EdgeSet(src, dst)
    dead = np.zeros(n + 64, np.uint8)
    ops, _ = W.random_mixed_batch(rng, n, es, dead, 30, protect=(0,), p_zero_row=0.05)
    # a row touched several times: insert, delete, re-insert the same edge
    extra = np.empty(3, W.UPDATE_DTYPE)
    extra[0] = (1, 2, W.OP_INSERT_EDGE)
    extra[1] = (1, 2, W.OP_DELETE_EDGE)
    extra[2] = (1, 3, W.OP_INSERT_EDGE)
    ops = np.concatenate([extra, ops])
    g_all, g_one = O.Graph(n, src, dst), O.Graph(n, src, dst)
    start = g_all.csr()
    r0 = O.dense_rwr(n, src, dst, 0, C_RESTART)
    assert g_all.apply(ops, protect=(0,)) == -1
    r_all, _, _, _ = O.osp(start, g_all.csr(), r0, C_RESTART, 1e-16)
    r_one, cur = r0, start
    for k in range(ops.size):
        assert g_one.apply(ops[k:k + 1], protect=(0,)) == -1
        new = g_one.csr()
        r_one, _, _, _ = O.osp(cur, new, r_one, C_RESTART, 1e-16)
        cur = new
    assert edges_of(g_all) == edges_of(g_one)
    n_new = cur[0].size - 1
    want = O.dense_rwr(n_new, *dense_from_csr(*cur), 0, C_RESTART)
    assert np.abs(r_all - want).sum() < 1e-12
    assert np.abs(r_one - want).sum() < 1e-11


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_error_accumulates_at_most_linearly_over_batches(eps):
    # Reading c5: each batch leaves an untaken tail whose residual is the last
    # step's x(k+1), of norm <= (1-c) eps, and the residuals add up; so after B
    # batches from a CPI start at eps_init, ||r - r*||_1 <= ||rho||_1 / c with
    # ||rho||_1 <= (1-c) eps_init + B (1-c) eps. Checked against the dense
    # solve and the residual computed directly.
    rng = np.random.default_rng(int(-math.log10(eps)) * 31)
    n = 60
    src, dst = random_graph(rng, n, 0.08)
    g = O.Graph(n, src, dst)
    es = W.EdgeSet(src, dst)
    dead = np.zeros(n + 400, np.uint8)
    cur = g.csr()
    eps_init = 1e-4
    r, _, _ = O.cpi(*cur, 0, C_RESTART, eps_init)
    B = 12
    for b in range(B):
        ops, _ = W.random_mixed_batch(rng, g.n, es, dead, 15, protect=(0,))
        assert g.apply(ops, protect=(0,)) == -1
        new = g.csr()
        r, _, _, _ = O.osp(cur, new, r, C_RESTART, eps)
        cur = new
        rho = O.residual_l1(*cur, 0, C_RESTART, r)
        assert rho <= (1 - C_RESTART) * (eps_init + (b + 1) * eps) + 1e-13
        want = O.dense_rwr(cur[0].size - 1, *dense_from_csr(*cur), 0, C_RESTART)
        assert np.abs(r - want).sum() <= rho / C_RESTART + 1e-12
