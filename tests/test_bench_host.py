"""Host-side logic of the benchmark: algorithmic byte counts, the committed
traffic record, and the replica timing reduction over two gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def test_alg_bytes_pull_and_push():
    st = {"iterations": 3, "push_iterations": 1, "visited_edges": 100 + 2 * 1000,
          "push_frontier": 10, "push_reached": 40, "pull_dst_nodes": 30, "pull_src_nodes": 35}
    n, m = 50, 1000
    pull = 2 * (4 * m + 4 * 31 + 4 * 35 + 20 * 30 + 8)
    push = 4 * 100 + 12 * 10 + 20 * 40
    assert bench.alg_bytes(st, n, m, 4, 4) == pull + push


def test_alg_bytes_seed_block():
    st = {"iterations": 2, "pull_dst_nodes": 30, "pull_src_nodes": 35}
    m, S = 1000, 64
    step = 4 * m + 4 * 31 + S * 2 * 35 + S * (2 + 16) * 30 + 8 * S
    assert bench.multi_alg_bytes(st, m, S, 2) == 2 * step


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})

    class A:
        gpus = world

    r, w = bench.dist_setup(A)
    bench.dist_barrier(w)
    q.put((r, w, bench.dist_max(1.0 + r, w)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replica_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    assert got == [(0, 2, 2.0), (1, 2, 2.0)]


def test_rank_accuracy_matches_scipy_spearman():
    scipy_stats = pytest.importorskip("scipy.stats")
    import numpy as np
    rng = np.random.default_rng(0)
    a = rng.random(2000)
    b = a + rng.normal(0, 0.01, a.size)
    b[:80] = b[0]  # ties
    got = bench.rank_accuracy(a, b)
    assert got["spearman"] == pytest.approx(scipy_stats.spearmanr(a, b).correlation, abs=1e-12)
    top_a = set(np.argsort(-a, kind="stable")[:100].tolist())
    assert bench.rank_accuracy(a, a) == {"spearman": 1.0, "top100_overlap": 1.0}
    assert 0.0 <= got["top100_overlap"] <= 1.0 and len(top_a) == 100
