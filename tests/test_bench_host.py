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
    # two steps; seeds that propagate ran 2 + 1 + 2 steps (col_steps = 5)
    st = {"iterations": 2, "pull_dst_nodes": 30, "pull_src_nodes": 35}
    m = 1000
    fixed = 4 * m + 4 * 31
    per_col = 2 * 35 + (2 + 16) * 30 + 8
    assert bench.multi_alg_bytes(st, m, 5, 2) == 2 * fixed + 5 * per_col
    # every column running every step: the dense count of S columns per step
    S = 64
    assert bench.multi_alg_bytes(st, m, 2 * S, 2) == 2 * (fixed + S * per_col)


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


def test_clock_samples_parsing():
    hdr = ["index", " clocks.current.sm [MHz]", " clocks.max.sm [MHz]", " power.draw [W]",
           " clocks_event_reasons.active", " clocks_event_reasons.hw_slowdown",
           " clocks_event_reasons.hw_thermal_slowdown", " clocks_event_reasons.sw_thermal_slowdown",
           " clocks_event_reasons.sw_power_cap"]
    row = lambda mhz, cap: ["0", f" {mhz} MHz", " 2070 MHz", " 900.00 W", " 0x0", " Not Active",  # noqa: E731
                            " Not Active", " Not Active", " Active" if cap else " Not Active"]
    out = bench.parse_clock_samples([hdr, row(2070, False), row(1980, True), row(2070, False),
                                     ["0", "garbled"]])
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    assert bench.parse_clock_samples([hdr]) is None


def test_traffic_record_is_ignored_when_the_kernel_changed(monkeypatch):
    # the committed DRAM bytes belong to the kernel sources they were taken on
    cur = bench.kernel_source_hash()
    rec = bench.traffic_from_profile()
    if rec is not None:
        assert rec > 1e8
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16 if cur != "0" * 16 else "1")
    assert bench.traffic_from_profile() is None


def test_l1_lookup_roofline():
    """One gather per visited edge against one sector lookup per SM cycle."""
    stats = [{"visited_edges": 16_000_000}, {"visited_edges": 48_000_000}]
    r = bench.l1_lookup_roofline(stats, prop_ms=0.4, clk={"sm_mhz": 2000.0}, sms=150)
    assert r["achieved"] == pytest.approx(64e6 / 0.4e-3 / 1e9)   # G lookups/s
    assert r["peak"] == pytest.approx(150 * 2.0)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.l1_lookup_roofline(stats, 0.4, None, 150)["peak"] == pytest.approx(150 * 2.07)
