#!/usr/bin/env python
"""Benchmark of the OSP / OSP-T update path on one GB300 (or N independent replicas).

Workload (the paper's Table 3 graphs are stood in for by a seeded R-MAT graph):
directed R-MAT scale 20 (1,048,576 nodes, 16,777,216 unique edges,
a,b,c,d = .57,.19,.19,.05, ids permuted), c = 0.15, one seed (the node of
highest out-degree), a stream of batches of 1,000 updates (600 insertions of
absent edges with R-MAT endpoints, 400 deletions of existing edges). A step is
one batch through the whole path: ingest + validation, graph-store merge,
offset vector, propagation to ||x||_1 <= eps, merge into the scores.

Reported: update batches/s (FP32 products, FP64 accumulation, eps = 1e-6) with
the device-resident batch, the L1 distance of those scores to the plain FP64
path replaying the same iteration counts, the propagation kernel's algorithmic
GB/s against the measured HBM copy bandwidth, the FP64 path and an eps sweep,
the end-to-end rate through the host API, and the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1712_00595_gb300 import workloads as W  # noqa: E402

METRIC = "edge-update batches/sec and propagation GB/s (% of HBM peak) at <=1e-5 L1 vs FP64"
C_RESTART = 0.15
N_INS, N_DEL = 600, 400
HUB_SEED_OFFSET = 2
STREAM_SEED_OFFSET = 202


# Several seeds at once (the n x Sp seed block). Sizes at full scale.
MULTI_WORKLOADS = {
    # undirected Chung-Lu (exponent 2.1, mean degree 16): 4,194,304 nodes,
    # 33,554,432 undirected edges stored in both directions; 64 uniform seeds;
    # batches of log-uniform 10 .. 10,000 undirected edges (each = 2 directed ops,
    # half insertions, half deletions); FP32 gather vectors, FP64 sums
    "chunglu22_s64": {"graph": "chunglu", "log2n": 22, "m": 33554432, "S": 64,
                      "precision": "fp32", "eps": 1e-6, "batches": 50},
    # directed R-MAT scale 24: 16,777,216 nodes, 268,435,456 edges; 256 uniform
    # seeds; batches of 10,000 ops: 500 edge ops, 1,000 new nodes with 8
    # out-edges each, 500 node deletions; bf16 gather vectors, FP64 sums
    "rmat24_s256": {"graph": "rmat", "log2n": 24, "m": 268435456, "S": 256,
                    "precision": "bf16", "eps": 1e-6, "batches": 20},
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--scale", type=int, default=20)
    p.add_argument("--eps", type=float, default=1e-6)
    p.add_argument("--eps-init", type=float, default=1e-10)
    p.add_argument("--no-extras", action="store_true", help="headline only (profiling runs)")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="CPU time bound of the cpu_baseline sample (whole batches)")
    p.add_argument("--node-order", type=int, default=0, choices=[0, 1],
                   help="internal node order: 0 = caller ids, 1 = descending out-degree")
    p.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="keep the default pull-step schedule (osp_init_scores tunes it otherwise)")
    p.add_argument("--launch", default="graphs", choices=["graphs", "eager"],
                   help="batch kernels replayed from CUDA graphs, or launched one by one")
    p.add_argument("--workload", default="rmat20",
                   choices=["rmat20", "serve22", "location", "growshrink"] + sorted(MULTI_WORKLOADS),
                   help="rmat20: the one-seed headline; the others track many seeds at once")
    p.add_argument("--serve-policy", default="latest", choices=["ordered", "latest"],
                   help="serve22: queries read in arrival order, or the newest scores")
    p.add_argument("--log2n", type=int, default=0,
                   help="several-seed workloads: nodes 2^log2n (edges scaled alike; 0 = full size)")
    p.add_argument("--seed-gather", default="auto", choices=["auto", "regs", "bulk"],
                   help="seed-block workloads: source rows gathered into registers, or "
                        "staged in shared memory by bulk asynchronous copies (auto: the "
                        "engine's choice by row size)")
    p.add_argument("--fp64-seeds", type=int, default=8,
                   help="several-seed workloads: seeds compared with the FP64 replay (0 = skip)")
    return p.parse_args()


STREAM_MIN_BATCHES = 64  # both arms draw the same stream (its batches depend on its length)


def make_workload(scale, batches):
    batches = max(batches, STREAM_MIN_BATCHES)
    gen, src, dst = W.rmat_graph(scale, 16 << scale, seed=W.BASE_SEED + HUB_SEED_OFFSET)
    n = gen.n
    seed = W.max_out_degree_seed(n, src)
    stream = W.edge_update_stream(src, dst, n, batches, N_INS, N_DEL,
                                  seed=W.BASE_SEED + STREAM_SEED_OFFSET, sampler=gen.sample)
    return n, src, dst, seed, stream


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def alg_bytes(st, n, m, bx, bs, S=1):
    """Algorithmic bytes of one propagation launch (each operand once), for S
    seeds, gather vectors of bx bytes and FP64 sums:
    pull step  4 m (in-list ids) + 4 (|V| + 1) (list starts) + S bx |src| (each
               source's y once) + S (bx + 16) |V| (write y, read and write r)
               + 8 S (|x| partials), V = nodes with an in-edge, src = nodes with
               an out-edge
    push step  4 E_F + (8 + bx) |F| + (bx + 16) |F'|  (one seed).
    bs (scale bytes) is not an operand of this count; nodes without in-edges
    need no r update and are not counted."""
    del n, bs
    pull_steps = st["iterations"] - st["push_iterations"]
    V, src = st["pull_dst_nodes"], st["pull_src_nodes"]
    pull = pull_steps * (4 * m + 4 * (V + 1) + S * bx * src + S * (bx + 16) * V + 8 * S)
    if st["push_iterations"] == 0:
        return pull
    ef = st["visited_edges"] - pull_steps * m
    push = 4 * ef + (8 + bx) * st["push_frontier"] + (bx + 16) * st["push_reached"]
    return pull + push


TRAFFIC_SOURCES = ("propagate.cu", "common.cuh")


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the propagation kernel's sources."""
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1712_00595_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profile():
    """Per-launch DRAM bytes of the propagation kernel from the committed ncu
    summary, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "propagate_rmat20_traffic.txt")
    try:
        vals = {}
        with open(path) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("source_sha256_16") != kernel_source_hash():
            return None
        return float(vals["dram_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = list(csv.reader(open(self.path)))
        keep = os.environ.get("OSP_CLOCKS_LOG")  # optional copy of the raw samples
        if keep:
            with open(keep, "w") as f:
                f.write(open(self.path).read())
        os.unlink(self.path)
        return parse_clock_samples(rows)


def parse_clock_samples(rows):
    """nvidia-smi CSV rows (header first) -> median SM clock, max clock and the
    throttle reasons seen active during the samples (None without samples)."""
    if len(rows) < 2:
        return None
    hdr = [h.strip() for h in rows[0]]
    sm, smax, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows[1:]:
        if len(r) != len(hdr):
            continue
        d = dict(zip(hdr, [x.strip() for x in r]))
        try:
            sm.append(float(d["clocks.current.sm [MHz]"].split()[0]))
            smax = max(smax, float(d["clocks.max.sm [MHz]"].split()[0]))
        except Exception:
            continue
        for nm in names:
            key = [k for k in d if k.startswith("clocks_event_reasons." + nm)]
            if key and d[key[0]].lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


def dist_setup(args):
    rank, world = 0, 1
    if args.gpus > 1 or "WORLD_SIZE" in os.environ:
        import torch.distributed as dist
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if world > 1:
            dist.init_process_group("gloo")
    return rank, world


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores: each step applies one batch and
    runs Algorithm 1 (graph update, CSR export, offset, propagation)."""
    if rank != 0:
        return
    from oracle import oracle as O
    n, src, dst, seed, stream = make_workload(args.scale, args.warmup + args.steps)
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r, _, _ = O.cpi(*cur, seed, C_RESTART, args.eps_init)

    def step(ops):
        nonlocal cur, r
        assert g.apply(ops, protect=(seed,)) == -1
        new = g.csr()
        r, _, st, _ = O.osp(cur, new, r, C_RESTART, args.eps)
        cur = new
        return st

    for b in range(args.warmup):
        step(stream[b])
    t0 = time.perf_counter()
    for b in range(args.warmup, args.warmup + args.steps):
        step(stream[b])
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "batches/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args, n, len(src), seed, "fp64 (CPU oracle)"),
                       l2="n/a (host)", inputs="update batches in host memory"),
        "cpu_baseline": {"value": v, "unit": "batches/s", "cores": 1, "kind": "oracle",
                         "sample": "%d batches of the workload, single-threaded C oracle" % args.steps},
        "e2e": {"value": v, "unit": "batches/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def rank_accuracy(r, ref, k=100):
    """Spearman rank correlation of two score vectors (average ranks for ties)
    and the overlap of their top-k sets (ids ranked by score, then id)."""
    def ranks(x):
        order = np.lexsort((np.arange(x.size), -x))
        rk = np.empty(x.size, np.float64)
        rk[order] = np.arange(x.size, dtype=np.float64)
        # average the ranks of equal scores
        xs = x[order]
        bounds = np.flatnonzero(np.diff(xs)) + 1
        starts = np.concatenate([[0], bounds])
        ends = np.concatenate([bounds, [x.size]])
        avg = (starts + ends - 1) / 2.0
        rk[order] = np.repeat(avg, ends - starts)
        return rk
    a, b = ranks(np.asarray(r)), ranks(np.asarray(ref))
    a -= a.mean()
    b -= b.mean()
    rho = float((a * b).sum() / np.sqrt((a * a).sum() * (b * b).sum()))
    ta = set(np.lexsort((np.arange(r.size), -np.asarray(r)))[:k].tolist())
    tb = set(np.lexsort((np.arange(ref.size), -np.asarray(ref)))[:k].tolist())
    return {"spearman": rho, "top%d_overlap" % k: len(ta & tb) / k}


def workload_config(args, n, m, seed, precision):
    return {"workload": "rmat%d_osp_t" % args.scale, "graph": "R-MAT scale %d (a,b,c,d=.57,.19,.19,.05), "
            "ids permuted" % args.scale, "nodes": n, "edges": m, "seed_node": int(seed),
            "seed_rule": "highest out-degree", "c": C_RESTART, "eps": args.eps,
            "batch": {"updates": N_INS + N_DEL, "insertions": N_INS, "deletions": N_DEL},
            "precision": precision, "l2": "flushed between steps (256 MiB write)",
            "inputs": "update batches resident in HBM before the timed region"}


def cpu_baseline(args, n, src, dst, seed, stream):
    """The oracle as it stands on a bounded sample: whole batches, after its own CPI,
    until --cpu-seconds have passed."""
    from oracle import oracle as O
    g = O.Graph(n, src, dst)
    cur = g.csr()
    r, _, _ = O.cpi(*cur, seed, C_RESTART, args.eps_init)
    k = 0
    t0 = time.perf_counter()
    while k < len(stream) and (k == 0 or time.perf_counter() - t0 < args.cpu_seconds):
        assert g.apply(stream[k], protect=(seed,)) == -1
        new = g.csr()
        r, _, _, _ = O.osp(cur, new, r, C_RESTART, args.eps)
        cur = new
        k += 1
    dt = time.perf_counter() - t0
    # the paper's baseline: CPI from scratch on the updated graph, same eps
    t1 = time.perf_counter()
    _, cst, _ = O.cpi(*cur, seed, C_RESTART, args.eps)
    dt_cpi = time.perf_counter() - t1
    return {"value": k / dt, "unit": "batches/s", "cores": 1, "kind": "oracle",
            "sample": "first %d batches of the same stream (graph update + Algorithm 1, FP64, "
                      "one thread; %.1f s)" % (k, dt),
            "cpi_from_scratch": {"ms": 1e3 * dt_cpi, "iterations": int(cst["iterations"])}}


def run_ours(args, rank, world):
    import torch

    from paper_1712_00595_gb300 import native as N

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K, Wm = args.steps, args.warmup
    total = Wm + K
    n, src, dst, seed, stream = make_workload(args.scale, total)
    U = N_INS + N_DEL
    ops_all = np.concatenate(stream).view(np.int32)
    ops_dev = torch.from_numpy(ops_all.copy()).to(dev)
    base_ptr = ops_dev.data_ptr()
    step_bytes = U * 12
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tstream = torch.cuda.Stream(device=dev)

    def new_engine(prec, graphs=args.launch == "graphs"):
        e = N.Engine(precision=prec, device=local, stream=tstream.cuda_stream, use_graphs=graphs,
                     autotune=args.autotune, node_order=args.node_order)
        e.load_graph(n, src, dst)
        e.set_seeds([seed], C_RESTART)
        e.init_scores(args.eps_init)
        return e

    def run(eng, eps, warm_n, force=None):
        """Warm up on batches [0, warm_n), then time batches [Wm, Wm + K): CUDA events
        around each step on the engine stream, L2 flushed between steps."""
        for b in range(warm_n):
            if force is not None:
                eng.set_fixed_iterations(force[b])
            eng.apply_updates_device(base_ptr + b * step_bytes, U, eps)
        torch.cuda.synchronize()
        dist_barrier(world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        stats = []
        for k in range(K):
            b = Wm + k
            with torch.cuda.stream(tstream):
                flush.fill_(k & 0xFF)
            if force is not None:
                eng.set_fixed_iterations(force[b])
            ev[k][0].record(tstream)
            stats.append(eng.apply_updates_device(base_ptr + b * step_bytes, U, eps))
            ev[k][1].record(tstream)
        torch.cuda.synchronize()
        dist_barrier(world)
        ms = [a.elapsed_time(b) for a, b in ev]
        eng.set_fixed_iterations(0)
        return ms, stats

    # ---- headline: FP32 products / FP64 accumulation at eps ----
    eng = new_engine(N.OSP_PREC_FP32_ACC64)
    warm_iters = []
    clocks = Clocks(local)
    # warm-up steps also record iteration counts for the lock-step FP64 replay
    for b in range(Wm):
        warm_iters.append(eng.apply_updates_device(base_ptr + b * step_bytes, U, args.eps)["iterations"])
    torch.cuda.synchronize()
    dist_barrier(world)
    clocks.start()
    ms, stats = run(eng, args.eps, 0)
    clk = clocks.stop()
    iters = warm_iters + [s["iterations"] for s in stats]
    st_us = eng.get_step_times()
    step_profile = {"x0": float(st_us[0]), "steps": [round(float(x), 1) for x in st_us[1:]]}
    r_mixed = eng.query()
    schedule = eng.get_schedule()
    # the paper's baseline on the GPU: CPI from scratch on the final graph at the same eps
    cpi_gpu = None
    if not args.no_extras:
        st_cpi = eng.init_scores(args.eps)
        cpi_gpu = {"ms": st_cpi["ms_update"] + st_cpi["ms_propagate"],
                   "iterations": int(st_cpi["iterations"])}
    t_local = sum(ms) / 1e3
    t_max = dist_max(t_local, world)
    value = world * K / t_max
    prop_ms = sum(s["ms_propagate"] for s in stats)
    upd_ms = sum(s["ms_update"] for s in stats)
    ab = sum(alg_bytes(s, s["n_nodes"], s["m_edges"], 4, 4) for s in stats)
    peak, peak_kind = peaks()
    achieved = ab / (prop_ms / 1e3) / 1e9
    eng.close()

    out = {
        "metric": METRIC, "value": value, "unit": "batches/s", "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": 1e3 * t_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "accumulate": "f64", "data": "synthetic",
        "config": dict(workload_config(args, n, len(src), seed, "fp32 products, fp64 accumulation"),
                       launch=args.launch, schedule=list(schedule)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_from_profile(),
                     "kernel": "k_propagate<float>", "peak_kind": peak_kind + " (hbm_gbs copy)",
                     "alg_bytes_per_launch": ab / K, "ms_per_launch": prop_ms / K},
        "phases_ms_per_step": {"update_merge_offset": upd_ms / K, "propagation": prop_ms / K},
        "batch_ms": {"median": float(np.median(ms)), "p99": float(np.percentile(ms, 99)),
                     "max": float(max(ms))},
        "iterations_per_step": float(np.mean([s["iterations"] for s in stats])),
        "push_iterations_per_step": float(np.mean([s["push_iterations"] for s in stats])),
        "qoff_l1_mean": float(np.mean([s["qoff_l1"] for s in stats])),
        "visited_edges_per_step": float(np.mean([s["visited_edges"] for s in stats])),
        "visited_edges_per_s": float(sum(s["visited_edges"] for s in stats)) / t_local,
        "cpi_from_scratch": cpi_gpu,
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "clocks": clk,
        "last_step_profile_us": step_profile,
    }

    if not args.no_extras:
        # ---- plain FP64 path, replaying the same iteration counts (lock-step) ----
        e64 = new_engine(N.OSP_PREC_FP64)
        ms64, st64 = run(e64, args.eps, Wm, force=iters)
        r64 = e64.query()
        e64.close()
        out["fp64_path"] = {"value": K / (sum(ms64) / 1e3), "unit": "batches/s",
                            "ms_propagation_per_step": sum(s["ms_propagate"] for s in st64) / K}
        out["l1_vs_fp64"] = float(np.abs(r_mixed - r64).sum())
        out["speedup_vs_fp64"] = value / world / out["fp64_path"]["value"]
        # ---- near-exact scores after the same batches (FP64, eps 1e-12) ----
        ex = new_engine(N.OSP_PREC_FP64)
        run(ex, 1e-12, Wm)
        r_exact = ex.query()
        ex.close()
        # ---- OSP-T eps sweep (FP32 products / FP64 accumulation) ----
        sweep = []
        for eps in (1e-4, 1e-6, 1e-8):
            e = new_engine(N.OSP_PREC_FP32_ACC64)
            ms_e, st_e = run(e, eps, Wm)
            r_e = e.query()
            e.close()
            sweep.append({"eps": eps, "batches_per_s": K / (sum(ms_e) / 1e3),
                          "iterations": float(np.mean([s["iterations"] for s in st_e])),
                          "ms_propagation": sum(s["ms_propagate"] for s in st_e) / K,
                          "l1_vs_exact": float(np.abs(r_e - r_exact).sum()),
                          "rank_vs_exact": rank_accuracy(r_e, r_exact)})
        out["eps_sweep"] = sweep
        out["rank_accuracy_fp32_vs_fp64"] = rank_accuracy(r_mixed, r64)
        # ---- the other launch mode (graph replays vs one launch per kernel) ----
        e = new_engine(N.OSP_PREC_FP32_ACC64, graphs=args.launch != "graphs")
        ms_o, _ = run(e, args.eps, Wm)
        e.close()
        out["other_launch_mode"] = {"launch": "eager" if args.launch == "graphs" else "graphs",
                                    "value": K / (sum(ms_o) / 1e3), "unit": "batches/s"}
        # ---- end to end through the host API: host batch in, top of the scores out ----
        e = new_engine(N.OSP_PREC_FP32_ACC64)
        host_ops = [np.ascontiguousarray(s) for s in stream]
        for b in range(Wm):
            e.apply_updates(host_ops[b], args.eps)
        # the scores land in a page-locked host buffer (node ids only grow by the
        # stream's additions, at most one per op)
        res = torch.empty(n + sum(int(s.size) for s in host_ops), dtype=torch.float64,
                          pin_memory=True).numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        per = []
        for k in range(K):
            ta = time.perf_counter()
            e.apply_updates(host_ops[Wm + k], args.eps)
            e.query(out=res)
            per.append(time.perf_counter() - ta)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e.close()
        out["e2e"] = {"value": K / dt, "unit": "batches/s", "h2d_bytes_per_step": step_bytes,
                      "d2h_bytes_per_step": 8 * n, "result": "full score vector (osp_query)",
                      "batch_ms": {"median": 1e3 * float(np.median(per)),
                                   "p99": 1e3 * float(np.percentile(per, 99))}}
    else:
        out["e2e"] = None

    if rank == 0 and world == 1 and not args.no_extras:
        out["cpu_baseline"] = cpu_baseline(args, n, src, dst, seed, stream)
    if rank == 0:
        print(json.dumps(out), flush=True)


def make_multi_workload(name, log2n):
    cfg = MULTI_WORKLOADS[name]
    full = cfg["log2n"]
    log2n = log2n or full
    n = 1 << log2n
    m = cfg["m"] >> (full - log2n) if log2n <= full else cfg["m"] << (log2n - full)
    S, batches = cfg["S"], cfg["batches"]
    base = W.BASE_SEED + (3 if cfg["graph"] == "chunglu" else 5)
    if cfg["graph"] == "chunglu":
        gen, lo, hi = W.chung_lu_graph(n, m, seed=base)
        src = np.concatenate([lo, hi])
        dst = np.concatenate([hi, lo])
        sizes = W.log_uniform_sizes(batches, 10, 10000, seed=base + 300)
        stream = W.undirected_update_stream(lo, hi, n, sizes, base + 301, gen.sample)
        seeds = W.rng_for(base + 302).choice(n, S, replace=False).astype(np.int32)
        desc = ("undirected Chung-Lu (exponent 2.1, mean degree 16), both directions stored; "
                "batches of log-uniform 10..10000 undirected edges, half insertions")
    else:
        gen, src, dst = W.rmat_graph(log2n, m, seed=base)
        seeds = W.rng_for(base + 302).choice(n, S, replace=False).astype(np.int32)
        stream = W.node_op_stream(src, dst, n, batches, 1000, 8, 500, 500, base + 301,
                                  protect=tuple(int(s) for s in seeds))
        desc = ("directed R-MAT (a,b,c,d=.57,.19,.19,.05), ids permuted; batches of 10,000 ops: "
                "500 edge ops, 1,000 new nodes x 8 out-edges, 500 node deletions")
    config = {"workload": name if log2n == full else "%s_at_log2n_%d" % (name, log2n),
              "graph": desc, "nodes": n, "edges": int(src.size), "seeds": S,
              "seed_rule": "uniform", "c": C_RESTART, "eps": cfg["eps"],
              "batches": len(stream), "gather_vectors": cfg["precision"], "sums": "fp64",
              "inputs": "update batches resident in HBM before the timed region",
              "l2": "working set (score block) larger than L2"}
    return cfg, n, src, dst, seeds, stream, config


def multi_alg_bytes(st, m, S, by):
    """Algorithmic bytes of one seed-block launch: its pull steps, counted as in
    alg_bytes for S seeds (the seed block never pushes)."""
    return alg_bytes(dict(st, push_iterations=0), 0, m, by, 0, S=S)


def run_multi(args, rank, world):
    import torch

    from paper_1712_00595_gb300 import native as N

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, n, src, dst, seeds, stream, config = make_multi_workload(args.workload, args.log2n)
    K = min(args.steps, len(stream) - 3)
    Wm = min(args.warmup, len(stream) - K)
    prec = {"fp32": N.OSP_PREC_FP32_ACC64, "bf16": N.OSP_PREC_BF16_ACC64}[cfg["precision"]]
    by = {"fp32": 4, "bf16": 2}[cfg["precision"]]
    S = len(seeds)
    Sp = 32 * (1 if S <= 32 else 2 if S <= 64 else 4 if S <= 128 else 8)
    offs = np.cumsum([0] + [b.size for b in stream])
    ops_dev = torch.from_numpy(np.concatenate(stream).view(np.int32).copy()).to(dev)
    base_ptr = ops_dev.data_ptr()
    tstream = torch.cuda.Stream(device=dev)
    eps = cfg["eps"]
    eps_init = 1e-8
    sample = np.linspace(0, S - 1, min(args.fp64_seeds, S)).astype(int) if args.fp64_seeds else []

    gather = {"auto": 0, "regs": N.SEED_GATHER_REGISTERS, "bulk": N.SEED_GATHER_BULK}[args.seed_gather]

    def engine(p):
        e = N.Engine(precision=p, device=local, stream=tstream.cuda_stream, seed_gather=gather,
                     autotune=args.autotune)
        e.load_graph(n, src, dst)
        e.set_seeds(seeds, C_RESTART)
        return e

    eng = engine(prec)
    eng.init_scores(eps_init)
    counts = [eng.get_seed_stats()[0].copy()]
    for b in range(Wm):
        eng.apply_updates_device(base_ptr + 12 * int(offs[b]), int(stream[b].size), eps)
        counts.append(eng.get_seed_stats()[0].copy())
    torch.cuda.synchronize()
    dist_barrier(world)
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    for k in range(K):
        b = Wm + k
        ev[k][0].record(tstream)
        stats.append(eng.apply_updates_device(base_ptr + 12 * int(offs[b]), int(stream[b].size), eps))
        ev[k][1].record(tstream)
        counts.append(eng.get_seed_stats()[0].copy())
    torch.cuda.synchronize()
    clk = clocks.stop()
    dist_barrier(world)
    ms = [a.elapsed_time(b) for a, b in ev]
    steps_us = eng.get_step_times()
    r_s = {int(j): eng.query(int(j)) for j in sample}
    schedule = list(eng.get_schedule())
    eng.close()
    t = dist_max(sum(ms) / 1e3, world)
    value = world * K / t
    prop_ms = sum(s["ms_propagate"] for s in stats)
    ab = sum(multi_alg_bytes(s, s["m_edges"], S, by) for s in stats)
    peak, peak_kind = peaks()
    step_bytes = multi_alg_bytes(dict(stats[-1], iterations=1), stats[-1]["m_edges"], S, by)
    med_step = float(np.median(steps_us[1:])) if len(steps_us) > 1 else float("nan")
    out = {
        "metric": METRIC, "value": value, "unit": "batches/s", "seed_batches_per_s": value * S,
        "n_gpus": world, "steps": K, "warmup": Wm, "ms_per_step": 1e3 * t / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": cfg["precision"], "accumulate": "f64", "data": "synthetic", "config": dict(config, seed_gather=args.seed_gather, autotune=bool(args.autotune),
                       schedule=schedule),
        "roofline": {"bound": "hbm", "achieved": ab / (prop_ms / 1e3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": ab / (prop_ms / 1e3) / 1e9 / peak, "traffic": None,
                     "kernel": "k_propagate_multi", "peak_kind": peak_kind + " (hbm_gbs copy)",
                     "alg_bytes_per_launch": ab / K, "ms_per_launch": prop_ms / K,
                     "pull_step": {"alg_bytes": step_bytes, "median_us": med_step,
                                   "frac": step_bytes / (med_step * 1e-6) / 1e9 / peak}},
        "phases_ms_per_step": {"update_merge_offset": sum(s["ms_update"] for s in stats) / K,
                               "propagation": prop_ms / K},
        "iterations_per_step": float(np.mean([s["iterations"] for s in stats])),
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "clocks": clk,
        "last_step_profile_us": {"x0": float(steps_us[0]),
                                 "steps": [round(float(x), 1) for x in steps_us[1:]]},
    }
    if len(sample):
        # the plain FP64 path, replaying every seed's step counts (lock-step)
        e64 = engine(N.OSP_PREC_FP64)
        e64.set_seed_iterations(counts[0])
        e64.init_scores(eps_init)
        ms64 = []
        for b in range(Wm + K):
            e64.set_seed_iterations(counts[b + 1])
            st = e64.apply_updates_device(base_ptr + 12 * int(offs[b]), int(stream[b].size), eps)
            if b >= Wm:
                ms64.append(st["ms_update"] + st["ms_propagate"])
        l1s = [float(np.abs(r_s[j] - e64.query(j)).sum()) for j in r_s]
        e64.close()
        out["l1_vs_fp64"] = {"max": max(l1s), "mean": float(np.mean(l1s)), "seeds": len(l1s)}
        out["fp64_path"] = {"value": K / (sum(ms64) / 1e3), "unit": "batches/s"}
        out["speedup_vs_fp64"] = value / world / out["fp64_path"]["value"]
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_serve(args, rank, world):
    """The serving loop on R-MAT scale 22 with 256 tracked seeds: Poisson
    arrivals at 2,000 requests/s, half update requests (log-uniform 1..5,000
    ops, half insertions) and half top-100 queries for 1..32 seeds."""
    import torch

    from paper_1712_00595_gb300 import native as N
    from paper_1712_00595_gb300 import serve as SV

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    log2n = args.log2n or 22
    n_req, warm = 4000, 200
    rate, qfrac, S = 2000.0, 0.5, 256
    base = W.BASE_SEED + 7
    gen, src, dst = W.rmat_graph(log2n, 16 << log2n, seed=base)
    n = gen.n
    seeds = W.rng_for(base + 1).choice(n, S, replace=False).astype(np.int32)
    sizes = W.log_uniform_sizes(n_req + warm, 1, 5000, seed=base + 2)
    stream = W.sized_update_stream(src, dst, n, sizes, base + 3, gen.sample)
    reqs = SV.poisson_requests(rate, n_req + 2 * warm, S, stream, qfrac, base + 4)
    eng = N.Engine(precision=N.OSP_PREC_FP32_ACC64, device=local, use_graphs=True)
    eng.load_graph(n, src, dst)
    eng.set_seeds(seeds, C_RESTART)
    eng.init_scores(1e-8)
    nc = n + n // 4 + 4096
    budget = 2 << 30
    slots = int(min(64, budget // SV.slot_bytes(nc)))
    srv = SV.Server(eng, slots, eps=1e-6, policy=args.serve_policy)
    srv.run(reqs[:warm], realtime=False)  # first graph captures, warm caches
    t_first = reqs[warm].t
    timed = [type(r)(r.t - t_first, *[getattr(r, f) for f in r.__dataclass_fields__ if f != "t"])
             for r in reqs[warm:]]
    b0 = len(srv.batches)
    t0 = time.perf_counter()
    got = srv.run(timed, realtime=True)
    wall = time.perf_counter() - t0
    eng.close()
    upd = SV.latency_summary(got, SV.Update)
    qry = SV.latency_summary(got, SV.Query)
    sizes_b = srv.batches[b0:]
    out = {
        "metric": "served requests/s with p50/p99 latency (update batches and top-100 queries)",
        "value": len(got) / wall, "unit": "requests/s", "n_gpus": world, "steps": len(got),
        "warmup": warm, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "accumulate": "f64", "data": "synthetic",
        "config": {"workload": "serve22" if log2n == 22 else "serve_at_log2n_%d" % log2n,
                   "graph": "R-MAT scale %d, ids permuted" % log2n, "nodes": n, "edges": int(src.size),
                   "tracked_seeds": S, "offered_rate": rate, "query_fraction": qfrac,
                   "update_ops": "log-uniform 1..5000, half insertions", "query": "top-100 of 1..32 seeds",
                   "eps": 1e-6, "query_slots": slots, "query_hbm_budget_bytes": budget,
                   "policy": args.serve_policy},
        "latency": {"update": upd, "query": qry},
        "offered_seconds": timed[-1].t, "served_seconds": wall,
        "engine_batches": len(sizes_b),
        "ops_per_batch_mean": float(np.mean(sizes_b)) if sizes_b else 0.0,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_location(args, rank, world):
    """Cost of one update against the score of the node it touches (Sec. 3.3:
    ||q_offset||_1 <= (1-c) r[u] times 2): nodes with out-edges are ranked by
    their score into 100 buckets and 10 nodes per bucket each lose one
    out-edge, one batch per deletion (exact mode, eps = 1e-9)."""
    import torch

    from paper_1712_00595_gb300 import native as N

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n, src, dst, seed, _ = make_workload(args.scale, 1)
    eng = N.Engine(precision=N.OSP_PREC_FP32_ACC64, use_graphs=True)
    eng.load_graph(n, src, dst)
    eng.set_seeds([seed], C_RESTART)
    eng.init_scores(1e-10)
    r = eng.query()
    ptr, idx = eng.export_graph(0)
    outdeg = np.diff(ptr)
    cand = np.flatnonzero(outdeg > 0)
    cand = cand[np.lexsort((cand, -r[cand]))]
    rng = W.rng_for(W.BASE_SEED + 11)
    rows = []
    for b, part in enumerate(np.array_split(cand, 100)):
        pick = rng.choice(part, min(10, part.size), replace=False)
        ms, it, q = [], [], []
        for u in pick:
            v = idx[ptr[u] + int(rng.integers(0, outdeg[u]))]
            ops = np.zeros(1, W.UPDATE_DTYPE)
            ops["u"], ops["v"], ops["op"] = u, v, W.OP_DELETE_EDGE
            st = eng.apply_updates(ops, 1e-9)
            ms.append(st["ms_update"] + st["ms_propagate"])
            it.append(st["iterations"])
            q.append(st["qoff_l1"])
            outdeg[u] = 0  # one deletion per node
        rows.append({"bucket": b, "score_mean": float(r[pick].mean()), "ms_mean": float(np.mean(ms)),
                     "iterations_mean": float(np.mean(it)), "qoff_l1_mean": float(np.mean(q))})
    eng.close()
    ms = np.array([x["ms_mean"] for x in rows])
    out = {"metric": "one-edge update cost by score bucket of its source (exact OSP, eps 1e-9)",
           "value": float(ms[:10].mean() / ms[-10:].mean()), "unit": "cost ratio, top 10 vs bottom 10 buckets",
           "n_gpus": world, "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "location_sweep_rmat%d" % args.scale, "buckets": 100, "per_bucket": 10},
           "buckets": rows}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_growshrink(args, rank, world):
    """Cost of a fixed-size batch (1,000 edges) against the graph size: the
    graph grows from half of its edges to all of them in 32 steps and then
    shrinks back; each step applies one measured 1,000-edge batch (insertions
    while growing, deletions while shrinking) and then the rest of its 1/32
    share as one large untimed batch (OSP-T, eps = 1e-6)."""
    import torch

    from paper_1712_00595_gb300 import native as N

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    gen, src, dst = W.rmat_graph(args.scale, 16 << args.scale, seed=W.BASE_SEED + HUB_SEED_OFFSET)
    n = gen.n
    seed = W.max_out_degree_seed(n, src)
    order = W.rng_for(W.BASE_SEED + 12).permutation(src.size)
    half = src.size // 2
    base, extra = order[:half], order[half:]
    eng = N.Engine(precision=N.OSP_PREC_FP32_ACC64, use_graphs=True)
    eng.load_graph(n, src[base], dst[base])
    eng.set_seeds([seed], C_RESTART)
    eng.init_scores(1e-10)
    steps = 32
    chunk = extra.size // steps
    rows = []

    def batch(sel, op):
        ops = np.zeros(sel.size, W.UPDATE_DTYPE)
        ops["u"], ops["v"], ops["op"] = src[sel], dst[sel], op
        return eng.apply_updates(ops, 1e-6)

    for phase in ("grow", "shrink"):
        op = W.OP_INSERT_EDGE if phase == "grow" else W.OP_DELETE_EDGE
        for k in range(steps):
            part = extra[k * chunk:(k + 1) * chunk]
            st = batch(part[:1000], op)  # the measured batch of fixed size
            rows.append({"phase": phase, "m": int(st["m_edges"]), "iterations": int(st["iterations"]),
                         "ms": float(st["ms_update"] + st["ms_propagate"]),
                         "qoff_l1": float(st["qoff_l1"])})
            batch(part[1000:], op)  # the rest of the chunk: the graph moves on
    eng.close()
    out = {"metric": "update cost as the graph grows and shrinks (1,000-edge batches, eps 1e-6)",
           "value": float(np.mean([x["ms"] for x in rows])), "unit": "ms per batch (mean)",
           "n_gpus": world, "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "growshrink_rmat%d" % args.scale, "batches_per_phase": steps},
           "batches": rows}
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "serve22":
        run_serve(args, rank, world)
    elif args.workload == "location":
        run_location(args, rank, world)
    elif args.workload == "growshrink":
        run_growshrink(args, rank, world)
    elif args.workload != "rmat20":
        run_multi(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
