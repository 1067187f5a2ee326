#!/usr/bin/env python
"""Benchmark of the OSP / OSP-T update path on one GB300 (or N independent replicas).

Headline workload (the paper's Table 3 graphs are stood in for by seeded
synthetic graphs): directed R-MAT scale 24 (16,777,216 nodes, 268,435,456
unique edges, a,b,c,d = .57,.19,.19,.05, ids permuted), c = 0.15, 256 uniform
seeds tracked as one n x 256 score block, bf16 gather vectors with FP32
products and FP64 sums, OSP-T eps = 1e-6; batches of 10,000 ops: 500 edge ops
(half insertions of absent edges, half deletions), 1,000 new nodes with 8
out-edges each, 500 deletions of existing nodes (Sec. 3.4.1). A step is one
batch through the whole path: ingest + validation, graph-store merge, offset
block, propagation of every seed to its own ||x||_1 <= eps, merge into the
scores.

Reported on one line: batches/s with the batches resident in HBM, the
propagation kernel's algorithmic GB/s against the measured HBM copy bandwidth,
the L1 distance of sampled seeds to the plain FP64 path replaying each seed's
step counts, the end-to-end rate through the host API, the FP64 CPU oracle on
a bounded sample of the same workload, and (unless --no-extras) the one-seed
R-MAT scale-20 benchmark, the 64-seed Chung-Lu workload, the serving loop and
the Sec. 3.3 / scalability sweeps as nested fields.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import math
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
HEADLINE = "rmat24_s256"


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


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--scale", type=int, default=20, help="rmat20 workload: R-MAT scale")
    p.add_argument("--eps", type=float, default=1e-6)
    p.add_argument("--eps-init", type=float, default=1e-10)
    p.add_argument("--no-extras", action="store_true",
                   help="the workload's own line only (profiling runs)")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="rmat20: CPU time bound of the cpu_baseline sample (whole batches)")
    p.add_argument("--cpu-batches", type=int, default=3,
                   help="seed-block workloads: batches in the oracle's cpu_baseline sample")
    p.add_argument("--node-order", type=int, default=0, choices=[0, 1],
                   help="rmat20: internal node order, 0 = caller ids, 1 = descending out-degree")
    p.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="keep the default pull-step schedule (osp_init_scores tunes it otherwise)")
    p.add_argument("--launch", default="graphs", choices=["graphs", "eager"],
                   help="batch kernels replayed from CUDA graphs, or launched one by one")
    p.add_argument("--workload", default=HEADLINE,
                   choices=["rmat20", "serve22", "location", "growshrink"] + sorted(MULTI_WORKLOADS),
                   help="rmat24_s256 (default): 256 seeds at R-MAT scale 24; rmat20: one seed")
    p.add_argument("--serve-policy", default="latest", choices=["ordered", "latest"],
                   help="serve22: queries read in arrival order, or the newest scores")
    p.add_argument("--log2n", type=int, default=0,
                   help="several-seed workloads: nodes 2^log2n (edges scaled alike; 0 = full size)")
    p.add_argument("--seed-gather", default="auto", choices=["auto", "regs", "bulk"],
                   help="seed-block workloads: source rows gathered into registers, or "
                        "staged in shared memory by bulk asynchronous copies (auto: the "
                        "engine's choice by row size)")
    p.add_argument("--seed-group", type=int, default=0, choices=[0, 32, 64, 128, 256],
                   help="seed-block workloads: columns per column group (0: the engine's default)")
    p.add_argument("--l2-hot-bytes", type=int, default=0,
                   help="seed-block workloads: L2 bytes for the rows of high out-degree "
                        "sources (0: the engine's default, -1: none)")
    p.add_argument("--fp64-seeds", type=int, default=8,
                   help="several-seed workloads: seeds compared with the FP64 replay (0 = skip)")
    p.add_argument("--e2e-batches", type=int, default=8,
                   help="several-seed workloads: batches timed through the host API")
    return p.parse_args(argv)


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


# DRAM traffic records (profiles/*_traffic.txt): bytes per launch from one ncu
# capture, valid only for the kernel sources they were taken on.
TRAFFIC_RECORDS = {
    "k_propagate<float>": ("propagate_rmat20_traffic.txt", ("propagate.cu", "common.cuh")),
    "k_propagate_multi": ("propagate_multi_rmat24_s256_traffic.txt", ("multi.cu", "common.cuh")),
}
TRAFFIC_SOURCES = TRAFFIC_RECORDS["k_propagate<float>"][1]


def kernel_source_hash(sources=TRAFFIC_SOURCES):
    """First 16 hex digits of the SHA-256 of a kernel's sources."""
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_1712_00595_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel="k_propagate<float>"):
    """The committed traffic record of a kernel as a dict, if it was taken on
    the current kernel sources (else None)."""
    name, sources = TRAFFIC_RECORDS[kernel]
    try:
        vals = {}
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("source_sha256_16") != kernel_source_hash(sources):
            return None
        return vals
    except Exception:
        return None


def traffic_from_profile():
    """Per-launch DRAM bytes of the one-seed propagation kernel from its
    committed ncu summary, if taken on the current kernel sources (else None)."""
    rec = traffic_record("k_propagate<float>")
    try:
        return float(rec["dram_bytes_per_launch"]) if rec else None
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


def log(msg):
    print("[bench] " + msg, file=sys.stderr, flush=True)


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


# ---------------------------------------------------------------------------
# Seed-block workloads
# ---------------------------------------------------------------------------
def multi_alg_bytes(st, m, col_steps, by):
    """Algorithmic bytes of one seed-block launch (the seed block never pushes):
    per pull step the in-list ids and list starts, 4 m + 4 (|V| + 1); per step
    of each seed that propagates (col_steps = the sum of those seeds' step
    counts) its column of the gather block once per source and its y write and
    FP64 score read and write per destination, by |src| + (by + 16) |V|, plus
    its 8-byte |x| partial. A seed whose offset is zero has nothing to move."""
    steps = st["iterations"]
    V, src = st["pull_dst_nodes"], st["pull_src_nodes"]
    return steps * (4 * m + 4 * (V + 1)) + col_steps * (by * src + (by + 16) * V + 8)


def make_multi_workload(name, log2n, batches=None):
    """Graph, seeds and update stream of a seed-block workload; `batches`
    overrides the workload's stream length (the benchmark draws warm-up, timed
    and end-to-end batches of the same construction)."""
    cfg = MULTI_WORKLOADS[name]
    full = cfg["log2n"]
    log2n = log2n or full
    n = 1 << log2n
    m = cfg["m"] >> (full - log2n) if log2n <= full else cfg["m"] << (log2n - full)
    S = cfg["S"]
    batches = batches or cfg["batches"]
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
              "l2": "not flushed: the score block (%.1f GB) is larger than L2"
                    % (8.0 * n * S / 1e9)}
    return cfg, n, src, dst, seeds, stream, config


def oracle_multi_sample(n, src, dst, seeds, stream, batches, skip=0, cpi_steps=8, eps=1e-6,
                        c=C_RESTART, log_fn=None):
    """The FP64 CPU oracle, as it stands, on a bounded sample of a seed-block
    workload: two of the seeds, one with out-edges ("live") and one without
    (a dead-end seed, whose scores stay c e_s unless a batch gives it
    out-edges).

    The live seed starts from the oracle's own CPI cut after `cpi_steps`
    steps, the dead-end seed from its exact CPI. The first `skip` batches only
    update the oracle's graph. For each later batch the oracle applies the
    batch and exports the new CSR (t_graph), then runs Algorithm 1 to its own
    stopping rule for each sampled seed (t_live, t_dead). A batch for all S
    seeds is t_graph + S_live t_live + S_dead t_dead, with S_live / S_dead the
    seeds with / without out-edges in the loaded graph. Returns per-batch
    records and the sample's totals."""
    from oracle import oracle as O
    say = log_fn or (lambda m: None)
    t0 = time.perf_counter()
    g = O.Graph(n, src, dst)
    cur = g.csr()
    outdeg = np.diff(cur[0])
    has_out = outdeg[np.asarray(seeds, np.int64)] > 0
    live = int(seeds[int(np.argmax(has_out))]) if has_out.any() else None
    dead = int(seeds[int(np.argmin(has_out))]) if not has_out.all() else None
    n_live, n_dead = int(has_out.sum()), int((~has_out).sum())
    r_live = O.cpi(*cur, live, c, eps, force_iters=cpi_steps)[0] if live is not None else None
    r_dead = O.cpi(*cur, dead, c, eps)[0] if dead is not None else None
    say("oracle set-up (graph + CPI) %.1f s" % (time.perf_counter() - t0))
    recs = []
    protect = tuple(int(x) for x in seeds)
    for b in range(batches):
        t1 = time.perf_counter()
        assert g.apply(stream[b], protect=protect) == -1
        new = g.csr()
        t_graph = time.perf_counter() - t1
        if b < skip:
            cur = new
            continue
        t_live = t_dead = 0.0
        k_live = 0
        if live is not None:
            t2 = time.perf_counter()
            r_live, _, st, _ = O.osp(cur, new, r_live, c, eps)
            t_live = time.perf_counter() - t2
            k_live = int(st["iterations"])
        if dead is not None:
            t3 = time.perf_counter()
            r_dead, _, _, _ = O.osp(cur, new, r_dead, c, eps)
            t_dead = time.perf_counter() - t3
        recs.append({"t_graph": t_graph, "t_live": t_live, "t_dead": t_dead, "k_live": k_live,
                     "batch_s": t_graph + n_live * t_live + n_dead * t_dead,
                     "cpu_s": t_graph + t_live + t_dead})
        cur = new
        say("oracle batch %d: %.1f s of CPU (live seed %d steps), %.1f s estimated for %d seeds"
            % (b, recs[-1]["cpu_s"], k_live, recs[-1]["batch_s"], len(seeds)))
    return {"live_seed": live, "dead_seed": dead, "n_live": n_live, "n_dead": n_dead,
            "records": recs, "batches_per_s": len(recs) / sum(x["batch_s"] for x in recs),
            "cpu_seconds": sum(x["cpu_s"] for x in recs)}


def _oracle_sample_child(path, out_path, batches):
    """Spawned process: the oracle sample on the inputs saved at `path`."""
    z = np.load(path)
    offs = z["offs"]
    ops = z["ops"]
    stream = [ops[offs[i]:offs[i + 1]] for i in range(offs.size - 1)]
    res = oracle_multi_sample(int(z["n"]), z["src"], z["dst"], z["seeds"], stream, batches,
                              eps=float(z["eps"]))
    with open(out_path, "w") as f:
        json.dump(res, f)


class OracleSample:
    """The cpu_baseline leg of a seed-block workload: the oracle sample runs in
    a spawned process (one host core) while the GPU part of the benchmark runs."""

    def __init__(self, n, src, dst, seeds, stream, eps, batches):
        import multiprocessing as mp
        self.dir = tempfile.mkdtemp(prefix="osp_oracle_")
        path = os.path.join(self.dir, "in.npz")
        offs = np.cumsum([0] + [b.size for b in stream[:batches]])
        np.savez(path, n=n, src=src, dst=dst, seeds=seeds, eps=eps, offs=offs,
                 ops=np.concatenate(stream[:batches]))
        self.out = os.path.join(self.dir, "out.json")
        self.proc = mp.get_context("spawn").Process(target=_oracle_sample_child,
                                                    args=(path, self.out, batches))
        self.proc.start()

    def result(self, timeout=1800.0):
        self.proc.join(timeout)
        if self.proc.is_alive():
            self.proc.terminate()
            self.proc.join(10)
            return None
        try:
            with open(self.out) as f:
                return json.load(f)
        except Exception:
            return None
        finally:
            for name in ("in.npz", "out.json"):
                try:
                    os.unlink(os.path.join(self.dir, name))
                except OSError:
                    pass
            try:
                os.rmdir(self.dir)
            except OSError:
                pass


def cpu_baseline_multi(res, S):
    """The cpu_baseline object of a seed-block workload from an oracle sample."""
    if not res:
        return None
    recs = res["records"]
    return {"value": res["batches_per_s"], "unit": "batches/s", "cores": 1, "kind": "oracle",
            "sample": ("%d batches of the workload for two seeds, one with out-edges (from the "
                       "oracle's CPI cut after 8 steps) and one dead-end seed: graph update and "
                       "CSR export, then Algorithm 1 to the oracle's own stopping rule per seed; "
                       "a batch for all %d seeds = t_graph + %d t_live + %d t_dead (seeds with / "
                       "without out-edges); single-threaded FP64 C"
                       % (len(recs), S, res["n_live"], res["n_dead"])),
            "seconds_of_cpu": res["cpu_seconds"],
            "per_batch_s": [round(x["batch_s"], 2) for x in recs],
            "live_seed_steps": [x["k_live"] for x in recs]}


def run_multi(args, rank, world, name=None, steps=None, warmup=None, extras=True):
    """A seed-block workload: warm-up and timed batches on the device-resident
    stream, then end-to-end batches through the host API, the FP64 replay of
    sampled seeds in lock-step, and the oracle's cpu_baseline sample."""
    import torch

    from paper_1712_00595_gb300 import native as N

    name = name or args.workload
    K = steps if steps is not None else args.steps
    Wm = warmup if warmup is not None else args.warmup
    E = min(K, args.e2e_batches) if extras else 0
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_setup = time.perf_counter()
    cfg, n, src, dst, seeds, stream, config = make_multi_workload(name, args.log2n, Wm + K + E)
    log("%s drawn in %.1f s" % (config["workload"], time.perf_counter() - t_setup))
    oracle = None
    if extras and rank == 0 and world == 1:
        oracle = OracleSample(n, src, dst, seeds, stream, cfg["eps"], args.cpu_batches)
    prec = {"fp32": N.OSP_PREC_FP32_ACC64, "bf16": N.OSP_PREC_BF16_ACC64}[cfg["precision"]]
    by = {"fp32": 4, "bf16": 2}[cfg["precision"]]
    S = len(seeds)
    offs = np.cumsum([0] + [b.size for b in stream])
    ops_dev = torch.from_numpy(np.concatenate(stream[:Wm + K]).view(np.int32).copy()).to(dev)
    base_ptr = ops_dev.data_ptr()
    tstream = torch.cuda.Stream(device=dev)
    eps = cfg["eps"]
    eps_init = 1e-8
    sample = (np.linspace(0, S - 1, min(args.fp64_seeds, S)).astype(int)
              if args.fp64_seeds and extras else np.zeros(0, int))
    gather = {"auto": 0, "regs": N.SEED_GATHER_REGISTERS, "bulk": N.SEED_GATHER_BULK}[args.seed_gather]

    def engine(p, seed_set):
        e = N.Engine(precision=p, device=local, stream=tstream.cuda_stream, seed_gather=gather,
                     autotune=args.autotune, node_order=1, seed_group=args.seed_group,
                     l2_hot_bytes=args.l2_hot_bytes)
        e.load_graph(n, src, dst)
        e.set_seeds(seed_set, C_RESTART)
        return e

    t0 = time.perf_counter()
    eng = engine(prec, seeds)
    log("graph loaded in %.1f s" % (time.perf_counter() - t0))
    t0 = time.perf_counter()
    eng.init_scores(eps_init)
    log("scores initialised in %.1f s" % (time.perf_counter() - t0))
    it0, q0, _ = eng.get_seed_stats()
    counts, qs = [it0.copy()], [q0.copy()]
    for b in range(Wm):
        eng.apply_updates_device(base_ptr + 12 * int(offs[b]), int(stream[b].size), eps)
        it, q, _ = eng.get_seed_stats()
        counts.append(it.copy())
        qs.append(q.copy())
    torch.cuda.synchronize()
    dist_barrier(world)
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed batches
    for k in range(K):
        b = Wm + k
        ev[k][0].record(tstream)
        stats.append(eng.apply_updates_device(base_ptr + 12 * int(offs[b]), int(stream[b].size), eps))
        ev[k][1].record(tstream)
        it, q, _ = eng.get_seed_stats()
        counts.append(it.copy())
        qs.append(q.copy())
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    dist_barrier(world)
    ms = [a.elapsed_time(b) for a, b in ev]
    steps_us = eng.get_step_times()
    t = dist_max(sum(ms) / 1e3, world)
    value = world * K / t
    prop_ms = sum(s["ms_propagate"] for s in stats)
    # column-steps of the timed batches: each seed's steps, for seeds whose offset is nonzero
    col_steps = [int(counts[Wm + 1 + k][qs[Wm + 1 + k] > 0].sum()) for k in range(K)]
    ab = sum(multi_alg_bytes(s, s["m_edges"], cs, by) for s, cs in zip(stats, col_steps))
    peak, peak_kind = peaks()
    achieved = ab / (prop_ms / 1e3) / 1e9
    dense_step = multi_alg_bytes(dict(stats[-1], iterations=1), stats[-1]["m_edges"], S, by)
    hist = np.bincount(np.concatenate(counts[Wm + 1:]).astype(np.int64))
    rec = traffic_record("k_propagate_multi")
    traffic = None
    if rec and config["workload"] == HEADLINE:
        # DRAM bytes per algorithmic byte of the small-case capture, times this run's bytes
        traffic = float(rec["dram_bytes_per_alg_byte"]) * ab / K
    out = {
        "metric": METRIC, "value": value, "unit": "batches/s", "seed_batches_per_s": value * S,
        "n_gpus": world, "steps": K, "warmup": Wm, "ms_per_step": 1e3 * t / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if cfg["precision"] == "bf16" else "f32", "accumulate": "f64",
        "data": "synthetic",
        "config": dict(config, seed_gather=args.seed_gather, autotune=bool(args.autotune),
                       schedule=list(eng.get_schedule()), node_order="descending out-degree",
                       seed_group=args.seed_group or (32 if cfg["precision"] == "bf16"
                                                      else 32 * ((S + 31) // 32)),
                       column_groups="packed per batch by offset size" if cfg["precision"] == "bf16"
                       and S > 32 and args.seed_group in (0, 32) else "fixed"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_per_alg_byte": float(rec["dram_bytes_per_alg_byte"])
                     if traffic is not None else None,
                     "traffic_source": rec.get("source") if traffic is not None else None,
                     "kernel": "k_propagate_multi", "peak_kind": peak_kind + " (hbm_gbs copy)",
                     "alg_bytes_per_launch": ab / K, "ms_per_launch": prop_ms / K,
                     "dense_step_alg_bytes": dense_step},
        "phases_ms_per_step": {"update_merge_offset": sum(s["ms_update"] for s in stats) / K,
                               "propagation": prop_ms / K},
        "batch_ms": {"median": float(np.median(ms)), "p99": float(np.percentile(ms, 99)),
                     "max": float(max(ms))},
        "iterations_per_step": float(np.mean([s["iterations"] for s in stats])),
        "column_steps_per_batch": float(np.mean(col_steps)),
        "seed_step_histogram": [int(x) for x in hist],
        "zero_offset_seeds_per_batch": float(np.mean([(q <= 0).sum() for q in qs[Wm + 1:]])),
        "pull_nodes": {"dst": int(stats[-1]["pull_dst_nodes"]), "src": int(stats[-1]["pull_src_nodes"])},
        "residual_bound_max": float(max(s["residual_bound"] for s in stats)),
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "clocks": clk,
        "last_step_profile_us": {"x0": float(steps_us[0]),
                                 "steps": [round(float(x), 1) for x in steps_us[1:]]},
    }
    # ---- end to end through the host API: host batch in, top-100 of sampled seeds out ----
    if E > 0:
        host_ops = [np.ascontiguousarray(stream[Wm + K + k]) for k in range(E)]
        q_seeds = [int(j) for j in (sample if sample.size else range(min(8, S)))]
        torch.cuda.synchronize()
        per = []
        t0 = time.perf_counter()
        for k in range(E):
            ta = time.perf_counter()
            eng.apply_updates(host_ops[k], eps)
            for j in q_seeds:
                eng.topk(100, seed_idx=j)
            per.append(time.perf_counter() - ta)
            it, q, _ = eng.get_seed_stats()
            counts.append(it.copy())
            qs.append(q.copy())
        dt = time.perf_counter() - t0
        out["e2e"] = {"value": E / dt, "unit": "batches/s",
                      "h2d_bytes_per_step": int(np.mean([12 * o.size for o in host_ops])),
                      "d2h_bytes_per_step": len(q_seeds) * 100 * 12,
                      "result": "top-100 (ids, scores) of %d tracked seeds per batch (osp_topk)"
                                % len(q_seeds),
                      "batches": E, "batch_ms": {"median": 1e3 * float(np.median(per)),
                                                 "p99": 1e3 * float(np.percentile(per, 99))}}
    else:
        out["e2e"] = None
    r_s = {int(j): eng.query(int(j)) for j in sample}
    eng.close()
    total = Wm + K + E
    if sample.size:
        # the plain FP64 path on the sampled seeds, replaying every seed's step
        # counts batch by batch (lock-step)
        e64 = engine(N.OSP_PREC_FP64, seeds[sample])
        e64.set_seed_iterations(counts[0][sample])
        e64.init_scores(eps_init)
        ops_all = torch.from_numpy(np.concatenate(stream[:total]).view(np.int32).copy()).to(dev)
        p64 = ops_all.data_ptr()
        ms64 = []
        for b in range(total):
            e64.set_seed_iterations(counts[b + 1][sample])
            st = e64.apply_updates_device(p64 + 12 * int(offs[b]), int(stream[b].size), eps)
            if Wm <= b < Wm + K:
                ms64.append(st["ms_update"] + st["ms_propagate"])
        l1s, rk = [], []
        for i, j in enumerate(sample):
            r64 = e64.query(i)
            l1s.append(float(np.abs(r_s[int(j)] - r64).sum()))
            rk.append(rank_accuracy(r_s[int(j)], r64))
        e64.close()
        del ops_all
        out["l1_vs_fp64"] = {"max": max(l1s), "mean": float(np.mean(l1s)), "seeds": len(l1s),
                             "batches": total}
        out["rank_vs_fp64"] = {"spearman_min": min(x["spearman"] for x in rk),
                               "top100_overlap_min": min(x["top100_overlap"] for x in rk)}
        out["fp64_path"] = {"value": K / (sum(ms64) / 1e3), "unit": "batches/s",
                            "seeds": len(sample),
                            "note": "FP64 block of the sampled seeds only, same batches"}
    if oracle is not None:
        out["cpu_baseline"] = cpu_baseline_multi(oracle.result(), S)
    return out


# ---------------------------------------------------------------------------
# One seed: R-MAT scale 20
# ---------------------------------------------------------------------------
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


def l1_lookup_roofline(stats, prop_ms, clk, sms):
    """Gathers per second of the one-seed propagation against one L1 sector
    lookup per SM cycle (sms SMs at the median SM clock sampled during the
    timed region)."""
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    lookups = float(sum(s["visited_edges"] for s in stats))
    achieved = lookups / (prop_ms / 1e3) / 1e9
    peak = sms * mhz * 1e6 / 1e9
    return {"bound": "l1 lookups", "achieved": achieved, "peak": peak, "unit": "G lookups/s",
            "frac": achieved / peak, "basis": "one random 4-byte gather per visited edge, one "
            "32-byte sector lookup per SM cycle (%d SMs at %.0f MHz)" % (sms, mhz)}


def run_ours(args, rank, world, steps=None, warmup=None, extras=True):
    import torch

    from paper_1712_00595_gb300 import native as N

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K = steps if steps is not None else args.steps
    Wm = warmup if warmup is not None else args.warmup
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
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed batches
    ms, stats = run(eng, args.eps, 0)
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    iters = warm_iters + [s["iterations"] for s in stats]
    st_us = eng.get_step_times()
    step_profile = {"x0": float(st_us[0]), "steps": [round(float(x), 1) for x in st_us[1:]]}
    r_mixed = eng.query()
    schedule = eng.get_schedule()
    # the paper's baseline on the GPU: CPI from scratch on the final graph at the same eps
    cpi_gpu = None
    if extras:
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
        # the working set of this kernel lives in L2; its ceiling is the rate of
        # the random 4-byte gathers (one per visited edge), each a 32-byte sector
        # lookup in L1, at one lookup per SM cycle
        "roofline_l1": l1_lookup_roofline(
            stats, prop_ms, clk, torch.cuda.get_device_properties(local).multi_processor_count),
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

    if extras:
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

    if rank == 0 and world == 1 and extras:
        out["cpu_baseline"] = cpu_baseline(args, n, src, dst, seed, stream)
    return out



# ---------------------------------------------------------------------------
# Serving and the sweeps
# ---------------------------------------------------------------------------
def run_serve(args, rank, world, n_req=4000):
    """The serving loop on R-MAT scale 22 with 256 tracked seeds: Poisson
    arrivals at 2,000 requests/s, half update requests (log-uniform 1..5,000
    ops, half insertions) and half top-100 queries for 1..32 seeds."""
    import torch

    from paper_1712_00595_gb300 import native as N
    from paper_1712_00595_gb300 import serve as SV

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    log2n = args.log2n or 22
    warm = 200
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
    return {
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
        "topk_seeds": {"ranked": srv.topk_computed, "reused_same_version": srv.topk_reused},
        "ops_per_batch_mean": float(np.mean(sizes_b)) if sizes_b else 0.0,
    }


def run_location(args, rank, world, per_bucket=10):
    """Cost of one update against the score of the node it touches (Sec. 3.3:
    ||q_offset||_1 <= (1-c) r[u] times 2): nodes with out-edges are ranked by
    their score into 100 buckets and `per_bucket` nodes per bucket each lose one
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
    push_steps = 0
    for b, part in enumerate(np.array_split(cand, 100)):
        pick = rng.choice(part, min(per_bucket, part.size), replace=False)
        ms, it, q = [], [], []
        for u in pick:
            v = idx[ptr[u] + int(rng.integers(0, outdeg[u]))]
            ops = np.zeros(1, W.UPDATE_DTYPE)
            ops["u"], ops["v"], ops["op"] = u, v, W.OP_DELETE_EDGE
            st = eng.apply_updates(ops, 1e-9)
            ms.append(st["ms_update"] + st["ms_propagate"])
            it.append(st["iterations"])
            q.append(st["qoff_l1"])
            push_steps += st["push_iterations"]
            outdeg[u] = 0  # one deletion per node
        rows.append({"bucket": b, "score_mean": float(r[pick].mean()), "ms_mean": float(np.mean(ms)),
                     "iterations_mean": float(np.mean(it)), "qoff_l1_mean": float(np.mean(q))})
    eng.close()
    ms = np.array([x["ms_mean"] for x in rows])
    return {"metric": "one-edge update cost by score bucket of its source (exact OSP, eps 1e-9)",
           "value": float(ms[:10].mean() / ms[-10:].mean()), "unit": "cost ratio, top 10 vs bottom 10 buckets",
           "n_gpus": world, "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "location_sweep_rmat%d" % args.scale, "buckets": 100,
                      "per_bucket": per_bucket},
           "push_steps_total": int(push_steps),
           "buckets": rows}


def run_growshrink(args, rank, world, steps=32):
    """Cost of a fixed-size batch (1,000 edges) against the graph size: the
    graph grows from half of its edges to all of them in `steps` steps and then
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
    return {"metric": "update cost as the graph grows and shrinks (1,000-edge batches, eps 1e-6)",
           "value": float(np.mean([x["ms"] for x in rows])), "unit": "ms per batch (mean)",
           "n_gpus": world, "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "growshrink_rmat%d" % args.scale, "batches_per_phase": steps},
           "batches": rows}



def summary(line, keys=("value", "unit", "ms_per_step", "steps", "warmup")):
    """A nested benchmark's main figures."""
    out = {k: line.get(k) for k in keys if k in line}
    for k in ("roofline", "roofline_l1", "l1_vs_fp64", "e2e", "cpu_baseline", "fp64_path", "latency",
              "iterations_per_step", "column_steps_per_batch", "phases_ms_per_step", "config",
              "gpu_launches", "push_iterations_per_step", "engine_batches", "offered_seconds",
              "served_seconds", "clocks"):
        if k in line and line[k] is not None:
            out[k] = line[k]
    return out


def run_headline(args, rank, world):
    """The seed-block headline line, with the other workloads nested under it."""
    out = run_multi(args, rank, world, name=HEADLINE, extras=not args.no_extras)
    if args.no_extras or world > 1:
        return out
    nested = {}
    t0 = time.perf_counter()
    nested["rmat20"] = summary(run_ours(args, rank, world))
    log("rmat20 nested in %.1f s" % (time.perf_counter() - t0))
    t0 = time.perf_counter()
    nested["chunglu22_s64"] = summary(run_multi(args, rank, world, name="chunglu22_s64", steps=10,
                                                warmup=3, extras=False))
    log("chunglu22_s64 nested in %.1f s" % (time.perf_counter() - t0))
    t0 = time.perf_counter()
    nested["serve22"] = summary(run_serve(args, rank, world, n_req=2000))
    log("serve22 nested in %.1f s" % (time.perf_counter() - t0))
    t0 = time.perf_counter()
    loc = run_location(args, rank, world, per_bucket=3)
    nested["location_sweep"] = {k: loc[k] for k in ("metric", "value", "unit", "config",
                                                   "push_steps_total")}
    nested["location_sweep"]["ms_by_bucket"] = [round(x["ms_mean"], 3) for x in loc["buckets"]]
    gs = run_growshrink(args, rank, world, steps=8)
    nested["growshrink_sweep"] = {k: gs[k] for k in ("metric", "value", "unit", "config")}
    nested["growshrink_sweep"]["batches"] = [(x["phase"], x["m"], x["iterations"], round(x["ms"], 3))
                                             for x in gs["batches"]]
    log("sweeps nested in %.1f s" % (time.perf_counter() - t0))
    out["nested"] = nested
    return out


# ---------------------------------------------------------------------------
# The reference arm: the FP64 CPU oracle on the same workload
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores, on the same workload and metric.
    Seed-block workloads: each step is the bounded one-seed sample of
    oracle_multi_sample scaled to a whole batch of all seeds; rmat20: each step
    applies one batch and runs Algorithm 1 (graph update, CSR export, offset,
    propagation)."""
    if rank != 0:
        return None
    if args.workload in MULTI_WORKLOADS:
        cfg, n, src, dst, seeds, stream, config = make_multi_workload(
            args.workload, args.log2n, args.warmup + args.steps)
        res = oracle_multi_sample(n, src, dst, seeds, stream, args.warmup + args.steps,
                                  skip=args.warmup, eps=cfg["eps"], log_fn=log)
        recs = res["records"]
        dt = sum(x["batch_s"] for x in recs)
        v = len(recs) / dt
        cb = cpu_baseline_multi(res, len(seeds))
        return {
            "impl": "reference", "metric": METRIC, "value": v, "unit": "batches/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / len(recs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config, gather_vectors="fp64 (CPU oracle)", sums="fp64",
                           l2="n/a (host)", inputs="update batches in host memory"),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "batches/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
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
    return {
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


def main():
    args = parse()
    rank, world = dist_setup(args)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == HEADLINE:
        out = run_headline(args, rank, world)
    elif args.workload == "serve22":
        out = run_serve(args, rank, world)
    elif args.workload == "location":
        out = run_location(args, rank, world)
    elif args.workload == "growshrink":
        out = run_growshrink(args, rank, world)
    elif args.workload in MULTI_WORKLOADS:
        out = run_multi(args, rank, world, extras=not args.no_extras)
    else:
        out = run_ours(args, rank, world, extras=not args.no_extras)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
