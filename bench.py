"""Benchmark of the parallel chordality test on GB300.

Default workload (`--workload dense16k`): the dense N=16,384 pair — a
subtree-intersection chordal graph at edge density ~0.1 (32 MiB of bit-packed
rows) and its copy with 1-10 cycle-closing extra edges.  One step = the whole
test (LexBFS + perfect-elimination check + witness) on both graphs, issued as
one batched call; the metric is chordality tests per second.

Other workloads (same JSON line; not run by default):
  small1k    the N=1,000 pair (subtree model / planted C_k), one batched call
  sparse1m   the N=2^20 CSR pair (reversed-PEO chordal / cycle-closing edges),
             the two graphs on two streams
  sparse64k  the same recipe at N=65,536 (a small case for profiling)
  batch4096  4,096 graphs, N log-uniform in [16, 2048], one captured batch plan
  paper7     the paper's Section 7 families on GB300 beside the CPU oracle:
             cliques N = 1000..11000, dense random (p = 0.5), sparse random
             (M = 20N), trees and chordal graphs at N = 10,000; one table
  serve      Poisson stream of 100,000 queries (continuous-batching queue) drawn
             from a seeded pool of 64 graphs: N log-uniform in [64, 65536],
             density U[0.01, 0.2], dense below N = 8,192, CSR above; arrival
             rate 0.8 x the measured saturation throughput; p50 / p99 latency

`--workload sweep16k` / `sweep1m` time one multi-sweep LexBFS sweep (LexBFS+
of the plain LexBFS order) on each graph of the dense N=16,384 pair / the CSR
N=2^20 pair; unit sweeps/s.

`--order mcs` (dense16k, small1k) runs the same test with the Maximum
Cardinality Search order (Section 5.1) instead of LexBFS: one graph per call,
the two graphs on two streams.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload dense16k|small1k|sparse1m|batch4096|...] [--order lexbfs|mcs]

Timing: inputs resident in HBM; before every timed step a 256 MiB buffer is
written to flush L2; each step is bracketed by CUDA events on the launching
stream.  `e2e` repeats the metric through the public API with pinned host
inputs copied in and results copied out inside the timed region (dense
workloads: the library's host-buffer entry cg_chordal_test_batch_host).
`cpu_baseline` times the CPU oracle on a bounded sample.  For the
single-pair workloads `phases.floor` adds the step's latency floors measured
after the timed region (`cg_step_floor`: a CTA barrier pair, a dependent load
over a 32 MiB and a 1 GiB chain).  With N > 1
(torchrun) every rank runs its own replica (one graph's test does not shard);
value = tests on all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "chordality tests/sec and adjacency GB/s (% of HBM peak), bit-exact; p50/p99 latency"
UNIT = "tests/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_over_ranks(local_ms: float, tests_per_rank: int, device=None):
    """Whole-job timing of replicas: the slowest rank's timed total and the
    rate of all ranks' tests over it (a no-op without torch.distributed)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    return total_ms, tests_per_rank * world / (total_ms / 1e3)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------- workloads

def make_workload(name: str):
    import graphgen as gg
    if name == "dense16k":
        g, h, info = gg.large_dense_pair()
        return [g, h], {"workload": "dense N=16384 subtree-intersection chordal graph (density %.3f, tree %d nodes)"
                                    " + copy with %d cycle-closing edges" % (g.density(), info["tree_nodes"],
                                                                              info["r"]),
                        "n": g.n, "words_per_row": g.words, "graphs_per_step": 2,
                        "edges": [g.num_edges(), h.num_edges()], "bytes_per_graph": g.nbytes}
    if name == "sweep16k":
        g, h, info = gg.large_dense_pair()
        return [g, h], {"workload": "one LexBFS+ sweep (multi-sweep LexBFS) of each graph of the dense N=16384 pair "
                                    "(subtree-intersection chordal graph, density %.3f, + %d cycle-closing edges); "
                                    "previous sweep = the plain LexBFS order" % (g.density(), info["r"]),
                        "n": g.n, "words_per_row": g.words, "graphs_per_step": 2}
    if name == "sweep1m":
        g, h, info = gg.sparse_csr_pair()
        return [g, h], {"workload": "one LexBFS+ sweep (multi-sweep LexBFS) of each graph of the CSR N=2^20 pair "
                                    "(reversed-PEO chordal graph + %d cycle-closing edges); previous sweep = the "
                                    "plain LexBFS order" % info["r"],
                        "n": g.n, "graphs_per_step": 2, "edges": [g.num_edges(), h.num_edges()]}
    if name == "small1k":
        g, h, info = gg.small_dense_pair()
        return [g, h], {"workload": "dense N=1000 subtree-intersection chordal graph (500-node tree) + copy with a "
                                    "planted induced C_%d" % info["k"],
                        "n": g.n, "words_per_row": g.words, "graphs_per_step": 2,
                        "edges": [g.num_edges(), h.num_edges()], "bytes_per_graph": g.nbytes}
    if name in ("sparse1m", "sparse64k"):
        g, h, info = gg.sparse_csr_pair() if name == "sparse1m" else gg.sparse_csr_pair(n=1 << 16)
        return [g, h], {"workload": "CSR N=%s reversed-PEO chordal graph (cliques of size U{1..20}, shuffled ids) "
                                    "+ copy with %d cycle-closing edges" % ("2^20" if name == "sparse1m" else "65536", info["r"]),
                        "n": g.n, "graphs_per_step": 2, "edges": [g.num_edges(), h.num_edges()],
                        "bytes_per_graph": g.nbytes}
    if name == "batch4096":
        graphs = gg.batch_dense(4096)
        return graphs, {"workload": "4096 dense graphs, N log-uniform in [16, 2048] (sum N = %d); even: subtree "
                                    "model, odd: + planted induced C_k" % sum(g.n for g in graphs),
                        "graphs_per_step": len(graphs), "bytes": sum(g.nbytes for g in graphs)}
    if name == "serve":
        pool = gg.serve_pool()
        graphs = [g for g, _ in pool]
        return graphs, {"workload": "serving: Poisson stream of 100000 queries over a pool of %d graphs, N "
                                    "log-uniform [64, 65536], density U[0.01, 0.2], dense < 8192 <= CSR, half "
                                    "with a planted C_k" % len(graphs),
                        "pool": len(graphs), "pool_n": [g.n for g in graphs],
                        "pool_bytes": sum(g.nbytes for g in graphs)}
    raise SystemExit(f"unknown workload {name}")


# DRAM bytes (read + write) per launch of the dominant kernel come from the
# kept ncu summary of that kernel (the "dram_bytes_per_launch" line), which
# also records the SHA-256 of the kernel's sources at capture time
# ("source_sha256"); once the sources differ, the figure belongs to another
# kernel and the roofline's traffic is null.
TRAFFIC_SUMMARIES = {
    "dense16k": ("profiles/lexbfs_dense_n16384_pair.txt",
                 ["paper_1508_06329_gb300/csrc/lexbfs_dense.cuh", "paper_1508_06329_gb300/csrc/lexbfs_dense.cu",
                  "paper_1508_06329_gb300/csrc/common.cuh"]),
}


def sources_sha256(paths, root: str = ROOT) -> str:
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(root, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def ncu_traffic(key: str, root: str = ROOT):
    """(bytes per launch or None, note) from the kept summary of `key`'s kernel."""
    if key not in TRAFFIC_SUMMARIES:
        return None, "no ncu summary for this workload"
    summary, srcs = TRAFFIC_SUMMARIES[key]
    fields = {}
    try:
        with open(os.path.join(root, summary)) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
    except OSError:
        return None, f"{summary} missing"
    if "dram_bytes_per_launch" not in fields or "source_sha256" not in fields:
        return None, f"{summary} has no dram_bytes_per_launch / source_sha256 line"
    if fields["source_sha256"] != sources_sha256(srcs, root):
        return None, f"kernel sources changed since the capture in {summary}"
    return float(fields["dram_bytes_per_launch"]), f"ncu capture in {summary}"


def algorithmic_bytes(g) -> int:
    """Bytes the method must read per graph: each pivot row once (LexBFS) plus
    row v and row p(v) per vertex (the check); CSR: row_ptr + col per pass,
    plus the position gathers of the check."""
    if hasattr(g, "rows"):
        return 3 * g.n * g.words * 4
    return 3 * (8 * g.n + 4 * g.nnz) + 4 * g.nnz


def oracle_test_fn(order: str):
    """The oracle's whole test for the chosen ordering (LexBFS or MCS)."""
    import oracle
    return oracle.chordal_test_mcs if order == "mcs" else oracle.chordal_test


def oracle_rate(graphs, budget_s: float = 12.0, cap: int | None = None, order: str = "lexbfs"):
    """Oracle tests/s on a bounded sample of the workload (single thread)."""
    test = oracle_test_fn(order)
    t0 = time.perf_counter()
    done = 0
    while True:
        for g in graphs:
            test(g)
            done += 1
            el = time.perf_counter() - t0
            if el >= budget_s or (cap and done >= cap):
                return done / el, done, el


def _oracle_chunk(args):
    import graphgen as gg
    import oracle
    (seed, lo, hi) = args
    graphs = gg.batch_dense(4096, seed=seed)[lo:hi]
    t0 = time.perf_counter()
    for g in graphs:
        oracle.chordal_test(g)
    return hi - lo, time.perf_counter() - t0


def oracle_rate_all_cores(total: int = 4096):
    """Batch workload on all host cores: a spawn pool, each worker tests a
    slice of the same seeded graphs (generation excluded from its timing)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import graphgen as gg
    cores = os.cpu_count() or 1
    step = (total + cores - 1) // cores
    jobs = [(gg.SEED_BASE + 4, i, min(total, i + step)) for i in range(0, total, step)]
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        t0 = time.perf_counter()
        res = list(ex.map(_oracle_chunk, jobs))
        wall = time.perf_counter() - t0
    done = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return done / slowest, cores, done, wall


# --------------------------------------------------------------------------- reference arm

def check_order_option(args):
    if args.order == "mcs" and args.workload not in ("dense16k", "small1k", "paper7"):
        raise SystemExit("--order mcs applies to the dense workloads dense16k, small1k and paper7")


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    graphs, cfg = make_workload(args.workload)
    check_order_option(args)
    if args.order == "mcs":
        cfg = dict(cfg, order="MCS (Section 5.1)")
    test = oracle_test_fn(args.order)
    if args.workload in ("sweep16k", "sweep1m"):
        import oracle
        prev = {id(g): oracle.lexbfs(g) for g in graphs}

        def test(g):
            return oracle.lexbfs_plus(g, prev[id(g)])
    sample = graphs if args.workload != "batch4096" else graphs[:512]
    for _ in range(args.warmup):
        test(sample[0])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for g in sample:
            test(g)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = len(sample) * args.steps / total
    unit = UNIT if not args.workload.startswith("sweep") else "sweeps/s"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32 bitsets / int32",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT if not args.workload.startswith("sweep") else "sweeps/s",
                             "cores": 1,
                             "kind": "oracle",
                             "sample": f"{args.steps} steps x {len(sample)} graphs of the workload, "
                                       "single-threaded C oracle"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- GPU arm

def run_serve(args):
    """Continuous batching under a Poisson stream (rank 0 only; other ranks exit)."""
    # many concurrent slot streams: give them separate hardware work queues
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import numpy as np
    import torch
    rank, world, local = dist_info()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1508_06329_gb300 import build as cbuild
    cbuild.build()
    from paper_1508_06329_gb300 import binding as B
    graphs, cfg = make_workload("serve")
    pool = []
    for g in graphs:
        if hasattr(g, "rows"):
            pool.append(("dense", torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).to(dev), g.n))
        else:
            pool.append(("csr", (torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev)), g.n))
    ctx = B.Context(local)

    def submit(q, k):
        kind, data, n = pool[k]
        return q.submit_dense(data, n) if kind == "dense" else q.submit_csr(data[0], data[1], n)

    # results alone (the single-query path through the same queue, one at a time)
    q = B.Queue(ctx, mem_budget_bytes=64 << 30, max_inflight=64, max_batch=256, max_batch_large=2)
    alone, alone_s = [], []
    for k in range(len(pool)):
        t0 = time.perf_counter()
        t = submit(q, k)
        q.drain()
        alone.append(q.poll(t)[1])
        alone_s.append(time.perf_counter() - t0)
    nq = 100000
    rs = np.random.Generator(np.random.PCG64(1508063295))
    picks = rs.integers(0, len(pool), size=nq)
    # saturation: a burst of 4,000 queries submitted at once
    burst = picks[:4000]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tk = [submit(q, int(k)) for k in burst]
    q.drain()
    sat = len(burst) / (time.perf_counter() - t0)
    for t in tk:
        q.poll(t)
    lam = 0.8 * sat
    gaps = rs.exponential(1.0 / lam, size=nq)
    arrivals = np.cumsum(gaps)
    sampler = ClockSampler(local)
    sampler.start()
    tickets = []
    t0 = time.perf_counter()
    for k, at in zip(picks, arrivals):
        while True:
            now = time.perf_counter() - t0
            if now >= at:
                break
            if at - now > 0.002:
                time.sleep(0.001)
        while True:
            try:
                tickets.append(submit(q, int(k)))
                break
            except B.ChordalError as e:
                if e.status != B.CG_EAGAIN:
                    raise
                time.sleep(0.0002)
    q.drain()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    lat, bad = [], 0
    for k, t in zip(picks, tickets):
        st, res, l = q.poll(t)
        if st != B.CG_OK or res != alone[int(k)]:
            bad += 1
        lat.append(l)
    info = q.stats()
    q.close()
    lat = np.array(lat)
    # the one-at-a-time path: the plain single-graph call per query, waited for,
    # on one stream (no queue), each pool graph timed and weighted by the picks
    ctx1 = B.Context(local)
    r1 = torch.empty(4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    single_s = []
    for kind, data, n in pool:
        def once():
            if kind == "dense":
                B.chordal_test_dense(ctx1, data, n, r1, None, stream)
            else:
                B.chordal_test_csr(ctx1, data[0], data[1], n, r1, None, stream)
            torch.cuda.synchronize()
        once()   # workspace sized
        reps = 3 if n <= 8192 else 1
        t1 = time.perf_counter()
        for _ in range(reps):
            once()
        single_s.append((time.perf_counter() - t1) / reps)
    ctx1.close()
    mean_single = float(np.mean([single_s[int(k)] for k in picks]))
    one_at_a_time = 1.0 / mean_single
    value = nq / wall
    # latency per admission lane (n <= 4096 and larger) and the graphs behind the p99 tail
    pool_n = np.array([n for _, _, n in pool])
    qn = pool_n[picks]
    lanes = {}
    for name, sel in (("n<=4096", qn <= 4096), ("n>4096", qn > 4096)):
        if sel.any():
            lanes[name] = {"queries": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50) * 1e3),
                           "p99_ms": float(np.percentile(lat[sel], 99) * 1e3)}
    p99 = np.percentile(lat, 99)
    tail = lat >= p99
    tail_n = qn[tail]
    tail_info = {"queries": int(tail.sum()), "n_min": int(tail_n.min()), "n_median": int(np.median(tail_n)),
                 "share_n_over_16384": float((tail_n > 16384).mean()),
                 "single_call_ms_of_tail_graphs_median": float(np.median([single_s[int(k)] for k in picks[tail]]) * 1e3)}
    # the oracle on all host cores over a bounded sample of the same stream
    cpu_rate, cpu_cores, cpu_done, cpu_wall = serve_oracle_all_cores(picks, len(pool))
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 bitsets / int32 (exact)", "data": "synthetic",
            "config": dict(cfg, arrival_rate_qps=lam, saturation_qps=sat, queries=nq,
                           parallelism="single GPU (queue: 64 slots, 64 GiB pool, large-graph batches of 2, 32 hardware queues)"),
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                           "mean": float(lat.mean() * 1e3), "max": float(lat.max() * 1e3), "by_lane": lanes,
                           "p99_tail": tail_info},
            "results_differing_from_alone": bad, "queue": info,
            "one_at_a_time": {"value": one_at_a_time, "unit": "queries/s",
                              "sample": "each pool graph through the plain single-graph call (cg_chordal_test_dense "
                                        "or _csr) and a stream synchronise, weighted by the stream's picks",
                              "served_over_one_at_a_time": value / one_at_a_time},
            "cpu_baseline": {"value": cpu_rate, "unit": "queries/s", "cores": cpu_cores, "kind": "oracle",
                             "sample": f"{cpu_done} queries of the stream's picks on {cpu_cores} processes, "
                                       f"{cpu_wall:.1f} s wall"},
            "clocks": clocks}
    print(json.dumps(line))
    ctx.close()
    return 0 if bad == 0 else 1


def _serve_oracle_chunk(args):
    import graphgen as gg
    import oracle
    idx, ks, budget_s = args
    graphs = {i: gg.serve_pool_item(i)[0] for i in idx}   # this worker's share of the pool (untimed)
    t0 = time.perf_counter()
    done = 0
    for k in ks:
        oracle.chordal_test(graphs[k])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0


def serve_oracle_all_cores(picks, pool_size: int, budget_s: float = 12.0):
    """Oracle queries/s for the serving stream on all host cores: worker w
    builds the pool graphs with index = w (mod cores) and tests the stream's
    picks of those graphs, in stream order, for at most budget_s (pool
    generation excluded from its timing); rate = queries / the slowest
    worker's time."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = []
    for w in range(cores):
        idx = [i for i in range(pool_size) if i % cores == w]
        ks = [int(k) for k in picks if int(k) % cores == w]
        if ks:
            jobs.append((idx, ks, budget_s))
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_serve_oracle_chunk, jobs))
    wall = time.perf_counter() - t0
    done = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return done / slowest, len(jobs), done, wall


def paper7_graphs():
    """Seeded stand-ins for the paper's test classes (Section 7): it gives no
    generator parameters, so dense random uses p = 0.5 and the chordal class
    spans tree sizes 50..10000 (dense to sparse)."""
    import graphgen as gg
    out = []
    for n in range(1000, 12000, 1000):
        out.append(("clique", f"N={n}", gg.clique(n)))
    for t in range(5):
        out.append(("dense random", f"test{t + 1}", gg.random_dense(10000, 0.5, gg.SEED_BASE + 70 + t)))
    for t in range(5):
        out.append(("sparse random M=20N", f"test{t + 1}", gg.random_dense(10000, 40.0 / 9999, gg.SEED_BASE + 80 + t)))
    for t in range(7):
        out.append(("tree", f"test{t + 1}", gg.random_tree(10000, gg.SEED_BASE + 90 + t)))
    for t, tn in enumerate((50, 100, 200, 500, 1000, 2000, 5000, 10000)):
        out.append(("chordal (subtree model)", f"test{t + 1} tree={tn}", gg.subtree_dense(10000, tn, gg.SEED_BASE + 100 + t)))
    return out


def run_paper7(args):
    """GPU vs oracle on the paper's families, one graph at a time (rank 0)."""
    import numpy as np
    import torch
    import oracle
    rank, world, local = dist_info()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1508_06329_gb300 import build as cbuild
    cbuild.build()
    from paper_1508_06329_gb300 import binding as B
    ctx = B.Context(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    table, gpu_total_ms, tests = [], 0.0, 0
    for fam, label, g in paper7_graphs():
        rows = torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).to(dev)
        res = torch.empty(4, dtype=torch.int32, device=dev)
        B.chordal_test_dense(ctx, rows, g.n, res)
        torch.cuda.synchronize()
        ms = []
        for _ in range(3):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            B.chordal_test_dense(ctx, rows, g.n, res)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        hr = torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).pin_memory()
        t0 = time.perf_counter()
        got = B.chordal_test_dense_host(ctx, hr, g.n)
        e2e_ms = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        want = oracle.chordal_test(g)
        oracle_ms = (time.perf_counter() - t0) * 1e3
        if got != want.witness or tuple(res.cpu().tolist()) != want.witness:
            raise SystemExit(f"parity failure on {fam} {label}")
        # the same test with the MCS order (Section 5.1, Theorem 5.2)
        B.chordal_test_mcs_dense(ctx, rows, g.n, res)
        torch.cuda.synchronize()
        mms = []
        for _ in range(3):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            B.chordal_test_mcs_dense(ctx, rows, g.n, res)
            b.record()
            torch.cuda.synchronize()
            mms.append(a.elapsed_time(b))
        t0 = time.perf_counter()
        want_mcs = oracle.chordal_test_mcs(g)
        oracle_mcs_ms = (time.perf_counter() - t0) * 1e3
        if tuple(res.cpu().tolist()) != want_mcs.witness or want_mcs.chordal != want.chordal:
            raise SystemExit(f"MCS parity failure on {fam} {label}")
        gpu_ms = statistics.median(ms)
        gpu_total_ms += gpu_ms
        tests += 1
        table.append({"family": fam, "case": label, "n": g.n, "m": g.num_edges(), "chordal": want.chordal,
                      "gpu_ms": round(gpu_ms, 3), "gpu_e2e_ms": round(e2e_ms, 3), "oracle_ms": round(oracle_ms, 3),
                      "oracle_over_gpu": round(oracle_ms / gpu_ms, 2),
                      "gpu_mcs_ms": round(statistics.median(mms), 3), "oracle_mcs_ms": round(oracle_mcs_ms, 3)})
    line = {"metric": METRIC, "value": tests / (gpu_total_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 3,
            "warmup": 1, "ms_per_step": gpu_total_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 bitsets / int32 (exact)", "data": "synthetic",
            "config": {"workload": "paper Section 7 families, one graph at a time (median of 3, L2 flushed)",
                       "gpu_ms": "LexBFS + check kernels, CUDA events",
                       "gpu_e2e_ms": "host rows -> device -> result (cg_chordal_test_dense_host)",
                       "oracle_ms": "single-threaded C oracle, input already in memory",
                       "gpu_mcs_ms / oracle_mcs_ms": "the same test with the MCS order (Section 5.1)"},
            "table": table}
    print(json.dumps(line))
    ctx.close()
    return 0


def run_sweep(args):
    """One LexBFS+ sweep per graph of the N=16,384 dense pair (sweep16k) or the
    N=2^20 CSR pair (sweep1m), two streams, each fed the plain LexBFS order as
    the previous sweep; the sweep relabels the graph on the GPU and runs the
    LexBFS on the copy."""
    import numpy as np
    import torch
    import oracle
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1508_06329_gb300 import build as cbuild
    cbuild.build()
    from paper_1508_06329_gb300 import binding as B
    graphs, cfg = make_workload(args.workload)
    dense = hasattr(graphs[0], "rows")
    prev_h = [oracle.lexbfs(g) for g in graphs]
    want = [oracle.lexbfs_plus(g, p) for g, p in zip(graphs, prev_h)]
    if dense:
        rows = [torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).to(dev) for g in graphs]
    else:
        rows = [(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev)) for g in graphs]
    prev = [torch.from_numpy(p.astype(np.int32)).to(dev) for p in prev_h]
    orders = [torch.empty(g.n, dtype=torch.int32, device=dev) for g in graphs]
    stream = torch.cuda.current_stream()
    side = [torch.cuda.Stream(dev) for _ in graphs]
    ctxs = [B.Context(local) for _ in graphs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(plain=False):
        ev = torch.cuda.Event()
        ev.record(stream)
        for k, g in enumerate(graphs):
            side[k].wait_event(ev)
            if dense and plain:
                B.lexbfs_order_dense(ctxs[k], rows[k], g.n, orders[k], None, side[k])
            elif dense:
                B.lexbfs_plus_dense(ctxs[k], rows[k], g.n, prev[k], orders[k], None, stream=side[k])
            elif plain:
                B.lexbfs_order_csr(ctxs[k], rows[k][0], rows[k][1], g.n, orders[k], None, side[k])
            else:
                B.lexbfs_plus_csr(ctxs[k], rows[k][0], rows[k][1], g.n, prev[k], orders[k], None, stream=side[k])
        for s_ in side:
            stream.wait_stream(s_)

    def timed(plain, steps):
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(plain)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return ms

    warm = max(args.warmup, 3) if dense else 1
    timed(False, warm)
    for k in range(len(graphs)):
        if not np.array_equal(orders[k].cpu().numpy(), want[k]):
            raise SystemExit("parity failure in the sweep bench")
    for c in ctxs:
        c.read_profile()
        c.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = timed(False, args.steps)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    prof = {}
    for c in ctxs:
        for k, v in c.read_profile().items():
            prof[k] = prof.get(k, 0) + v
        c.profile(False)
    total_ms, value = aggregate_over_ranks(sum(ms), len(graphs) * args.steps, dev)
    plain_ms = timed(True, max(3, min(args.steps, 5)) if dense else 1)
    # end to end: previous order and rows from pinned host memory, the new order back
    if dense:
        host_rows = [[torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).pin_memory()] for g in graphs]
        dev_rows = [[r] for r in rows]
    else:
        host_rows = [[torch.from_numpy(g.row_ptr).pin_memory(), torch.from_numpy(g.col).pin_memory()] for g in graphs]
        dev_rows = [list(r) for r in rows]
    host_prev = [p.cpu().pin_memory() for p in prev]
    host_out = [torch.empty(g.n, dtype=torch.int32).pin_memory() for g in graphs]
    e2e_steps = max(1, min(args.steps, 5)) if dense else 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for hrs, drs, hp, dp in zip(host_rows, dev_rows, host_prev, prev):
            for hr, dr in zip(hrs, drs):
                dr.copy_(hr, non_blocking=True)
            dp.copy_(hp, non_blocking=True)
        step()
        for ho, o in zip(host_out, orders):
            ho.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if rank == 0 and any(not np.array_equal(ho.numpy(), w) for ho, w in zip(host_out, want)):
        raise SystemExit("parity failure on the host-buffer path")
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    n = graphs[0].n
    sweep_ms = prof["lexbfs_ms"] / max(1, prof["lexbfs_launches"])
    lex_bytes = n * graphs[0].words * 4 if dense else 8 * n + 4 * graphs[0].nnz
    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps, "warmup": warm,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 bitsets / int32 (exact)", "data": "synthetic",
        "config": dict(cfg, l2="flushed before each timed step (256 MiB write)",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": {"bound": "hbm", "kernel": ("lexbfs_dense_kernel" if dense else "lexbfs_csr_kernel")
                     + " on the relabelled copy", "achieved":
                     lex_bytes / (sweep_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": lex_bytes / (sweep_ms * 1e-3) / 1e9 / hbm, "traffic": None,
                     "peak_kind": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": lex_bytes},
        "phases": {"sweep_ms_per_graph": sweep_ms, "step_ms_p50": statistics.median(ms),
                   "plain_lexbfs_step_ms_p50": statistics.median(plain_ms),
                   "relabel_overhead_ms_per_step": statistics.median(ms) - statistics.median(plain_ms)},
        "e2e": {"value": len(graphs) * e2e_steps * world / e2e_s, "unit": "sweeps/s",
                "h2d_bytes_per_step": sum(g.nbytes + 4 * g.n for g in graphs),
                "d2h_bytes_per_step": sum(4 * g.n for g in graphs),
                "path": "pinned host graph + previous order -> device, cg_lexbfs_sweep_%s (LexBFS+), order -> host"
                        % ("dense" if dense else "csr")},
        "gpu_launches": int(prof["kernel_launches"]),
        "clocks": clocks,
    }
    if rank == 0 and world == 1:
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < (10.0 if dense else 4.0):
            for g, p in zip(graphs, prev_h):
                oracle.lexbfs_plus(g, p)
                done += 1
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / el, "unit": "sweeps/s", "cores": 1, "kind": "oracle",
                                "sample": f"{done} LexBFS+ sweeps of the two graphs, {el:.1f} s, single-threaded C"}
    if rank == 0:
        print(json.dumps(line))
    for c in ctxs:
        c.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1508_06329_gb300 import build as cbuild
    cbuild.build()
    from paper_1508_06329_gb300 import binding as B
    import oracle

    wl = args.workload
    check_order_option(args)
    mcs = args.order == "mcs"
    graphs, cfg = make_workload(wl)
    if mcs:
        cfg = dict(cfg, order="MCS (Section 5.1), one graph per stream")
    ngraph = len(graphs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ctx = B.Context(local)
    dense = hasattr(graphs[0], "rows")
    res = torch.empty((ngraph, 4), dtype=torch.int32, device=dev)
    plan = None
    if dense:
        # all graphs' rows in one pinned host buffer and one device buffer (each graph
        # 16-byte aligned), so the end-to-end path copies them with one transfer
        offs, tot = [], 0
        for g in graphs:
            offs.append(tot)
            tot += (g.rows.size + 3) & ~3
        flat = np.zeros(max(tot, 4), dtype=np.int32)
        for g, o in zip(graphs, offs):
            flat[o:o + g.rows.size] = np.ascontiguousarray(g.rows).view(np.int32).ravel()
        host_flat = torch.from_numpy(flat).pin_memory()
        dev_flat = host_flat.to(dev)
        rows = [dev_flat[o:o + g.rows.size].view(g.n, g.words) for g, o in zip(graphs, offs)]
        batch = [(r, g.n) for r, g in zip(rows, graphs)]
        orders = torch.empty(max(1, sum(g.n for g in graphs)), dtype=torch.int32, device=dev)
        if mcs:
            side = [torch.cuda.Stream(dev) for _ in graphs]
            side_ctx = [ctx] + [B.Context(local) for _ in graphs[1:]]

            def step():
                ev = torch.cuda.Event()
                ev.record(stream)
                for k, (r, g) in enumerate(zip(rows, graphs)):
                    side[k].wait_event(ev)
                    B.chordal_test_mcs_dense(side_ctx[k], r, g.n, res[k], None, side[k])
                for s in side:
                    stream.wait_stream(s)
        elif wl == "batch4096":
            B.batch_autotune(ctx, batch)
            plan = B.BatchPlan(ctx, batch, res, orders)

            def step():
                plan.run(stream)
        else:
            def step():
                B.chordal_test_batch(ctx, batch, res, orders, None, stream)
    else:
        csr = [(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev)) for g in graphs]
        side = [torch.cuda.Stream(dev) for _ in graphs]
        # overlapping calls need their own workspaces: one context per stream
        side_ctx = [ctx] + [B.Context(local) for _ in graphs[1:]]

        def step():
            ev = torch.cuda.Event()
            ev.record(stream)
            for k, (g, (rp, col)) in enumerate(zip(graphs, csr)):
                side[k].wait_event(ev)
                B.chordal_test_csr(side_ctx[k], rp, col, g.n, res[k], None, side[k])
            for s in side:
                stream.wait_stream(s)

    warm = max(args.warmup, 3) if wl != "sparse1m" else max(1, min(args.warmup, 1))
    for _ in range(warm):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    # parity guard on the timed configuration
    got = [tuple(r) for r in res.cpu().tolist()]
    if rank == 0:
        want = [oracle_test_fn(args.order)(g).witness for g in graphs]
        if got != want:
            raise SystemExit(f"parity failure in bench: {got[:4]} vs {want[:4]}")

    all_ctx = side_ctx if (not dense or mcs) else [ctx]
    for c in all_ctx:
        c.read_profile()
        c.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    prof = {}
    for c in all_ctx:
        for k, v in c.read_profile().items():
            prof[k] = prof.get(k, 0) + v
        c.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, value = aggregate_over_ranks(sum(step_ms), ngraph * args.steps, dev)

    # ---- end to end through the public API with host buffers
    e2e_steps = max(1, min(args.steps, 5 if wl != "sparse1m" else 1))
    if mcs:
        host_res = torch.empty((ngraph, 4), dtype=torch.int32).pin_memory()
        h2d = 4 * host_flat.numel()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            dev_flat.copy_(host_flat, non_blocking=True)
            step()
            host_res.copy_(res, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        out = [tuple(r) for r in host_res.tolist()]
        e2e_path = "pinned host rows -> device (one copy), cg_chordal_test_mcs_dense per graph, results -> pinned host"
    elif dense:
        # the library's host-buffer entry: pinned host rows in, the copies, the
        # batched run and the results' copy back all inside cg_chordal_test_batch_host
        # the descriptors of the host buffers are built once (B.HostBatch); every timed
        # call still copies all rows in and the results out
        host_graphs = B.HostBatch([(host_flat[o:o + g.rows.size].view(g.n, g.words), g.n)
                                   for g, o in zip(graphs, offs)])
        host_res = torch.empty((ngraph, 4), dtype=torch.int32).pin_memory()
        h2d = sum(4 * g.rows.size for g in graphs)
        B.chordal_test_batch_host(ctx, host_graphs, host_res)   # sizes the workspace (untimed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            B.chordal_test_batch_host(ctx, host_graphs, host_res)
        e2e_s = time.perf_counter() - t0
        out = [tuple(r) for r in host_res.tolist()]
        e2e_path = "cg_chordal_test_batch_host: pinned host rows -> device -> results back to pinned host"
    else:
        host_csr = [(torch.from_numpy(g.row_ptr).pin_memory(), torch.from_numpy(g.col).pin_memory()) for g in graphs]
        host_res = torch.empty((ngraph, 4), dtype=torch.int32).pin_memory()
        h2d = sum(g.nbytes for g in graphs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for (hrp, hcol), (drp, dcol) in zip(host_csr, csr):
                drp.copy_(hrp, non_blocking=True)
                dcol.copy_(hcol, non_blocking=True)
            step()
            host_res.copy_(res, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        out = [tuple(r) for r in host_res.tolist()]
        e2e_path = "pinned host CSR -> device, cg_chordal_test_csr per graph on two streams, results -> pinned host"
    if rank == 0 and out != want:
        raise SystemExit("parity failure on the host-buffer path")
    e2e_value = ngraph * e2e_steps * world / e2e_s

    # ---- roofline of the dominant kernel
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    alg = sum(algorithmic_bytes(g) for g in graphs)
    phases = {"step_ms_p50": statistics.median(step_ms),
              "step_ms_p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]}
    if wl in ("dense16k", "sparse1m", "sparse64k") or mcs:
        lex_ms = prof["lexbfs_ms"] / max(1, prof["lexbfs_launches"])
        chk_ms = prof["check_ms"] / max(1, prof["check_launches"])
        if mcs:
            lex_bytes = graphs[0].n * graphs[0].words * 4           # each pivot row once, one graph per launch
            chk_bytes = 2 * graphs[0].n * graphs[0].words * 4
            per_launch = 1
        elif wl == "dense16k":
            lex_bytes = sum(g.n * g.words * 4 for g in graphs)      # each pivot row once, both graphs per launch
            chk_bytes = sum(2 * g.n * g.words * 4 for g in graphs)
            per_launch = 1
        else:
            lex_bytes = 8 * graphs[0].n + 4 * graphs[0].nnz           # one graph per launch
            chk_bytes = 2 * (8 * graphs[0].n + 4 * graphs[0].nnz) + 4 * graphs[0].nnz
            per_launch = 1
        kernel = "lexbfs_dense_kernel" if wl == "dense16k" else "lexbfs_csr_kernel"
        if mcs:
            kernel = "mcs_dense_kernel"
        lex_gbs = lex_bytes / (lex_ms * 1e-3) / 1e9
        chk_gbs = chk_bytes / (chk_ms * 1e-3) / 1e9
        dom_share = prof["lexbfs_ms"] / max(1e-9, prof["lexbfs_ms"] + prof["check_ms"])
        traffic, traffic_note = ncu_traffic(wl + ("/mcs" if mcs else ""))
        roof = {"bound": "hbm", "kernel": f"{kernel} ({100 * dom_share:.1f}% of GPU time)", "achieved": lex_gbs,
                "peak": hbm, "unit": "GB/s", "frac": lex_gbs / hbm, "traffic": traffic, "traffic_source": traffic_note,
                "peak_kind": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": lex_bytes * per_launch}
        phases.update({"lexbfs_ms_per_launch": lex_ms, "check_ms_per_launch": chk_ms,
                       "lexbfs_ns_per_step": lex_ms * 1e6 / graphs[0].n, "check_gbs": chk_gbs,
                       "check_frac_of_hbm": chk_gbs / hbm})
        phases["floor"] = step_floor(all_ctx[0], stream, phases["lexbfs_ns_per_step"])
    else:
        run_ms = prof["batch_ms"] / max(1, prof["batch_calls"])
        gbs = alg / (run_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "chordal_dense_fused_kernel (size buckets, concurrent)", "achieved": gbs,
                "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                "peak_kind": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": alg}
        phases.update({"batch_ms_per_call": run_ms, "fused_ms_sum": prof["fused_ms"] / max(1, args.steps),
                       "lexbfs_ms_sum": prof["lexbfs_ms"] / max(1, args.steps)})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": warm,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 bitsets / int32 (exact)", "data": "synthetic",
        "config": dict(cfg, l2="flushed before each timed step (256 MiB write)",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "adjacency_gbs": alg * args.steps * world / (total_ms * 1e-3) / 1e9,
        "roofline": roof, "phases": phases,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16 * ngraph,
                "path": e2e_path},
        "gpu_launches": int(prof["kernel_launches"]),
        "clocks": clocks,
    }
    if wl == "batch4096" and rank == 0 and world == 1:
        # the plain one-graph-at-a-time GPU path on the same graphs (bounded sample)
        r1 = torch.empty(4, dtype=torch.int32, device=dev)
        sample = batch[:512]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t, n in sample:
            B.chordal_test_dense(ctx, t, n, r1, None, stream)
        torch.cuda.synchronize()
        one = len(sample) / (time.perf_counter() - t0)
        line["one_at_a_time"] = {"value": one, "unit": UNIT, "sample": "first 512 graphs, cg_chordal_test_dense "
                                                                       "looped on one stream",
                                 "batched_over_one_at_a_time": value / one}
    if rank == 0 and world == 1:
        if wl == "batch4096":
            rate, cores, done, wall = oracle_rate_all_cores()
            r1c, d1, e1 = oracle_rate(graphs, budget_s=10.0)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"all {done} graphs on {cores} processes (slowest worker's time); "
                                              f"single thread: {r1c:.0f} tests/s on {d1} graphs"}
        else:
            rate, done, el = oracle_rate(graphs, budget_s=12.0 if wl != "sparse1m" else 4.0, order=args.order)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"{done} tests of the workload's graphs, {el:.1f} s, "
                                              "single-threaded C" + (" (MCS + check)" if mcs else "")}
    if rank == 0:
        print(json.dumps(line))
    if plan is not None:
        plan.close()
    for c in all_ctx:
        c.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def step_floor(ctx, stream, ns_per_step: float) -> dict:
    """Latency floors of one sequential step, measured after the timed region:
    a pair of CTA barriers (1,024 threads), one dependent load over a 32 MiB
    chain (L2-resident, like the 32 MiB dense graph) and over a 1 GiB chain
    (mostly DRAM)."""
    from paper_1508_06329_gb300 import binding as B
    try:
        l2 = B.step_floor(ctx, threads=1024, iters=16384, chain_bytes=32 << 20, loads=100000, stream=stream)
        dram = B.step_floor(ctx, threads=1024, iters=1024, chain_bytes=1 << 30, loads=20000, stream=stream)
    except B.ChordalError as e:   # an auxiliary figure: the benchmark line is printed without it
        return {"error": str(e)}
    floor = l2["barrier_pair_ns"] + l2["load_ns"]
    return {"barrier_pair_ns": l2["barrier_pair_ns"], "l2_load_ns": l2["load_ns"], "dram_load_ns": dram["load_ns"],
            "barrier_pair_plus_l2_load_ns": floor, "step_over_that": ns_per_step / floor,
            "step_in_l2_loads": ns_per_step / l2["load_ns"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--order", default="lexbfs", choices=["lexbfs", "mcs"],
                    help="vertex ordering of the test (dense workloads): LexBFS (default) or MCS")
    ap.add_argument("--workload", default="dense16k",
                    choices=["dense16k", "small1k", "sparse1m", "sparse64k", "batch4096", "serve", "paper7",
                             "sweep16k", "sweep1m"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "paper7":
        return run_paper7(args)
    if args.workload in ("sweep16k", "sweep1m"):
        return run_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
