"""Benchmark of the parallel chordality test on GB300.

Workload (default): the dense N=16,384 pair — a subtree-intersection chordal
graph at edge density ~0.1 (32 MiB of bit-packed rows) and its copy with
1-10 cycle-closing extra edges.  One step = the whole test (LexBFS + the
perfect-elimination check + witness) on both graphs, issued as one batched
call; the metric is chordality tests per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Timing: inputs resident in HBM; before every timed step a 256 MiB buffer is
written to flush L2 (the inputs are smaller than L2); each step is bracketed
by CUDA events on the launching stream.  `e2e` repeats the metric through the
C ABI's host-buffer entry (pinned host rows in, result out, copies inside the
timed region).  `cpu_baseline` times the CPU oracle on a bounded sample.
With N > 1 (torchrun) every rank runs its own replica of the workload (the
test of one graph does not shard); value = tests on all ranks / max time.
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


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload():
    import graphgen as gg
    g, h, info = gg.large_dense_pair()
    return [g, h], {"workload": "dense N=16384 subtree-intersection chordal graph (density %.3f, tree %d nodes) "
                                "+ copy with %d cycle-closing edges" % (g.density(), info["tree_nodes"], info["r"]),
                    "n": g.n, "words_per_row": g.words, "graphs_per_step": 2,
                    "edges": [g.num_edges(), h.num_edges()], "bytes_per_graph": g.nbytes}


def cpu_oracle_rate(graphs, budget_s: float = 12.0):
    """Oracle tests/s on a bounded sample: repeat the pair until ~budget_s."""
    import oracle
    t0 = time.perf_counter()
    done = 0
    while True:
        for g in graphs:
            oracle.chordal_test(g)
            done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or done >= 64:
            break
    return done / el, done, el


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    graphs, cfg = workload()
    import oracle
    for _ in range(args.warmup):
        oracle.chordal_test(graphs[0])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for g in graphs:
            oracle.chordal_test(g)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = len(graphs) * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32 bitsets / int32",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps x {len(graphs)} graphs, single-threaded C oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
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

    graphs, cfg = workload()
    n, words = graphs[0].n, graphs[0].words
    rows = [torch.from_numpy(g.rows.view(np.int32)).to(dev) for g in graphs]
    res = torch.empty((len(graphs), 4), dtype=torch.int32, device=dev)
    orders = torch.empty(sum(g.n for g in graphs), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ctx = B.Context(local)
    batch = [(r, g.n) for r, g in zip(rows, graphs)]

    def step():
        B.chordal_test_batch(ctx, batch, res, orders, None, stream)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    # parity guard on the timed configuration
    import oracle
    want = [oracle.chordal_test(g).witness for g in graphs] if rank == 0 else None
    got = [tuple(r) for r in res.cpu().tolist()]
    if rank == 0 and got != want:
        raise SystemExit(f"parity failure in bench: {got} vs {want}")

    ctx.read_profile()
    ctx.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = []
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
    prof = ctx.read_profile()
    ctx.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    tests = len(graphs) * args.steps * world
    value = tests / (total_ms / 1e3)

    # end to end through the host-buffer entry (pinned rows in, result out)
    host_rows = [torch.from_numpy(g.rows.view(np.int32)).pin_memory() for g in graphs]
    for g, hr in zip(graphs, host_rows):
        B.chordal_test_dense_host(ctx, hr, g.n, None, stream)
    e2e_steps = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        out = [B.chordal_test_dense_host(ctx, hr, g.n, None, stream) for g, hr in zip(graphs, host_rows)]
    e2e_s = time.perf_counter() - t0
    if rank == 0 and out != want:
        raise SystemExit("parity failure on the host-buffer path")
    e2e_value = len(graphs) * e2e_steps * world / e2e_s

    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    lex_ms = prof["lexbfs_ms"] / max(1, prof["lexbfs_launches"])
    total_ms_dev = prof["batch_ms"] if prof["batch_calls"] else total_ms
    chk_ms = prof["check_ms"] / max(1, prof["check_launches"])
    row_bytes = n * words * 4
    lex_bytes = len(graphs) * row_bytes            # each pivot row read once
    chk_bytes = len(graphs) * 2 * row_bytes        # own row + parent row per vertex
    lex_gbs = lex_bytes / (lex_ms * 1e-3) / 1e9
    chk_gbs = chk_bytes / (chk_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 bitsets / int32 (exact)", "data": "synthetic",
        "config": dict(cfg, l2="flushed before each timed step (256 MiB write)",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": {"bound": "hbm", "kernel": "lexbfs_dense_kernel (dominant: %.1f%% of step)" %
                     (100.0 * prof["lexbfs_ms"] / max(1e-9, total_ms_dev)),
                     "achieved": lex_gbs, "peak": hbm, "unit": "GB/s", "frac": lex_gbs / hbm,
                     "traffic": None, "peak_kind": f"{peak_kind} hbm_gbs"},
        "phases": {"lexbfs_ms_per_launch": lex_ms, "check_ms_per_launch": chk_ms,
                   "lexbfs_ns_per_step": lex_ms * 1e6 / n, "check_gbs": chk_gbs, "check_frac_of_hbm": chk_gbs / hbm,
                   "step_ms_p50": statistics.median(step_ms),
                   "step_ms_p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": len(graphs) * row_bytes,
                "d2h_bytes_per_step": len(graphs) * 16, "path": "cg_chordal_test_dense_host per graph"},
        "gpu_launches": int(prof["kernel_launches"]),
        "clocks": clocks,
    }
    if rank == 0 and world == 1:
        rate, done, el = cpu_oracle_rate(graphs)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{done} tests of the same two graphs, {el:.1f} s, single-threaded C"}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
