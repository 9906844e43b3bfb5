#!/usr/bin/env python3
"""Benchmark: large-batch SSSP source queries on R-MAT scale 24 (the largest workload).

One step = one fg_sssp_batch of B seeded sources (default 256) drawn in turn
from the workload's 16,384 sources, on the undirected R-MAT scale-24 graph
(16,777,216 vertices, 520,758,442 arcs, weights in [1, 255]), followed by
fg_sync. Prints ONE JSON line (rank 0) with the device-timed rate, the
end-to-end rate through the C ABI with host buffers, the roofline of the
engine kernel, the CPU oracle as a reported baseline, and extra keys: the
road-like grid workload (1,024 BFS + SSSP sources), the PPR error against the
FP64 oracle on R-MAT scale 22, and the plain per-query GPU form.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fg|reference] [--nq B]
    python bench.py --grid          # the grid BFS + SSSP workload as the main line

Under torchrun (N > 1) every rank runs its own batches of the 16,384 sources
on its own GPU (weak scaling; queries are independent, so nothing is
exchanged), and the slowest rank's time sets the whole-job rate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

WORKLOAD = "rmat24_sssp"
GRAPH_DESC = ("undirected R-MAT scale 24 (16,777,216 vertices, edge factor 16, a/b/c/d = 0.57/0.19/0.19/0.05, "
              "self-loops and duplicates removed, 520,758,442 arcs), int32 weights uniform in [1,255]")
WORKLOAD_SOURCES = 16384
NQ_STEP = 256
METRIC = "source-queries/s"
UNIT = "queries/s"

# the road-like grid workload (an extra key of the main line, or the main line with --grid)
GRID_WORKLOAD = "grid1024_bfs_sssp"
GRID_DESC = ("road-like 2D grid 1024x1024 (1,048,576 vertices), 4-neighbour edges with 5% dropped, "
             "1% diagonal shortcuts, int32 weights uniform in [100,10000]")
GRID_NQ = 1024
SOURCE_SETS = 3
# Scheduling for the grid workload (per-query priority windows, i.e. Delta-stepping
# across partitions, with yield heuristic 2's delta for SSSP): what fg_tune_opts
# picks on the workload's 1,024 sources (window 10x and delta 5x the mean weight)
TUNED_BFS = {"sched": 1, "sched_window": 24}
TUNED_SSSP = {"sched": 1, "sched_window": 50490, "delta": 25245}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fg", choices=["fg", "reference"])
    ap.add_argument("--nq", type=int, default=0,
                    help="sources per step (default: 256 on R-MAT s24, 1,024 on the grid)")
    ap.add_argument("--grid", action="store_true", help="the grid BFS + SSSP workload as the main line")
    ap.add_argument("--graph-scale", type=int, default=0,
                    help="plumbing tests only: a smaller R-MAT of the same recipe instead of scale 24")
    ap.add_argument("--no-ppr-check", action="store_true", help="skip the R-MAT s22 PPR error record")
    ap.add_argument("--no-grid-extra", action="store_true", help="skip the grid workload extra key")
    ap.add_argument("--no-group-sweep", action="store_true",
                    help="--ablation: skip the group-size sweep on the R-MAT s24 bench workload")
    ap.add_argument("--no-serving-extra", action="store_true", help="skip the R-MAT s25 serving extra key")
    ap.add_argument("--cpu-sources", type=int, default=0,
                    help="sources of the CPU oracle sample (default: one per host core, at most 16)")
    ap.add_argument("--opts-bfs", default="", help="JSON overrides of fg_opts for the BFS batches")
    ap.add_argument("--opts-sssp", default="", help="JSON overrides of fg_opts for the SSSP batches")
    ap.add_argument("--partition-vertices", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="use the hand-swept schedules instead of fg_tune_opts")
    ap.add_argument("--no-extras", action="store_true", help="skip the cpu/plain/e2e legs (profiling runs)")
    ap.add_argument("--cpu-sample", type=int, default=512)
    ap.add_argument("--plain-sample", type=int, default=8)
    ap.add_argument("--serve-lambda", type=float, default=1000.0, help="arrival rate of the serving leg (q/s)")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests in the serving leg")
    ap.add_argument("--serving", action="store_true",
                    help="only the serving measurement on the directed R-MAT scale-25 graph (mixed SSSP/BFS/PPR)")
    ap.add_argument("--serve-lambdas", default="2000,5000,10000,20000,50000")
    ap.add_argument("--configs", action="store_true",
                    help="only the other workloads (R-MAT s14 plain, s22 PPR, s24 SSSP) with their baselines")
    ap.add_argument("--ncp", action="store_true",
                    help="only the NCP application: PPRs from 0.01%% of R-MAT s22, sweep cuts, profile")
    ap.add_argument("--ncp-scale", type=int, default=22, help="R-MAT scale of the NCP run (22 = the PPR workload)")
    ap.add_argument("--ncp-top", type=int, default=4096, help="vertices per sweep")
    ap.add_argument("--bc", action="store_true",
                    help="only the BC application: 100 sampled sources, SSSP on the grid and BFS on R-MAT s22")
    ap.add_argument("--bc-sources", type=int, default=100, help="sampled sources per BC run")
    ap.add_argument("--bc-graphs", default="grid,rmat", help="BC runs to do: grid (SSSP), rmat (BFS)")
    ap.add_argument("--walks", action="store_true",
                    help="only the query types without a batch engine form: random walks and DFS")
    ap.add_argument("--local-ppr", action="store_true",
                    help="only local PPR: sparse per-query state against the dense batch on R-MAT s22, eps 1e-4")
    ap.add_argument("--ll", action="store_true",
                    help="only the LL application: 1,024 SSSPs on the grid, labels, 2^20 distance queries")
    ap.add_argument("--ll-pairs", type=int, default=1 << 20, help="pairs per query batch of the LL run")
    ap.add_argument("--ll-landmarks", type=int, default=GRID_NQ, help="landmarks of the LL run (1,024 = the workload)")
    ap.add_argument("--ablation", action="store_true",
                    help="only the scheduling / yield / partition-size ablation on the bench workload")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_rate(queries_per_rank: int, world_size: int, slowest_ms: float) -> float:
    """Whole-job source queries per second: every rank's queries over the slowest rank's time."""
    return queries_per_rank * world_size / (slowest_ms / 1000.0)


def source_sets(g, rank, nq=GRID_NQ):
    """The grid workload's seeded source sets of one rank (each rank draws its own)."""
    from paper_2103_14915_gb300 import inputs
    return [inputs.workload_sources(GRID_WORKLOAD, g, GRID_NQ, set_index=100 * rank + i)[:nq]
            for i in range(SOURCE_SETS)]


def step_sources(all_srcs: np.ndarray, rank: int, world: int, step: int, nb: int) -> np.ndarray:
    """Sources of one step of one rank: block (step * world + rank) of nb consecutive
    sources of the workload's list, wrapping around. Within a step the ranks take
    different blocks, so the job covers the list once before any source repeats."""
    blocks = max(1, len(all_srcs) // nb)
    b = (step * world + rank) % blocks
    return np.ascontiguousarray(all_srcs[b * nb:(b + 1) * nb])


def csr_sha256_check(g, name):
    """(computed, recorded, match) for a workload graph, against tests/golden/csr_sha256.txt."""
    h = hashlib.sha256()
    h.update(g.row_ptr.astype("<i8", copy=False).tobytes())
    h.update(g.col.astype("<i4", copy=False).tobytes())
    if g.w is not None:
        h.update(g.w.astype("<i4", copy=False).tobytes())
    got = h.hexdigest()
    rec = None
    f = ROOT / "tests" / "golden" / "csr_sha256.txt"
    if f.exists():
        for ln in f.read_text().splitlines():
            if ln.startswith(name + " "):
                rec = dict(x.split("=", 1) for x in ln.split()[1:]).get("csr")
    return got, rec, got == rec


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def engine_traffic():
    """DRAM bytes per engine launch from the committed ncu summary, if it matches the kernel source."""
    src = (ROOT / "paper_2103_14915_gb300" / "csrc" / "fg_engine.cu").read_bytes()
    sha = hashlib.sha256(src).hexdigest()[:16]
    f = ROOT / "profiles" / "engine_grid1024_traffic.txt"
    if not f.exists():
        return None
    kv = {}
    for ln in f.read_text().splitlines():
        if ":" in ln:
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("engine_source_sha256_16") != sha:
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def serve_stream(fg, h, g, lam, n_req, seed, lanes, max_batch, kinds=(0, 1, 2), alpha=0.15, eps=1e-6,
                 opts=None, continuous=0, slots=128):
    """Poisson stream of single-source requests through the serving loop (fg_server_*).

    Request i arrives at a seeded exponential-gap time, with a kind drawn
    uniformly from `kinds` and a seeded-uniform source. The host loop submits
    requests as their arrival time passes, polls, and releases completed ones.
    Latency = completion seen by fg_server_poll - scheduled arrival (host
    monotonic clock, the server's steady clock). continuous=1 runs SSSP and
    BFS with slot-level batching (`slots` query lanes per kind).
    """
    from paper_2103_14915_gb300 import inputs
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / lam, n_req)
    arrive = np.cumsum(gaps)
    kind = rng.choice(np.asarray(kinds, dtype=np.int32), n_req)
    pool = inputs.sources_uniform(g, min(n_req, 65536), seed + 1)
    src = pool[rng.integers(0, len(pool), n_req)]
    so = fg.fg_default_server_opts(lanes=lanes, max_batch=max_batch, alpha=alpha, eps=eps,
                                   continuous=continuous, slots=slots)
    for k, o in (opts or {}).items():
        for key, v in o.items():
            setattr(so.opts[k], key, v)
    st, srv = fg.fg_server_create(h, so)
    fg.check(st)
    arr_ns = {}
    lat = {0: [], 1: [], 2: []}
    batch = []
    i = done = 0
    t0 = time.monotonic_ns()
    first_ok = True
    try:
        while done < n_req:
            now = (time.monotonic_ns() - t0) / 1e9
            while i < n_req and arrive[i] <= now:
                st, rid = fg.fg_server_submit(srv, int(kind[i]), int(src[i]))
                fg.check(st)
                arr_ns[rid] = t0 + int(arrive[i] * 1e9)
                i += 1
            st, ids = fg.fg_server_poll(srv, 4096)
            if st != fg.FG_OK:
                first_ok = False
            for rid in ids:
                st, info = fg.fg_server_info(srv, rid)
                fg.check(st)
                if info.status != fg.FG_OK:
                    first_ok = False
                lat[info.kind].append((info.done_ns - arr_ns.pop(rid)) / 1e6)
                batch.append(info.batch_size)
                fg.check(fg.fg_server_release(srv, rid))
                done += 1
            if not ids and i < n_req:
                time.sleep(max(0.0, min(2e-4, arrive[i] - (time.monotonic_ns() - t0) / 1e9)))
        t_end = time.monotonic_ns()
    finally:
        fg.fg_server_destroy(srv)
    allv = np.concatenate([np.asarray(v) for v in lat.values() if v])
    names = {0: "sssp", 1: "bfs", 2: "ppr"}
    return {"lambda_qps": lam, "requests": n_req, "ok": first_ok,
            "throughput_qps": n_req / ((t_end - t0) / 1e9 - 0.0),
            "p50_ms": float(np.percentile(allv, 50)), "p99_ms": float(np.percentile(allv, 99)),
            "per_kind_p99_ms": {names[k]: float(np.percentile(v, 99)) for k, v in lat.items() if v},
            "mean_batch": float(np.mean(batch)), "lanes": lanes, "max_batch": max_batch,
            "mode": "slots" if continuous else "batches", **({"slots": slots} if continuous else {})}


def bench_graph(args):
    """The bench graph: the R-MAT scale-24 workload, or (for plumbing tests only) a
    smaller R-MAT of the same recipe with --graph-scale."""
    from paper_2103_14915_gb300 import inputs
    if args.graph_scale:
        g = inputs.rmat(args.graph_scale, 16, seed=args.graph_scale, weights=(1, 255))
        return g, f"rmat{args.graph_scale}_sssp", f"undirected R-MAT scale {args.graph_scale} (test size)"
    return inputs.workload_graph(WORKLOAD), WORKLOAD, GRAPH_DESC


def run_reference(args):
    """The oracle (CPU: binary-heap Dijkstra, OpenMP over queries, one query per host
    core at a time: the paper's t = 1 scheme) on a bounded sample of the bench
    workload: one source per step, the K timed steps' sources in one oracle call
    (so they run side by side on the host cores), after the W warm-up steps' sources
    in another."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2103_14915_gb300 import inputs
    if args.grid:
        return run_reference_grid(args)
    g, name, desc = bench_graph(args)
    all_srcs = inputs.workload_sources(WORKLOAD, g) if not args.graph_scale else inputs.sources_uniform(
        g, int((np.diff(g.row_ptr) > 0).sum()) // 2, 1)
    cores = oracle.num_threads()
    warm = step_sources(all_srcs, 0, 1, 0, max(1, args.warmup))
    timed = step_sources(all_srcs, 0, 1, 1, max(1, args.steps)) if args.steps > 0 else warm[:0]
    if args.warmup > 0:
        oracle.sssp(g, warm[:args.warmup])
    t0 = time.perf_counter()
    oracle.sssp(g, timed)
    dt = time.perf_counter() - t0
    value = len(timed) / dt
    sample = (f"one source per step ({len(timed)} timed, {args.warmup} warm-up) from the {len(all_srcs):,}-source "
              f"list, run side by side on {cores} host cores")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": name, "graph": desc, "queries_per_step": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference_grid(args):
    """The oracle on a bounded sample of the grid workload (32 sources per step, BFS + SSSP)."""
    import oracle
    from paper_2103_14915_gb300 import inputs
    g = inputs.workload_graph(GRID_WORKLOAD)
    sets = source_sets(g, 0)
    per_step = 32
    cores = oracle.num_threads()
    for i in range(args.warmup):
        s = sets[i % SOURCE_SETS][:per_step]
        oracle.bfs(g, s)
        oracle.sssp(g, s)
    t0 = time.perf_counter()
    for i in range(args.steps):
        s = sets[i % SOURCE_SETS][:per_step]
        oracle.bfs(g, s)
        oracle.sssp(g, s)
    dt = time.perf_counter() - t0
    value = 2 * per_step * args.steps / dt
    sample = f"{per_step} sources per step (BFS + SSSP each), {args.steps} steps"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": GRID_WORKLOAD, "graph": GRID_DESC, "queries_per_step": 2 * per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_serving(args):
    """Serving sweep on the directed R-MAT scale-25 graph: one JSON line with p50/p99 per arrival rate."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2103_14915_gb300 import fg, inputs
    name = "rmat25_serving"
    g = inputs.workload_graph(name)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    runs = []
    try:
        # schedules for this graph from the autotuner on a 64-source sample
        sample = torch.from_numpy(inputs.sources_uniform(g, 64, 4242)).to("cuda:0")
        opts = {}
        for kind in (fg.FG_QUERY_SSSP, fg.FG_QUERY_BFS):
            st, best, _ = fg.fg_tune_opts(h, kind, sample, 64)
            fg.check(st)
            opts[kind] = {k: int(getattr(best, k)) for k in ("group", "sched", "sched_window", "delta",
                                                             "threads_per_vertex")}
        for lam in [float(x) for x in args.serve_lambdas.split(",") if x]:
            runs.append(serve_stream(fg, h, g, lam, args.serve_requests, seed=int(lam), lanes=4, max_batch=256,
                                     kinds=(0, 1, 2), alpha=0.15, eps=1e-6, opts=opts))
            # slot-level batching of SSSP and BFS (group engine, 32 lanes per group)
            sopts = {k: dict(v, group=32) for k, v in opts.items()}
            runs.append(serve_stream(fg, h, g, lam, args.serve_requests, seed=int(lam), lanes=2, max_batch=256,
                                     kinds=(0, 1, 2), alpha=0.15, eps=1e-6, opts=sopts, continuous=1, slots=128))
    finally:
        fg.fg_graph_destroy(h)
    best = max(r["throughput_qps"] for r in runs)
    print(json.dumps({"metric": "serving p99 latency", "value": runs[0]["p99_ms"], "unit": "ms", "n_gpus": 1,
                      "higher_is_better": False, "data": "synthetic",
                      "config": {"workload": name, "graph": "directed R-MAT scale 25, edge factor 24, weights [1,255]",
                                 "mix": "1/3 SSSP, 1/3 BFS, 1/3 PPR(alpha=0.15, eps=1e-6)",
                                 "requests_per_rate": args.serve_requests},
                      "sustained_qps": best,
                      "sustained_qps_by_mode": {m: max(r["throughput_qps"] for r in runs if r["mode"] == m)
                                                for m in ("batches", "slots")},
                      "opts": {"sssp": opts[0], "bfs": opts[1]}, "runs": runs}), flush=True)


def run_ablation(args):
    """Scheduling / yield / partition-size ablation on the bench workload (GPU form of Tab. 4, Fig. 7, Fig. 11).

    One JSON line: for each configuration, the batch time of BFS and SSSP over
    the first source set and the engine counters (rounds, visits, arcs scanned,
    operations), all results checked against the first configuration's.
    """
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2103_14915_gb300 import fg, inputs
    g = inputs.workload_graph(GRID_WORKLOAD)
    nq = args.nq or GRID_NQ
    src = torch.from_numpy(source_sets(g, 0, nq)[0]).to(dev)
    mu_arcs = None
    rows = []

    def run(h, kind, opts):
        out = torch.empty((nq, g.n), dtype=torch.int32, device=dev)
        f = fg.fg_bfs_batch if kind == "bfs" else fg.fg_sssp_batch
        fg.check(f(h, src, nq, out, None, fg.fg_default_opts(**opts)))
        fg.check(fg.fg_sync())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fg.check(f(h, src, nq, out, None, fg.fg_default_opts(**opts)))
        b.record()
        fg.check(fg.fg_sync())
        torch.cuda.synchronize()
        st, stats = fg.fg_stats(h)
        d = stats.as_dict()
        return a.elapsed_time(b), d, out

    ref = {}
    for S, method in ((256, fg.FG_PART_GROW), (512, fg.FG_PART_GROW), (1024, fg.FG_PART_GROW),
                      (2048, fg.FG_PART_GROW), (1024, fg.FG_PART_RANGE)):
        st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0,
                                      fg.fg_default_graph_opts(partition_method=method, partition_vertices=S))
        fg.check(st)
        info = fg.fg_graph_info(h)[1]
        mu = g.m // max(1, info.num_partitions) // nq  # arcs per partition per query (yield heuristic 1 unit)
        mu_exact = g.m / max(1, info.num_partitions) / nq  # mu = |E_P| / |Q| (App. A)
        cfgs = [("fifo", {"group": 1}, {"group": 1}),
                ("priority-window (Shortest, Tab. 4A)", TUNED_BFS, TUNED_SSSP)]
        if S == 1024 and method == fg.FG_PART_GROW:
            # Tab. 4A: the four inter-partition schedulers (FIFO and Shortest above)
            cfgs += [("max-ops (Tab. 4A)", {"sched": fg.FG_SCHED_MAXOPS}, {"sched": fg.FG_SCHED_MAXOPS}),
                     ("random (Tab. 4A)", {"sched": fg.FG_SCHED_RANDOM}, {"sched": fg.FG_SCHED_RANDOM}),
                     ("priority-window/2", {"sched": 1, "sched_window": TUNED_BFS["sched_window"] // 2},
                      {"sched": 1, "sched_window": TUNED_SSSP["sched_window"] // 2}),
                     ("priority-window*2", {"sched": 1, "sched_window": TUNED_BFS["sched_window"] * 2},
                      {"sched": 1, "sched_window": TUNED_SSSP["sched_window"] * 2}),
                     ("delta-yield (heuristic 2)", {"delta": 8}, {"delta": 20000})]
            # Tab. 4B: edge budget (yield heuristic 1) of {0.25, 0.5, 1, 2, 4} mu on the priority window
            for f in (0.25, 0.5, 1.0, 2.0, 4.0):
                yb = max(1, int(round(f * mu_exact)))
                cfgs.append((f"edge-budget {f}*mu (Tab. 4B)", dict(TUNED_BFS, yield_edges=yb),
                             dict(TUNED_SSSP, yield_edges=yb)))
            cfgs += [("lane-per-vertex expansion", dict(TUNED_BFS, threads_per_vertex=1),
                      dict(TUNED_SSSP, threads_per_vertex=1)),
                     ("group engine G=16 (lanes = queries)", {"group": 16}, {"group": 16}),
                     ("group engine G=32 (lanes = queries)", {"group": 32}, {"group": 32}),
                     ("group engine G=64 (two queries per lane)", {"group": 64}, {"group": 64})]
        for name, ob, os_ in cfgs:
            row = {"S": S, "partition": "grow" if method == fg.FG_PART_GROW else "range", "config": name,
                   "cut_arcs": int(info.cut_arcs)}
            for kind, o in (("bfs", ob), ("sssp", os_)):
                ms, d, out = run(h, kind, o)
                key = kind
                if key not in ref:
                    ref[key] = out.cpu()
                exact = bool(torch.equal(out.cpu(), ref[key]))
                row[kind] = {"ms": round(ms, 2), "opts": o, "rounds": d["rounds"], "visits": d["visits"],
                             "arcs": d["edges"], "ops": d["ops"], "same_result": exact}
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
        fg.fg_graph_destroy(h)
    groups = [] if args.no_group_sweep else group_sweep_rmat24(fg, inputs, dev)
    print(json.dumps({"metric": "ablation", "workload": GRID_WORKLOAD, "sources": nq, "rows": rows,
                      "rmat24_groups": groups}), flush=True)


def group_sweep_rmat24(fg, inputs, dev):
    """Group sizes and the query order on the bench workload (R-MAT s24, the first
    256 sources of the bench line's list): one warm-up and one timed batch of SSSP
    and of BFS per setting, FIFO rounds, every result compared with the first
    setting's (rows identical whatever the group or order)."""
    import torch
    g = inputs.workload_graph(WORKLOAD)
    src = torch.from_numpy(step_sources(inputs.workload_sources(WORKLOAD, g), 0, 1, 0, NQ_STEP)).to(dev)
    nq = src.numel()
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    out = torch.empty((nq, g.n), dtype=torch.int32, device=dev)
    rows, ref = [], {}
    try:
        for group, order in ((16, 0), (32, 1), (32, 0), (64, 1), (64, 0)):
            row = {"group": group, "group_order": "as given" if order else "two-hop reach"}
            for kind, f in (("sssp", fg.fg_sssp_batch), ("bfs", fg.fg_bfs_batch)):
                o = fg.fg_default_opts(group=group, group_order=order)
                fg.check(f(h, src, nq, out, None, o))
                fg.check(fg.fg_sync())
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fg.check(f(h, src, nq, out, None, o))
                b.record()
                fg.check(fg.fg_sync())
                torch.cuda.synchronize()
                d = fg.fg_stats(h)[1].as_dict()
                if kind not in ref:
                    ref[kind] = out.cpu()
                ms = a.elapsed_time(b)
                row[kind] = {"ms": round(ms, 1), "qps": round(nq / (ms / 1000.0), 1), "rounds": d["rounds"],
                             "arcs_read": d["arcs_read"], "lane_relaxations": d["edges"],
                             "same_result": bool(torch.equal(out.cpu(), ref[kind]))}
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    finally:
        fg.fg_graph_destroy(h)
    return rows


def run_ncp(args):
    """NCP application (Sec. 1, 6.1): PPRs from 0.01% of the vertices of R-MAT s22
    (alpha 0.15, eps 1e-7), each swept to --ncp-top vertices, and the profile =
    best conductance per cluster size. One JSON line: PPR and sweep times, the
    sweep kernel's HBM roofline, sampled bit-exact parity, the CPU oracle's sweep."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2103_14915_gb300 import fg, inputs
    alpha, eps, top = 0.15, 1e-7, args.ncp_top
    if args.ncp_scale == 22:
        name, g = "rmat22_ncp", inputs.workload_graph("rmat22_ppr")
    else:
        name, g = f"rmat{args.ncp_scale}_ncp", inputs.rmat(args.ncp_scale, 16, seed=args.ncp_scale)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    seeds = inputs.ncp_seeds(g)
    nq = len(seeds)
    s_d = torch.from_numpy(seeds).to(dev)
    p = torch.empty((nq, g.n), dtype=torch.float32, device=dev)
    order = torch.empty((nq, top), dtype=torch.int32, device=dev)
    phi = torch.empty((nq, top), dtype=torch.float64, device=dev)
    count = torch.empty(nq, dtype=torch.int32, device=dev)
    ncp = torch.empty(top, dtype=torch.float64, device=dev)
    o = fg.fg_default_opts()
    stream = torch.cuda.current_stream().cuda_stream

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        fg.check(fg.fg_sync(stream))
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    ppr = lambda: fg.check(fg.fg_ppr_batch(h, s_d, nq, alpha, eps, p, None, None, stream, o))
    sweep = lambda: fg.check(fg.fg_ncp_sweep(h, p, nq, top, order, phi, count, ncp, False, stream))
    fg.check(fg.fg_ppr_batch(h, s_d[:64], 64, alpha, eps, p, None, None, stream, o))
    t_ppr = timed(ppr)
    for _ in range(2):
        sweep()  # the first call builds the degree table
    t_sweeps = sorted(timed(sweep) for _ in range(max(3, args.steps)))
    t_sweep = t_sweeps[len(t_sweeps) // 2]
    # algorithmic bytes: each PPR row once (4 B per vertex) plus the degree table once
    alg_bytes = 4 * g.n * nq + 4 * g.n
    achieved = alg_bytes / (t_sweep / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    prof = ncp.cpu().numpy()
    cnt = count.cpu().numpy()
    # parity and the CPU baseline on the oracle's own PPR rows (FP64 push rounded to FP32) for
    # a sample of the seeds: the GPU sweep of those rows against the oracle's sweep, bit for bit
    k_cpu = min(nq, 32)
    rows_o = np.stack([oracle.ppr_push(g, int(s), alpha, eps)[0] for s in seeds[:k_cpu]]).astype(np.float32)
    t0 = time.perf_counter()
    ro, rph, rc = oracle.ncp_sweep(g, rows_o, top)
    t_cpu = time.perf_counter() - t0
    po = torch.from_numpy(rows_o).to(dev)
    fg.check(fg.fg_ncp_sweep(h, po, k_cpu, top, order[:k_cpu], phi[:k_cpu], count[:k_cpu], None, False, stream))
    fg.check(fg.fg_sync(stream))
    exact = bool(np.array_equal(order[:k_cpu].cpu().numpy(), ro) and np.array_equal(count[:k_cpu].cpu().numpy(), rc)
                 and np.array_equal(phi[:k_cpu].cpu().numpy(), rph, equal_nan=True))
    finite = np.isfinite(prof)
    kbest = int(np.argmin(np.where(finite, prof, np.inf)))
    points = {str(k): float(prof[k - 1]) for k in (1, 10, 100, 1000, top) if k <= top and finite[k - 1]}
    res = {"metric": "NCP application", "workload": name, "n": g.n, "m": g.m, "seeds": nq,
           "seed_fraction": 1e-4, "alpha": alpha, "eps": eps, "top": top, "data": "synthetic",
           "ppr_ms": t_ppr, "sweep_ms": t_sweep, "ncp_total_ms": t_ppr + t_sweep,
           "ppr_per_s": nq / (t_ppr / 1e3), "sweeps_per_s": nq / (t_sweep / 1e3),
           "sweep_roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                              "frac": achieved / peak, "peak_kind": peak_kind,
                              "alg_bytes_per_launch": alg_bytes},
           "exact_sampled": exact, "parity_rows": f"oracle FP64 push rows of the first {k_cpu} seeds",
           "cpu_oracle_sweeps_per_s": k_cpu / t_cpu, "cpu_sample": k_cpu, "cpu_cores": oracle.num_threads(),
           "count_min": int(cnt.min()), "count_median": int(np.median(cnt)),
           "profile": {"best_phi": float(prof[kbest]), "best_size": kbest + 1, "points": points}}
    fg.fg_graph_destroy(h)
    print(json.dumps(res), flush=True)


def run_bc(args):
    """BC application (Sec. 1, 6.1): 100 random sources; one SSSP per source on the
    weighted grid workload, one BFS per source on the R-MAT s22 graph; then the
    Brandes dependency accumulation on the GPU. One JSON line per run with the
    batch and BC times, bit-exact parity of every vertex's centrality against the
    oracle chain (its own Dijkstra / BFS, path counts and dependencies), and the
    oracle's rate on the host cores."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2103_14915_gb300 import fg, inputs
    stream = torch.cuda.current_stream().cuda_stream
    bc_runs = {"grid": ("grid1024_bfs_sssp", True), "rmat": ("rmat22_ppr", False)}
    for name, weighted in [bc_runs[k] for k in args.bc_graphs.split(",")]:
        g = inputs.workload_graph(name)
        method = fg.FG_PART_GROW if weighted else fg.FG_PART_AUTO
        st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts(
            partition_method=method))
        fg.check(st)
        srcs = inputs.sources_uniform(g, args.bc_sources, seed=74)
        nq = len(srcs)
        s_d = torch.from_numpy(srcs).to(dev)
        dist = torch.empty((nq, g.n), dtype=torch.int32, device=dev)
        bc = torch.empty(g.n, dtype=torch.float64, device=dev)
        kind = fg.FG_QUERY_SSSP if weighted else fg.FG_QUERY_BFS
        st, opts, _ = fg.fg_tune_opts(h, kind, s_d, nq, stream)
        fg.check(st)
        batch = fg.fg_sssp_batch if weighted else fg.fg_bfs_batch

        def timed(fn):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b), out

        def run_bc_kernel():
            st, info = fg.fg_bc_accumulate(h, s_d, nq, dist, weighted, bc, False, stream)
            fg.check(st)
            return info

        fg.check(batch(h, s_d, nq, dist, stream, opts))
        fg.check(fg.fg_sync(stream))
        run_bc_kernel()  # scratch allocation and grid sizing happen here
        t_batch = sorted(timed(lambda: fg.check(batch(h, s_d, nq, dist, stream, opts)))[0]
                         for _ in range(3))[1]
        fg.check(fg.fg_sync(stream))
        runs = [timed(run_bc_kernel) for _ in range(max(3, args.steps))]
        t_bc = sorted(r[0] for r in runs)[len(runs) // 2]
        info = runs[-1][1]
        got = bc.cpu().numpy()
        t0 = time.perf_counter()
        ref, smax, exact = oracle.bc(g, srcs, weighted)
        t_cpu = time.perf_counter() - t0
        same = bool(np.array_equal(got, ref)) if exact else bool(np.allclose(got, ref, rtol=1e-9))
        top = np.argsort(-ref)[:5]
        res = {"metric": "BC application", "workload": f"{name.split('_')[0]}_bc_{'sssp' if weighted else 'bfs'}",
               "n": g.n, "m": g.m, "sources": nq, "weighted": weighted, "data": "synthetic",
               "batch_ms": t_batch, "bc_ms": t_bc, "bc_total_ms": t_batch + t_bc,
               "sources_per_s": nq / ((t_batch + t_bc) / 1e3), "waves": info.waves,
               "sigma_max": info.sigma_max, "inexact": info.inexact,
               "batch_opts": {k2: int(getattr(opts, k2)) for k2 in ("sched", "sched_window", "delta")},
               "parity": "bit-exact, every vertex" if exact else "rtol 1e-9 (a path count passed 2^53)",
               "matches_oracle": same, "cpu_oracle_sources_per_s": nq / t_cpu, "cpu_cores": oracle.num_threads(),
               "top_vertices": [int(v) for v in top]}
        fg.fg_graph_destroy(h)
        del dist
        print(json.dumps(res), flush=True)


def run_walks(args):
    """Random-walk and DFS queries (query types of the framework, Sec. 3). Walks:
    2^20 walks of 80 steps from uniform sources on R-MAT s22. DFS: 1,024 queries
    on R-MAT s18. One JSON line each with the GPU time, bit-exact parity of every
    output against the oracle, and the oracle's rate on the host cores."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2103_14915_gb300 import fg, inputs
    stream = torch.cuda.current_stream().cuda_stream
    peak, peak_kind = measured_peaks()

    def timed(fn, reps):
        out = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return sorted(out)[len(out) // 2]

    # random walks
    g = inputs.workload_graph("rmat22_ppr")
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    nw, L, seed = 1 << 20, 80, 2021
    srcs = np.random.default_rng(5).integers(0, g.n, size=nw).astype(np.int32)
    s_d = torch.from_numpy(srcs).to(dev)
    paths = torch.empty((nw, L + 1), dtype=torch.int32, device=dev)
    walk = lambda: fg.check(fg.fg_rw_batch(h, s_d, nw, L, seed, paths, stream))
    walk()
    t = timed(walk, max(5, args.steps))
    got = paths.cpu().numpy()
    t0 = time.perf_counter()
    ref = oracle.rw(g, srcs, L, seed)
    t_cpu = time.perf_counter() - t0
    steps = nw * L
    alg = nw * (L + 1) * 4 + steps * 12  # the paths written + per step the arc range and the chosen arc
    print(json.dumps({
        "metric": "random walks", "workload": "rmat22_rw", "n": g.n, "m": g.m, "walks": nw, "length": L,
        "data": "synthetic", "ms": t, "steps_per_s": steps / (t / 1e3), "walks_per_s": nw / (t / 1e3),
        "roofline": {"bound": "hbm (latency of dependent gathers)", "achieved": alg / (t / 1e3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": alg / (t / 1e3) / 1e9 / peak, "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg},
        "exact": bool(np.array_equal(got, ref)), "cpu_oracle_steps_per_s": steps / t_cpu,
        "cpu_cores": oracle.num_threads()}), flush=True)
    del paths
    fg.fg_graph_destroy(h)

    # DFS
    g = inputs.rmat(18, 16, seed=18)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    nq = 1024
    srcs = inputs.sources_uniform(g, nq, seed=6)
    s_d = torch.from_numpy(srcs).to(dev)
    disc = torch.empty((nq, g.n), dtype=torch.int32, device=dev)
    dfs = lambda: fg.check(fg.fg_dfs_batch(h, s_d, nq, disc, stream))
    dfs()
    t = timed(dfs, 3)
    got = disc.cpu().numpy().view(np.uint32)
    t0 = time.perf_counter()
    ref = oracle.dfs(g, srcs)
    t_cpu = time.perf_counter() - t0
    print(json.dumps({
        "metric": "DFS queries", "workload": "rmat18_dfs", "n": g.n, "m": g.m, "queries": nq, "data": "synthetic",
        "ms": t, "queries_per_s": nq / (t / 1e3), "exact": bool(np.array_equal(got, ref)),
        "cpu_oracle_queries_per_s": nq / t_cpu, "cpu_cores": oracle.num_threads(),
        "bound": "latency: one dependent step chain per query, one warp per query"}), flush=True)
    fg.fg_graph_destroy(h)


def run_local_ppr(args):
    """Local PPR on R-MAT s22 (the 4,096 log-degree seeds, alpha 0.15, eps 1e-4):
    sparse per-query state (fg_ppr_local_batch, tables of 2^17 slots) against the
    dense batch (fg_ppr_batch) at the same eps. One JSON line with both rates,
    the scratch each needs, the mass error, and sampled rows against the
    oracle's FP64 push at eps / 100 (bound eps * d + eps / 100 * d + 1e-6)."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2103_14915_gb300 import fg, inputs
    alpha, eps, cap = 0.15, 1e-4, 1 << 17
    g = inputs.workload_graph("rmat22_ppr")
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    srcs = inputs.workload_sources("rmat22_ppr", g)
    nq = len(srcs)
    s_d = torch.from_numpy(srcs).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    vert = torch.empty((nq, cap), dtype=torch.int32, device=dev)
    pl = torch.empty((nq, cap), dtype=torch.float32, device=dev)
    cnt = torch.empty(nq, dtype=torch.int32, device=dev)
    mass = torch.empty(nq, dtype=torch.float64, device=dev)

    def timed(fn, reps=3):
        out = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return sorted(out)[len(out) // 2]

    local = lambda: fg.check(fg.fg_ppr_local_batch(h, s_d, nq, alpha, eps, cap, vert, pl, cnt, mass, stream))
    local()
    t_local = timed(local)
    c = cnt.cpu().numpy()
    m_err = float((mass - 1.0).abs().max())
    rows = [0, nq // 2, nq - 1]
    deg = np.maximum(np.diff(g.row_ptr), 1).astype(np.float64)
    ok = True
    for q in rows:
        ref = oracle.ppr_push(g, int(srcs[q]), alpha, eps / 100)[0]
        got = np.zeros(g.n)
        k = int(c[q])
        if k >= 0:
            got[vert[q, :k].cpu().numpy()] = pl[q, :k].cpu().numpy()
            ok &= bool(np.all(np.abs(got - ref) <= eps * deg * 1.01 + 1e-6))
    del vert, pl
    # the dense batch at the same eps (the library splits the batch to fit HBM)
    pd = torch.empty((256, g.n), dtype=torch.float32, device=dev)
    dense = lambda: fg.check(fg.fg_ppr_batch(h, s_d[:256], 256, alpha, eps, pd, None, None, stream, None))
    dense()
    fg.check(fg.fg_sync(stream))
    t_dense = timed(dense)
    print(json.dumps({
        "metric": "local PPR", "workload": "rmat22_ppr_local", "n": g.n, "m": g.m, "seeds": nq, "alpha": alpha,
        "eps": eps, "data": "synthetic", "sparse_ms": t_local, "sparse_qps": nq / (t_local / 1e3),
        "sparse_scratch_bytes": 24 * nq * cap, "table_slots": cap, "tables_full": int((c < 0).sum()),
        "support_median": int(np.median(c[c >= 0])) if (c >= 0).any() else None,
        "mass_err_max": m_err, "bound_ok_sampled": ok,
        "dense_qps": 256 / (t_dense / 1e3), "dense_bytes_per_query": 12 * g.n,
        "dense_sample": 256}), flush=True)
    fg.fg_graph_destroy(h)


def run_ll(args):
    """LL application (Sec. 1, 6.1): 1,024 SSSPs from random landmarks on the grid
    workload, label construction (query-major rows to vertex-major labels) and a
    batch of distance queries answered from the labels. One JSON line: the three
    stages' times, the two label kernels' HBM rooflines, sampled bit-exact parity
    against the oracle chain (its own SSSP rows, labels, queries), the oracle's rates."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2103_14915_gb300 import fg, inputs
    g = inputs.workload_graph(GRID_WORKLOAD)
    lms = inputs.workload_sources(GRID_WORKLOAD, g, k=args.ll_landmarks)
    K, n, Q = len(lms), g.n, args.ll_pairs
    gopts = fg.fg_default_graph_opts(partition_method=fg.FG_PART_GROW, partition_vertices=args.partition_vertices)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, gopts)
    fg.check(st)
    stream = torch.cuda.current_stream().cuda_stream
    s_d = torch.from_numpy(lms).to(dev)
    dist = torch.empty((K, n), dtype=torch.int32, device=dev)
    lab = torch.empty((n, K), dtype=torch.int32, device=dev)
    rng = np.random.default_rng(2024)
    pairs = rng.integers(0, n, size=(Q, 2)).astype(np.int32)
    pr = torch.from_numpy(pairs).to(dev)
    est = torch.empty(Q, dtype=torch.int64, device=dev)
    if args.no_tune:
        opts = fg.fg_default_opts(**TUNED_SSSP)
    else:
        st, opts, _ = fg.fg_tune_opts(h, fg.FG_QUERY_SSSP, s_d, K, stream)
        fg.check(st)

    def timed(fn, reps):
        out = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            fg.check(fg.fg_sync(stream))
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return sorted(out)[len(out) // 2]

    sssp = lambda: fg.check(fg.fg_sssp_batch(h, s_d, K, dist, stream, opts))
    build = lambda: fg.check(fg.fg_ll_build_labels(dist, K, n, lab, stream))
    query = lambda: fg.check(fg.fg_ll_query(lab, n, K, pr, Q, est, stream))
    t_sssp = timed(sssp, 3)
    build()
    query()
    reps = max(5, args.steps)
    t_build = timed(build, reps)  # inputs (4 GB each way) far exceed L2: no flush needed
    t_query = timed(query, reps)
    peak, peak_kind = measured_peaks()
    b_build = 8 * K * n
    b_query = Q * (8 * K + 16)
    got = est.cpu().numpy().view(np.uint64)
    vs = rng.choice(n, size=2000, replace=False)
    lab_s = lab[torch.from_numpy(vs).to(dev)].cpu().numpy().view(np.uint32)
    del dist
    # the oracle chain: its own SSSP rows (all landmarks), labels, queries on a sample
    rows = oracle.sssp(g, lms)
    t0 = time.perf_counter()
    ref = oracle.ll_labels(rows)
    t_cpu_build = time.perf_counter() - t0
    del rows
    sample = rng.choice(Q, size=min(Q, 20000), replace=False)
    t0 = time.perf_counter()
    ref_est = oracle.ll_query(ref, pairs[sample])
    t_cpu_query = time.perf_counter() - t0
    exact = bool(np.array_equal(lab_s, ref[vs]) and np.array_equal(got[sample], ref_est))
    finite = got[got != np.iinfo(np.uint64).max]
    res = {"metric": "LL application", "workload": f"grid1024_ll_k{K}", "n": n, "m": g.m, "landmarks": K, "pairs": Q,
           "data": "synthetic", "sssp_ms": t_sssp, "labels_ms": t_build, "queries_ms": t_query,
           "ll_total_ms": t_sssp + t_build + t_query, "queries_per_s": Q / (t_query / 1e3),
           "labels_roofline": {"bound": "hbm", "achieved": b_build / (t_build / 1e3) / 1e9, "peak": peak,
                               "unit": "GB/s", "frac": b_build / (t_build / 1e3) / 1e9 / peak,
                               "peak_kind": peak_kind, "alg_bytes_per_launch": b_build},
           "query_roofline": {"bound": "hbm", "achieved": b_query / (t_query / 1e3) / 1e9, "peak": peak,
                              "unit": "GB/s", "frac": b_query / (t_query / 1e3) / 1e9 / peak,
                              "peak_kind": peak_kind, "alg_bytes_per_launch": b_query},
           "sssp_opts": {k2: int(getattr(opts, k2)) for k2 in ("sched", "sched_window", "delta")},
           "exact_sampled": exact, "parity_sample": "2,000 vertices' labels, 20,000 pairs",
           "cpu_oracle_labels_s": t_cpu_build, "cpu_oracle_queries_per_s": len(sample) / t_cpu_query,
           "cpu_cores": oracle.num_threads(),
           "estimate_mean": float(finite.mean()) if finite.size else None}
    fg.fg_graph_destroy(h)
    print(json.dumps(res), flush=True)


def run_configs(args):
    """The other workloads (R-MAT s14 plain SSSP, R-MAT s22 PPR, R-MAT s24 SSSP): buffered engine,
    plain per-query GPU form and the CPU oracle on the host cores, one JSON line."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2103_14915_gb300 import fg, inputs
    res = {"metric": "other workloads", "n_gpus": 1, "data": "synthetic", "cpu_cores": oracle.num_threads()}

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        fg.check(fg.fg_sync())
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def graph(name):
        g = inputs.workload_graph(name)
        st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
        fg.check(st)
        return g, h

    # cfg 1: R-MAT s14, 64 SSSP sources one at a time (plain), and as one buffered batch
    name = "rmat14_plain_sssp"
    g, h = graph(name)
    src = inputs.workload_sources(name, g)
    s_d = torch.from_numpy(src).to(dev)
    out = torch.empty((len(src), g.n), dtype=torch.int32, device=dev)
    fg.check(fg.fg_sssp_batch(h, s_d, len(src), out, None, fg.fg_default_opts(mode=fg.FG_MODE_PLAIN)))
    fg.check(fg.fg_sync())
    t_plain = timed(lambda: fg.check(fg.fg_sssp_batch(h, s_d, len(src), out, None,
                                                      fg.fg_default_opts(mode=fg.FG_MODE_PLAIN))))
    exact_plain = bool(np.array_equal(out.cpu().numpy().view(np.uint32), oracle.sssp(g, src)))
    st, ob, _ = fg.fg_tune_opts(h, fg.FG_QUERY_SSSP, s_d, len(src))
    fg.check(st)
    t_buf = timed(lambda: fg.check(fg.fg_sssp_batch(h, s_d, len(src), out, None, ob)))
    t0 = time.perf_counter()
    ref = oracle.sssp(g, src)
    t_cpu = time.perf_counter() - t0
    arcs = sum(oracle.reachable_arcs(g, r) for r in ref)
    res["rmat14_plain_sssp"] = {
        "plain_gpu_qps": len(src) / (t_plain / 1e3), "plain_gpu_ms_per_query": t_plain / len(src),
        "plain_gteps": arcs / (t_plain / 1e3) / 1e9, "buffered_qps": len(src) / (t_buf / 1e3),
        "cpu_oracle_qps": len(src) / t_cpu, "exact": exact_plain and bool(
            np.array_equal(out.cpu().numpy().view(np.uint32), ref)), "sources": len(src)}
    fg.fg_graph_destroy(h)

    # cfg 3: R-MAT s22 PPR, 4,096 log-degree seeds (sub-batched by the library)
    name = "rmat22_ppr"
    alpha, eps = 0.15, 1e-7
    g, h = graph(name)
    src = inputs.workload_sources(name, g)
    s_d = torch.from_numpy(src).to(dev)
    nq = len(src)
    p = torch.empty((nq, g.n), dtype=torch.float32, device=dev)
    mass = torch.empty(nq, dtype=torch.float64, device=dev)
    o = fg.fg_default_opts()
    fg.check(fg.fg_ppr_batch(h, s_d[:256], 256, alpha, eps, p, None, mass, None, o))
    fg.check(fg.fg_sync())
    t_buf = timed(lambda: fg.check(fg.fg_ppr_batch(h, s_d, nq, alpha, eps, p, None, mass, None, o)))
    _, stb = fg.fg_stats(h)
    mass_err = float((mass - 1.0).abs().max())
    k = 4
    po = fg.fg_default_opts(mode=fg.FG_MODE_PLAIN)
    t_plain = timed(lambda: fg.check(fg.fg_ppr_batch(h, s_d[:k], k, alpha, eps, p, None, None, None, po)))
    deg = np.maximum(np.diff(g.row_ptr), 1).astype(np.float64)
    sample = list(range(0, nq, nq // 16))[:16]
    t0 = time.perf_counter()
    pi = oracle.ppr_power(g, src[sample], alpha)
    t_cpu = time.perf_counter() - t0
    fg.check(fg.fg_ppr_batch(h, s_d, nq, alpha, eps, p, None, mass, None, o))
    fg.check(fg.fg_sync())
    ratio = max(float(np.max(np.abs(p[q].cpu().numpy().astype(np.float64) - pi[i]) / (eps * deg)))
                for i, q in enumerate(sample))
    res["rmat22_ppr"] = {"buffered_qps": nq / (t_buf / 1e3), "seeds": nq, "edge_pushes": int(stb.edges),
                         "plain_gpu_qps": k / (t_plain / 1e3), "plain_sample": k,
                         "cpu_oracle_qps": len(sample) / t_cpu, "cpu_sample": len(sample),
                         "max_err_over_eps_deg": ratio, "mass_err_max": mass_err}
    del p
    fg.fg_graph_destroy(h)

    # cfg 4: R-MAT s24 SSSP, batches of 256 of the 16,384 sources
    name = "rmat24_sssp"
    g, h = graph(name)
    src = inputs.workload_sources(name, g)
    nb = 256
    s_d = torch.from_numpy(src[:nb]).to(dev)
    out = torch.empty((nb, g.n), dtype=torch.int32, device=dev)
    st, ob, rep = fg.fg_tune_opts(h, fg.FG_QUERY_SSSP, s_d[:64], 64)
    fg.check(st)
    t_buf = timed(lambda: fg.check(fg.fg_sssp_batch(h, s_d, nb, out, None, ob)))
    _, stb = fg.fg_stats(h)
    k = 4
    t_plain = timed(lambda: fg.check(fg.fg_sssp_batch(h, s_d[:k], k, out, None,
                                                      fg.fg_default_opts(mode=fg.FG_MODE_PLAIN))))
    fg.check(fg.fg_sssp_batch(h, s_d, nb, out, None, ob))
    fg.check(fg.fg_sync())
    t0 = time.perf_counter()
    ref = oracle.sssp(g, src[:16])
    t_cpu = time.perf_counter() - t0
    got = out[:16].cpu().numpy().view(np.uint32)
    arcs = np.mean([oracle.reachable_arcs(g, r) for r in ref])
    qps = nb / (t_buf / 1e3)
    res["rmat24_sssp"] = {"buffered_qps": qps, "batch": nb, "gteps": qps * arcs / 1e9,
                          "arcs_scanned_over_dijkstra": float(stb.edges) / (arcs * nb),
                          "opts": {k2: int(getattr(ob, k2)) for k2 in ("sched", "sched_window", "delta")},
                          "plain_gpu_qps": k / (t_plain / 1e3), "plain_sample": k,
                          "cpu_oracle_qps": 16 / t_cpu, "cpu_sample": 16,
                          "exact_sampled": bool(np.array_equal(got, ref)),
                          "hbm_output_gbs": qps * 4 * g.n / 1e9}
    fg.fg_graph_destroy(h)
    print(json.dumps(res), flush=True)


def code_sha256_16(path) -> str:
    """SHA-256 prefix of a C++/CUDA source with its // comments and blank lines
    removed, so that a comment edit does not count as a change of the kernel."""
    import re
    lines = []
    for ln in path.read_text().splitlines():
        ln = re.sub(r"//.*$", "", ln).rstrip()
        if ln.strip():
            lines.append(ln)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def kernel_traffic(profile: str, source: str, sources: int, group: int):
    """DRAM bytes per launch from a committed ncu summary, while the kernel source it
    was taken from is unchanged apart from comments and the launch is the captured
    one (sources per launch, group size); else None."""
    sha = code_sha256_16(ROOT / "paper_2103_14915_gb300" / "csrc" / source)
    f = ROOT / "profiles" / profile
    if not f.exists():
        return None
    kv = {}
    for ln in f.read_text().splitlines():
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != sha:
        return None
    if kv.get("capture_sources") != str(sources) or kv.get("capture_group") != str(group):
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def ppr_error_record(fg, inputs, oracle, dev, k=8):
    """PPR forward push on R-MAT s22 (alpha 0.15, eps 1e-7), all 4,096 log-degree seeds, against
    the FP64 power iteration (to 1e-12) on k seeds spread over the log2-degree buckets, the
    top (hub) bucket included: max / mean / p99 over vertices of |p - pi| / (eps * d)."""
    import torch
    alpha, eps = 0.15, 1e-7
    g = inputs.workload_graph("rmat22_ppr")
    srcs = inputs.workload_sources("rmat22_ppr", g)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        nq = len(srcs)
        s_d = torch.from_numpy(srcs).to(dev)
        p = torch.empty((nq, g.n), dtype=torch.float32, device=dev)
        mass = torch.empty(nq, dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        fg.check(fg.fg_ppr_batch(h, s_d, nq, alpha, eps, p, None, mass, None, fg.fg_default_opts()))
        fg.check(fg.fg_sync())
        t_gpu = time.perf_counter() - t0
        deg = np.diff(g.row_ptr).astype(np.float64)
        order = np.argsort(deg[srcs], kind="stable")
        rows = [int(order[i]) for i in np.unique(np.round(np.linspace(0, nq - 1, k)).astype(np.int64))]
        t0 = time.perf_counter()
        pi = oracle.ppr_power(g, srcs[rows], alpha)
        t_cpu = time.perf_counter() - t0
        got = p[torch.as_tensor(rows, device=dev)].cpu().numpy().astype(np.float64)
        ratio = np.abs(got - pi) / (eps * np.maximum(deg, 1.0))
        within = bool(np.all(np.abs(got - pi) <= eps * deg + 1e-6))
        return {"workload": "rmat22_ppr", "alpha": alpha, "eps": eps, "seeds": nq, "checked_seeds": len(rows),
                "checked_seed_degrees": [int(deg[srcs[r]]) for r in rows],
                "max_err_over_eps_deg": float(ratio.max()), "mean_err_over_eps_deg": float(ratio.mean()),
                "p99_err_over_eps_deg": float(np.percentile(ratio, 99)), "within_bound": within,
                "mass_err_max": float((mass - 1.0).abs().max()), "batch_s": t_gpu, "oracle_s": t_cpu,
                "bound": "|p - pi| <= eps * d + 1e-6 per vertex (undirected)"}
    finally:
        fg.fg_graph_destroy(h)


def grid_extra(fg, inputs, dev, stream):
    """The grid workload (1,024 BFS + 1,024 SSSP sources, one batch each, hand-swept schedules)."""
    import torch
    g = inputs.workload_graph(GRID_WORKLOAD)
    srcs = source_sets(g, 0)[0]
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0,
                                  fg.fg_default_graph_opts(partition_method=fg.FG_PART_GROW))
    fg.check(st)
    try:
        s_d = torch.from_numpy(srcs).to(dev)
        out = torch.empty((GRID_NQ, g.n), dtype=torch.int32, device=dev)
        res = {}
        for kind, opts in (("bfs", TUNED_BFS), ("sssp", TUNED_SSSP)):
            f = fg.fg_bfs_batch if kind == "bfs" else fg.fg_sssp_batch
            o = fg.fg_default_opts(**opts)
            fg.check(f(h, s_d, GRID_NQ, out, stream, o))
            fg.check(fg.fg_sync(stream))
            ms = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fg.check(f(h, s_d, GRID_NQ, out, stream, o))
                b.record(stream)
                fg.check(fg.fg_sync(stream))
                ms.append(a.elapsed_time(b))
            d = fg.fg_stats(h)[1].as_dict()
            res[kind] = {"ms": statistics.median(ms), "opts": opts, "group": d["group"], "rounds": d["rounds"]}
        res["value"] = 2 * GRID_NQ / ((res["bfs"]["ms"] + res["sssp"]["ms"]) / 1e3)
        res["unit"] = UNIT
        res["graph"] = GRID_DESC
        return res
    finally:
        fg.fg_graph_destroy(h)


def serving_extra(fg, inputs, requests=300, lambdas=(2000.0, 50000.0)):
    """The serving workload (directed R-MAT s25, edge factor 24): Poisson streams of mixed
    SSSP / BFS / PPR(alpha 0.15, eps 1e-6) requests through fg_server_*, at the lowest and
    highest arrival rates of the workload; both are above what the loop sustains, so the
    runs measure the saturated throughput and the latency a queue of that depth gives."""
    g = inputs.workload_graph("rmat25_serving")
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        # batch lanes: SSSP in groups of 64, BFS in groups of 32 (a 64-query batch
        # is one group); slot lanes take 32 (the largest group of the serve mode)
        opts = {0: {"group": 64}, 1: {"group": 32}}
        runs = [serve_stream(fg, h, g, lam, requests, seed=int(lam), lanes=4, max_batch=64, kinds=(0, 1, 2),
                             alpha=0.15, eps=1e-6, opts=opts) for lam in lambdas]
        # slot-level batching: SSSP and BFS join running launches lane by lane,
        # PPR keeps two batch lanes
        runs += [serve_stream(fg, h, g, lam, requests, seed=int(lam), lanes=2, max_batch=64, kinds=(0, 1, 2),
                              alpha=0.15, eps=1e-6, opts=opts, continuous=1, slots=128) for lam in lambdas]
    finally:
        fg.fg_graph_destroy(h)
    return {"workload": "rmat25_serving", "graph": "directed R-MAT scale 25, edge factor 24, weights [1,255]",
            "mix": "1/3 SSSP, 1/3 BFS, 1/3 PPR(alpha=0.15, eps=1e-6)", "requests_per_rate": requests,
            "sustained_qps": max(r["throughput_qps"] for r in runs),
            "sustained_qps_by_mode": {m: max(r["throughput_qps"] for r in runs if r["mode"] == m)
                                      for m in ("batches", "slots")},
            "opts": {"sssp": opts[0], "bfs": opts[1]}, "runs": runs}


def run_rmat24(args):
    """The main line: SSSP batches of B sources on R-MAT scale 24 (see the module docstring)."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
        __graft_entry__.build()
    from paper_2103_14915_gb300 import fg, inputs

    t0 = time.perf_counter()
    g, name, desc = bench_graph(args)
    gen_s = time.perf_counter() - t0
    sha_got, sha_rec, sha_ok = csr_sha256_check(g, name)
    all_srcs = inputs.workload_sources(WORKLOAD, g) if not args.graph_scale else inputs.sources_uniform(
        g, int((np.diff(g.row_ptr) > 0).sum()) // 2, 1)
    nb = args.nq or NQ_STEP
    t0 = time.perf_counter()
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    create_s = time.perf_counter() - t0
    st, info = fg.fg_graph_info(h)
    fg.check(st)
    stream = torch.cuda.current_stream(dev)
    # schedule and query group: the library's autotuner on a 64-source sample taken
    # apart from the timed sources (outside the timed region)
    keys = ("group", "sched", "sched_window", "delta", "threads_per_vertex")
    if args.no_tune:
        opts_d = {}
        tune = {"chosen_by": "defaults (--no-tune)"}
    else:
        sample = torch.from_numpy(inputs.sources_uniform(g, 64, 4242)).to(dev)
        t0 = time.perf_counter()
        st, best, rep = fg.fg_tune_opts(h, fg.FG_QUERY_SSSP, sample, 64, stream)
        fg.check(st)
        opts_d = {k: int(getattr(best, k)) for k in keys}
        tune = {"chosen_by": "fg_tune_opts on 64 sources outside the timed set", "candidates": rep.candidates,
                "best_ms": rep.best_ms, "default_ms": rep.default_ms, "tune_s": time.perf_counter() - t0}
    opts_d.update(json.loads(args.opts_sssp) if args.opts_sssp else {})
    opts = fg.fg_default_opts(**opts_d)
    out = torch.empty((nb, g.n), dtype=torch.int32, device=dev)
    n_steps = args.warmup + args.steps
    src_d = [torch.from_numpy(step_sources(all_srcs, rank, ws, i, nb)).to(dev) for i in range(n_steps)]

    def step(i, ev=None):
        if ev is not None:
            ev[0].record(stream)
        fg.check(fg.fg_sssp_batch(h, src_d[i], nb, out, stream, opts))
        if ev is not None:
            ev[1].record(stream)
        fg.check(fg.fg_sync(stream))

    for i in range(args.warmup):
        step(i)
    st, stats = fg.fg_stats(h)
    fg.check(st)
    launches_per_step = int(stats.launches)

    clocks = ClockSampler(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_stats = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    t_start.record(stream)
    for i in range(args.steps):
        step(args.warmup + i, evs[i])
        step_stats.append(fg.fg_stats(h)[1].as_dict())
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), dev)
    value = job_rate(nb * args.steps, ws, elapsed_ms)
    batch_ms = [e[0].elapsed_time(e[1]) for e in evs]

    # GTEPS: arcs out of the vertices each query reaches (what a sequential Dijkstra scans), last step
    deg = torch.from_numpy(np.diff(g.row_ptr).astype(np.int64)).to(dev)
    reach_arcs = int(((out != -1).to(torch.int64) * deg[None, :]).sum().item())
    arcs_per_query = reach_arcs / nb
    gteps = arcs_per_query * value / 1e9

    # roofline of the engine launch (algorithmic bytes per launch / CUDA-event time per batch)
    peak, peak_kind = measured_peaks()
    mean = lambda k: statistics.mean(float(d[k]) for d in step_stats)
    group = int(step_stats[-1]["group"])
    out_bytes = 4 * g.n * nb
    arc_bytes = 8 * mean("arcs_read")
    op_bytes = 16 * mean("ops")
    alg_bytes = out_bytes + arc_bytes + op_bytes
    kern_ms = statistics.mean(batch_ms)
    achieved = alg_bytes / (kern_ms / 1000.0) / 1e9
    kernel = f"fg::group_kernel<0, {group}>" if group > 1 else "fg::engine_kernel<0>"
    traffic = (kernel_traffic("group_kernel_rmat24_traffic.txt", "fg_group.cu", nb, group)
               if group > 1 and not args.graph_scale else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": f"{peak_kind} hbm_gbs (STREAM-style copy)", "kernel": kernel,
                "algorithmic_bytes_per_launch": alg_bytes,
                "algorithmic_terms": {"output_4B_per_vertex_query": out_bytes, "arcs_8B_per_arc_read": arc_bytes,
                                      "operations_16B_each": op_bytes},
                "batch_ms": kern_ms, "timing": "CUDA events around each fg_sssp_batch on its stream "
                                               "(engine launch + its output transpose)"}
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": name, "graph": desc, "sources_per_step": nb, "kinds": ["sssp"],
                   "workload_sources": len(all_srcs),
                   "sources_timed": nb * args.steps * ws,
                   "fraction_of_workload_timed": min(1.0, nb * args.steps * ws / len(all_srcs)),
                   "partition": {"method": int(info.partition_method), "S": int(info.partition_vertices),
                                 "parts": int(info.num_partitions), "cut_arcs": int(info.cut_arcs)},
                   "opts": opts_d, "tuner": tune,
                   "l2": f"inputs larger than L2: each step writes {4 * nb * g.n / 1e9:.1f} GB of distances "
                         f"and the query state is {8 * nb * g.n / 1e9:.1f} GB",
                   "parallelism": f"queries sharded over {ws} GPU(s)"},
        "gteps": gteps, "arcs_per_query_dijkstra": arcs_per_query,
        "roofline": roofline,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "stats": step_stats[-1],
        "graph_build": {"generate_s": gen_s, "create_s": create_s, "csr_sha256": sha_got,
                        "csr_sha256_recorded": sha_rec, "csr_sha256_ok": sha_ok},
    }

    if not args.no_extras:
        # end to end through the C ABI with host buffers: every step copies its sources in
        # from pinned host memory and every distance row out to pinned host memory, with
        # asynchronous host I/O (host_io = 2) on two streams, so one batch's copy-out runs
        # behind the next batch's kernels
        o_h = fg.fg_default_opts(**opts_d)
        o_h.host_io = 2
        outs_h = [torch.empty((nb, g.n), dtype=torch.int32, pin_memory=True) for _ in range(2)]
        srcs_h = [torch.from_numpy(step_sources(all_srcs, rank, ws, i, nb)).pin_memory() for i in range(n_steps)]
        streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
        fg.check(fg.fg_sssp_batch(h, srcs_h[0].data_ptr(), nb, outs_h[0].data_ptr(), streams[0], o_h))
        fg.check(fg.fg_sync(streams[0]))
        e_steps = args.steps
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(e_steps):
            k = i & 1
            if i >= 2:
                fg.check(fg.fg_sync(streams[k]))  # this host buffer's previous batch is complete
            fg.check(fg.fg_sssp_batch(h, srcs_h[args.warmup + i].data_ptr(), nb, outs_h[k].data_ptr(),
                                      streams[k], o_h))
        for k in range(2):
            fg.check(fg.fg_sync(streams[k]))
        e_dt = time.perf_counter() - t0
        e_value = max_over_ranks(e_dt * 1000.0, dev)
        result["e2e"] = {"value": job_rate(nb * e_steps, ws, e_value), "unit": UNIT,
                         "h2d_bytes_per_step": 4 * nb, "d2h_bytes_per_step": 4 * nb * g.n, "steps": e_steps,
                         "api": "fg_sssp_batch with host_io=2 (pinned host buffers, two streams)"}
        del outs_h
        if rank == 0:
            import oracle
            # the plain per-query GPU form on a sample of the same sources
            k = max(1, args.plain_sample // 4)
            o_plain = fg.fg_default_opts(mode=fg.FG_MODE_PLAIN)
            s = src_d[0][:k].contiguous()
            fg.check(fg.fg_sssp_batch(h, s, 1, out, stream, o_plain))
            fg.check(fg.fg_sync(stream))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fg.check(fg.fg_sssp_batch(h, s, k, out, stream, o_plain))
            b.record(stream)
            fg.check(fg.fg_sync(stream))
            result["plain_gpu"] = {"value": k / (a.elapsed_time(b) / 1000.0), "unit": UNIT,
                                   "sample": f"{k} sources, one query at a time (FG_MODE_PLAIN)"}
            # BFS levels of the first timed step's sources, options from the
            # autotuner on the same 64-source sample as the SSSP line, two timed
            # batches after a warm-up one, four rows checked against the oracle
            if args.no_tune:
                ob = fg.fg_default_opts(group=int(opts.group))
            else:
                tune_src = torch.from_numpy(inputs.sources_uniform(g, 64, 4242)).to(dev)
                st, ob, _ = fg.fg_tune_opts(h, fg.FG_QUERY_BFS, tune_src, 64, stream)
                fg.check(st)
            s_b = src_d[0]
            fg.check(fg.fg_bfs_batch(h, s_b, nb, out, stream, ob))
            fg.check(fg.fg_sync(stream))
            a.record(stream)
            for _ in range(2):
                fg.check(fg.fg_bfs_batch(h, s_b, nb, out, stream, ob))
            b.record(stream)
            fg.check(fg.fg_sync(stream))
            bfs_ms = a.elapsed_time(b) / 2
            kb = 4
            ref_b = oracle.bfs(g, s_b[:kb].cpu().numpy())
            result["bfs_same_batch"] = {
                "value": nb / (bfs_ms / 1000.0), "unit": UNIT, "ms_per_batch": bfs_ms, "group": int(ob.group),
                "exact_sampled": {"rows": kb, "exact": bool(np.array_equal(out[:kb].cpu().numpy().view(np.uint32),
                                                                             ref_b))}}
            # parity of the timed path on a sampled row, and the CPU oracle on the host cores
            cores = oracle.num_threads()
            kc = args.cpu_sources or max(1, min(cores, 16))
            cs = step_sources(all_srcs, 0, 1, 0, kc)
            t0 = time.perf_counter()
            ref = oracle.sssp(g, cs)
            cdt = time.perf_counter() - t0
            fg.check(fg.fg_sssp_batch(h, torch.from_numpy(cs).to(dev), kc, out, stream, opts))
            fg.check(fg.fg_sync(stream))
            result["exact_sampled"] = {"rows": kc, "exact": bool(np.array_equal(
                out[:kc].cpu().numpy().view(np.uint32), ref))}
            result["cpu_baseline"] = {"value": kc / cdt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                      "sample": f"{kc} of the {len(all_srcs):,} sources (one per host core), "
                                                "binary-heap Dijkstra, OpenMP over queries"}
            fg.fg_graph_destroy(h)
            h = None
            del out
            torch.cuda.empty_cache()
            if not args.no_grid_extra:
                result["grid1024_bfs_sssp"] = grid_extra(fg, inputs, dev, stream)
            if not args.no_ppr_check:
                result["ppr_rmat22"] = ppr_error_record(fg, inputs, oracle, dev)
            if not args.no_serving_extra:
                result["serving_rmat25"] = serving_extra(fg, inputs)
    if h is not None:
        fg.fg_graph_destroy(h)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_grid(args):
    """The grid workload as the main line: one step = one BFS and one SSSP batch of the same
    1,024 seeded sources (2,048 source queries); three source sets rotate across steps."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
        __graft_entry__.build()
    from paper_2103_14915_gb300 import fg, inputs

    g = inputs.workload_graph(GRID_WORKLOAD)
    nq = args.nq or GRID_NQ
    sets = source_sets(g, rank, nq)
    gopts = fg.fg_default_graph_opts(partition_method=fg.FG_PART_GROW, partition_vertices=args.partition_vertices)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, gopts)
    fg.check(st)
    st, info = fg.fg_graph_info(h)
    fg.check(st)
    stream = torch.cuda.current_stream(dev)
    src_d = [torch.from_numpy(s).to(dev) for s in sets]
    # schedules: the library's autotuner on the first source set (outside the
    # timed region), or the hand-swept constants with --no-tune
    tune = {}
    if args.no_tune:
        base_b, base_s = dict(TUNED_BFS), dict(TUNED_SSSP)
    else:
        keys = ("sched", "sched_window", "delta", "threads_per_vertex")
        picked = []
        for kind in (fg.FG_QUERY_BFS, fg.FG_QUERY_SSSP):
            st, best, rep = fg.fg_tune_opts(h, kind, src_d[0], nq, stream)
            fg.check(st)
            picked.append({k: int(getattr(best, k)) for k in keys})
            tune["bfs" if kind == fg.FG_QUERY_BFS else "sssp"] = {
                "candidates": rep.candidates, "best_ms": rep.best_ms, "default_ms": rep.default_ms}
        base_b, base_s = picked
    extra_b = dict(base_b, **(json.loads(args.opts_bfs) if args.opts_bfs else {}))
    extra_s = dict(base_s, **(json.loads(args.opts_sssp) if args.opts_sssp else {}))
    opts_b = fg.fg_default_opts(**extra_b)
    opts_s = fg.fg_default_opts(**extra_s)
    level = torch.empty((nq, g.n), dtype=torch.int32, device=dev)
    dist_t = torch.empty((nq, g.n), dtype=torch.int32, device=dev)

    def step(i, ev=None):
        s = src_d[i % SOURCE_SETS]
        if ev is not None:
            ev[0].record(stream)
        fg.check(fg.fg_bfs_batch(h, s, nq, level, stream, opts_b))
        if ev is not None:
            ev[1].record(stream)
        fg.check(fg.fg_sssp_batch(h, s, nq, dist_t, stream, opts_s))
        if ev is not None:
            ev[2].record(stream)
        fg.check(fg.fg_sync(stream))

    for i in range(args.warmup):
        step(i)
    # kernel launches per batch, from the library's own count
    fg.check(fg.fg_bfs_batch(h, src_d[0], nq, level, stream, opts_b))
    fg.check(fg.fg_sync(stream))
    st, sb = fg.fg_stats(h)
    fg.check(fg.fg_sssp_batch(h, src_d[0], nq, dist_t, stream, opts_s))
    fg.check(fg.fg_sync(stream))
    st, ss = fg.fg_stats(h)
    launches_per_step = int(sb.launches + ss.launches)

    clocks = ClockSampler(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    t_start.record(stream)
    for i in range(args.steps):
        step(args.warmup + i, evs[i])
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    elapsed_ms = max_over_ranks(elapsed_ms, dev)
    value = job_rate(2 * nq * args.steps, ws, elapsed_ms)
    bfs_ms = [e[0].elapsed_time(e[1]) for e in evs]
    sssp_ms = [e[1].elapsed_time(e[2]) for e in evs]

    # GTEPS: arcs out of reachable vertices (the edges a sequential Dijkstra / BFS scans)
    deg = torch.from_numpy(np.diff(g.row_ptr).astype(np.int64)).to(dev)
    arcs_per_set = []
    for i in range(SOURCE_SETS):
        fg.check(fg.fg_bfs_batch(h, src_d[i], nq, level, stream, opts_b))
        fg.check(fg.fg_sync(stream))
        reach = level.view(torch.int32) != -1
        arcs_per_set.append(int((reach.to(torch.int64) * deg[None, :]).sum().item()))
    arcs = sum(2 * arcs_per_set[(args.warmup + i) % SOURCE_SETS] for i in range(args.steps)) * ws
    gteps = arcs / (elapsed_ms / 1000.0) / 1e9

    peak, peak_kind = measured_peaks()
    graph_bytes = int(info.device_bytes)
    alg_bytes = 4 * nq * g.n + graph_bytes  # dense output written once + graph read once per launch
    kern_ms = statistics.mean(bfs_ms + sssp_ms)
    achieved = alg_bytes / (kern_ms / 1000.0) / 1e9
    traffic = engine_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": f"{peak_kind} hbm_gbs (STREAM-style copy)",
                "kernel": "fg::engine_kernel", "algorithmic_bytes_per_launch": alg_bytes,
                "kernel_ms": {"bfs": statistics.mean(bfs_ms), "sssp": statistics.mean(sssp_ms)}}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": GRID_WORKLOAD, "graph": GRID_DESC, "sources_per_batch": nq, "kinds": ["bfs", "sssp"],
                   "queries_per_step": 2 * nq, "source_sets": SOURCE_SETS,
                   "partition": {"method": "grow", "S": int(info.partition_vertices),
                                 "parts": int(info.num_partitions), "cut_arcs": int(info.cut_arcs)},
                   "opts": {"bfs": extra_b, "sssp": extra_s, "chosen_by": "hand sweep" if args.no_tune else
                            "fg_tune_opts on source set 0", "tuner": tune},
                   "l2": f"inputs larger than L2: each step writes {8 * nq * g.n / 1e9:.1f} GB of query state",
                   "parallelism": f"queries sharded over {ws} GPU(s)"},
        "gteps": gteps,
        "roofline": roofline,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "stats": {"bfs": sb.as_dict(), "sssp": ss.as_dict()},
    }

    if not args.no_extras:
        # end to end through the C ABI with host buffers: sources copied in from pinned host
        # memory, every result row copied out, each step; asynchronous host I/O (host_io = 2)
        # with BFS and SSSP on two streams, so one batch's copy-out overlaps the next kernels
        o_hb = fg.fg_default_opts(**extra_b)
        o_hb.host_io = 2
        o_hs = fg.fg_default_opts(**extra_s)
        o_hs.host_io = 2
        lv_h = torch.empty((nq, g.n), dtype=torch.int32, pin_memory=True)
        ds_h = torch.empty((nq, g.n), dtype=torch.int32, pin_memory=True)
        src_h = [torch.from_numpy(s).pin_memory() for s in sets]
        s_a, s_b = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        e_steps = max(1, min(args.steps, 4))
        fg.check(fg.fg_bfs_batch(h, src_h[0].data_ptr(), nq, lv_h.data_ptr(), s_a, o_hb))
        fg.check(fg.fg_sssp_batch(h, src_h[0].data_ptr(), nq, ds_h.data_ptr(), s_b, o_hs))
        fg.check(fg.fg_sync(s_a))
        fg.check(fg.fg_sync(s_b))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(e_steps):
            s = src_h[i % SOURCE_SETS].data_ptr()
            fg.check(fg.fg_bfs_batch(h, s, nq, lv_h.data_ptr(), s_a, o_hb))
            fg.check(fg.fg_sssp_batch(h, s, nq, ds_h.data_ptr(), s_b, o_hs))
        fg.check(fg.fg_sync(s_a))
        fg.check(fg.fg_sync(s_b))
        e_dt = time.perf_counter() - t0
        result["e2e"] = {"value": 2 * nq * e_steps / e_dt, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * nq,
                         "d2h_bytes_per_step": 2 * 4 * nq * g.n, "steps": e_steps,
                         "api": "fg_bfs_batch + fg_sssp_batch with host_io=2 (pinned host buffers, two streams)"}
        del lv_h, ds_h
        if rank == 0:
            # plain per-query GPU form on a sample of the same sources
            o_plain = fg.fg_default_opts(mode=fg.FG_MODE_PLAIN)
            k = args.plain_sample
            s = src_d[0][:k].contiguous()
            fg.check(fg.fg_bfs_batch(h, s, 1, level, stream, o_plain))
            fg.check(fg.fg_sync(stream))
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fg.check(fg.fg_bfs_batch(h, s, k, level, stream, o_plain))
            fg.check(fg.fg_sssp_batch(h, s, k, dist_t, stream, o_plain))
            b.record(stream)
            fg.check(fg.fg_sync(stream))
            pms = a.elapsed_time(b)
            result["plain_gpu"] = {"value": 2 * k / (pms / 1000.0), "unit": UNIT,
                                   "sample": f"{k} sources, BFS + SSSP, one query at a time (FG_MODE_PLAIN)"}
            # CPU oracle on the host cores
            import oracle
            cs = source_sets(g, rank)[0][: args.cpu_sample]
            t0 = time.perf_counter()
            oracle.bfs(g, cs)
            oracle.sssp(g, cs)
            cdt = time.perf_counter() - t0
            result["cpu_baseline"] = {"value": 2 * len(cs) / cdt, "unit": UNIT, "cores": oracle.num_threads(),
                                      "kind": "oracle",
                                      "sample": f"{len(cs)} of the 1,024 sources, BFS + SSSP, OpenMP over queries"}
            # serving loop on the same resident graph: Poisson stream of mixed requests
            result["serving"] = dict(
                serve_stream(fg, h, g, args.serve_lambda, args.serve_requests, seed=77, lanes=4, max_batch=128,
                             kinds=(0, 1, 2), alpha=0.15, eps=1e-6, opts={0: extra_s, 1: extra_b}),
                graph=GRID_WORKLOAD, mix="1/3 SSSP, 1/3 BFS, 1/3 PPR(alpha=0.15, eps=1e-6)")
    fg.fg_graph_destroy(h)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        dist.destroy_process_group()




def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serving:
        run_serving(args)
        return
    if args.ablation:
        run_ablation(args)
        return
    if args.ncp:
        run_ncp(args)
        return
    if args.ll:
        run_ll(args)
        return
    if args.bc:
        run_bc(args)
        return
    if args.walks:
        run_walks(args)
        return
    if args.local_ppr:
        run_local_ppr(args)
        return
    if args.configs:
        run_configs(args)
        return
    if args.grid:
        run_grid(args)
        return
    run_rmat24(args)


if __name__ == "__main__":
    main()
