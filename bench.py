#!/usr/bin/env python
"""Benchmark: betweenness TEPS of GPU plain Brandes and GPU Brandes++ on GB300.

Workload (default, the largest single-GPU configuration): undirected unweighted Chung-Lu graph
with planted communities, n = 1,000,000 in 1,000 communities of 1,000, degree exponent 2.2,
mean degree 16 (m = 8,000,000 edges), 85% of the edges drawn inside communities; the target
set S is 4,096 uniformly sampled nodes and the planted communities are the partition; FP64.
``--workload`` selects the other configurations (see ``gen.WORKLOADS``).

One step computes the target-set betweenness twice through the library's C ABI on resident
inputs: plain Brandes (Eq. 5-7) and Brandes++ (Alg. 1: Build_SK, Brandes_SK, Centrality).
TEPS counts |S| * m source-edge pairs per betweenness computation, so a step is 2 * |S| * m
units and Brandes++/plain is the time ratio.  The L2 cache (129 MB) is flushed before every
step by writing a 512 MiB buffer.

Under torchrun (N > 1 ranks, one GPU each) the step is source-sharded (strong scaling): every
rank computes its shard of the sources on its replica of the graph, and one FP64 NCCL sum
all-reduce per result gives every rank the full betweenness (``sharded.sharded_sum``).

--impl reference times the CPU oracle instead (the paper has no GPU implementation to run) on
all host cores, each step a bounded sample of the sources.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BC TEPS (sources x edges / s), Brandes++ vs plain GPU Brandes"
UNIT = "TEPS"
DEFAULT_WORKLOAD = "chunglu_1m"
# Workloads on which the CPU oracle's Brandes++ cannot be sampled within the baseline's time
# budget: its Build_SK runs Dijkstra_SK from every frontier before the first source (on
# chunglu_1m, about 650,000 frontiers: about 4 minutes on one core), so the CPU legs time the
# oracle's plain Brandes only there.
ORACLE_PP_SKIPPED = {"chunglu_1m": "the oracle's Build_SK alone (Dijkstra_SK from about 650,000 frontiers) "
                                   "takes about 4 minutes on one core"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of each CPU oracle leg")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end (host buffer) timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip the captured-plan (CUDA graph) measurement")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--no-roofline-model", action="store_true",
                    help="skip the distance samples behind the rooflines' tight-arc counts")
    ap.add_argument("--pp-all", action="store_true",
                    help="also time Brandes++All (Alg. 3, all pairs of parts; S = V workloads only) once")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.first = 0
        self.reader = None

    def start(self):
        """Start sampling and wait (up to 5 s) for the first sample, so that nvidia-smi's own
        start-up (driver and NVML initialisation) is over before the timed region begins."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.reader = threading.Thread(target=lambda: self.lines.extend(self.proc.stdout), daemon=True)
        self.reader.start()
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.first = len(self.lines)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        if self.reader is not None:
            self.reader.join(timeout=5)
        # the samples taken during the timed region, else the one taken just before it
        lines = self.lines[self.first:] or self.lines[:self.first]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    """(HBM GB/s, SM max MHz, source) from MEASURED_PEAKS.json, else the recipe's fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 2070.0, "fallback"


def alu_peak_ops(num_sms, sm_mhz):
    """32-bit integer lane operations per second: SMs x 4 schedulers x 32 lanes x clock (each
    scheduler issues one warp instruction per cycle)."""
    return num_sms * 4 * 32 * sm_mhz * 1e6


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("lockstep.cu", "lockstep.cuh", "lockstep_kernel.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1406_4173_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu record
    (profiles/<kernel>_<workload>.json), if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.json")
    try:
        with open(p) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, TypeError, ValueError):
        return None


def model_bytes_per_source(n, A, D, B=32, delta_bytes=8):
    """Algorithmic bytes of one source of plain Brandes (unit weights), per the traffic model:
    forward = A(4 col + 4 d-probe) + D*8 (parent sigma) + n(8 row_ptr + 4 d + 8 sigma),
    backward = A(4 col + 4 d-probe) + D(8 sigma + delta) + n(8 row_ptr + delta + 8 bc),
    with the col and row_ptr terms shared by the B sources of a batch."""
    fwd = A * (4 / B + 4) + D * 8 + n * (8 / B + 4 + 8)
    bwd = A * (4 / B + 4) + D * (8 + delta_bytes) + n * (8 / B + delta_bytes + 8)
    return fwd + bwd


def model_bytes_per_source_skeleton(N, A, D, B=32, delta_bytes=8, weighted=True, mult=True):
    """Algorithmic bytes of one source of Brandes_SK (Eq. 11-12) on a skeleton of N nodes and A
    arcs with D tight arcs: the plain-Brandes model plus, per arc and pass, the arc's weight
    (4 bytes) and multiplicity (8 bytes), read with the heads and shared by the B sources."""
    extra = A * 2 * ((4 if weighted else 0) + (8 if mult else 0)) / B
    return model_bytes_per_source(N, A, D, B, delta_bytes) + extra


def centrality_ops_per_source(interior_entries):
    """Algorithmic integer operations of the Centrality step per source: for every (frontier,
    non-frontier node) table entry, one add and one compare in the forward min-plus and one
    add and one compare in the backward tight-exit test."""
    return 4.0 * interior_entries


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0))) if a.size else 0.0


# ----------------------------------------------------------------------------- CPU oracle on all host cores
_G = {}


def _pool_init(path):
    """Worker initializer: the workload's arrays from the shared temporary file."""
    from paper_1406_4173_gb300 import gen
    import oracle
    oracle.build()
    z = np.load(path)
    w = z["w"] if z["w"].size else None
    _G["g"] = gen.EdgeList(n=int(z["n"]), src=z["src"], dst=z["dst"], w=w, directed=bool(z["directed"]),
                           part=z["part"] if z["part"].size else None)
    _G["S"] = z["S"]


def _pool_task(args):
    """The oracle's partial betweenness (unhalved) of the sources at positions [lo, hi) of S,
    all of S as targets; returns (partial, seconds)."""
    kind, lo, hi = args
    import oracle
    g, S = _G["g"], _G["S"]
    mine = S[lo:hi]
    order = np.concatenate([mine, np.setdiff1d(S, mine, assume_unique=True)]).astype(np.int32)
    t0 = time.perf_counter()
    if kind == "plain":
        bc, _ = oracle.brandes(g, order, nsrc=hi - lo, halve=False)
    else:
        bc, _, _ = oracle.brandes_pp(g, order, g.part, nsrc=hi - lo, halve=False)
    return bc, time.perf_counter() - t0


class OraclePool:
    """A spawned process pool (one worker per host core) running the CPU oracle on shards of
    the sources; the workload travels through a temporary file."""

    def __init__(self, g, S):
        import multiprocessing as mp
        self.cores = os.cpu_count() or 1
        self.dir = tempfile.mkdtemp(prefix="bcpp_oracle_")
        path = os.path.join(self.dir, "w.npz")
        np.savez(path, n=g.n, src=g.src, dst=g.dst, w=g.w if g.w is not None else np.zeros(0, np.uint32),
                 directed=g.directed, part=g.part if g.part is not None else np.zeros(0, np.int32),
                 S=np.asarray(S, np.int32))
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_pool_init, initargs=(path,))
        self.nS = len(S)

    def run(self, kind, lo, hi):
        """Partial over source positions [lo, hi) split across the workers: (sum, wall seconds)."""
        from paper_1406_4173_gb300 import api
        tasks = []
        for w in range(self.cores):
            a, b = api.shard_bounds(hi - lo, w, self.cores)
            if b > a:
                tasks.append((kind, lo + a, lo + b))
        t0 = time.perf_counter()
        res = self.pool.map(_pool_task, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        return np.sum([r[0] for r in res], axis=0), wall

    def probe(self, kind):
        """Seconds of one source on one worker (includes the oracle's per-call setup)."""
        _, t = self.pool.apply(_pool_task, ((kind, 0, 1),))
        return t

    def close(self):
        self.pool.terminate()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)


def _batch_task(graphs):
    """The oracle's full betweenness of each graph of a chunk; returns (results, seconds)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    out = [oracle.brandes(gi)[0] for gi in graphs]
    return out, time.perf_counter() - t0


class BatchOraclePool:
    """A spawned process pool (one worker per host core) running the CPU oracle on chunks of the
    batch workload's graphs."""

    def __init__(self, graphs):
        import multiprocessing as mp
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_batch_task, [graphs[:1]] * self.cores, chunksize=1)   # workers up, oracle loaded

    def run(self, graphs, chunk=8):
        """Full betweenness of every graph given, `chunk` graphs per task."""
        tasks = [graphs[i:i + chunk] for i in range(0, len(graphs), chunk)]
        out = []
        for res, _ in self.pool.map(_batch_task, tasks, chunksize=1):
            out.extend(res)
        return out

    def close(self):
        self.pool.terminate()
        self.pool.join()


def batch_oracle_sample(graphs, seconds, chunk=8):
    """The CPU oracle on the batch workload, on all host cores: rounds of one `chunk`-graph task
    per worker over the graphs in order, until `seconds` of wall time have passed (at least one
    round).  Returns
    (results of the first `done` graphs, done, units per second, cores)."""
    bp = BatchOraclePool(graphs)
    try:
        refs, done = [], 0
        t0 = time.perf_counter()
        while done < len(graphs) and (done == 0 or time.perf_counter() - t0 < seconds):
            take = graphs[done:done + bp.cores * chunk]
            refs.extend(bp.run(take, chunk))
            done += len(take)
        wall = time.perf_counter() - t0
    finally:
        bp.close()
    units = float(sum(gi.n * gi.m for gi in graphs[:done]))
    return refs, done, units / max(wall, 1e-9), bp.cores


def oracle_sample(pool, workload, seconds, m):
    """Time the oracle on a bounded sample: the first `ns` sources of S (shard 0 of `count`), sized
    so that each leg takes about `seconds` of wall time on all cores.  Returns a dict with the
    plain partial (for the error check) and the timings."""
    from paper_1406_4173_gb300 import api
    per = pool.probe("plain")
    want = int(max(pool.cores, min(pool.nS, pool.cores * seconds / max(per, 1e-6))))
    count = max(1, pool.nS // want)
    _, ns = api.shard_bounds(pool.nS, 0, count)
    ref, tp = pool.run("plain", 0, ns)
    out = {"ns": ns, "count": count, "t_plain": tp, "ref_plain": ref, "t_pp": None, "ns_pp": 0}
    if workload not in ORACLE_PP_SKIPPED:
        per_pp = pool.probe("pp")
        k = int(max(1, min(ns // pool.cores, seconds / max(per_pp, 1e-6))))
        ns_pp = min(ns, k * pool.cores)
        _, tpp = pool.run("pp", 0, ns_pp)
        out.update(t_pp=tpp, ns_pp=ns_pp)
    out["value"] = (ns + out["ns_pp"]) * m / (tp + (out["t_pp"] or 0.0))
    legs = f"oracle plain Brandes, first {ns} of {pool.nS} sources (targets = S), {tp:.1f} s"
    if out["t_pp"] is not None:
        legs += f"; oracle Brandes++, first {out['ns_pp']} sources, {out['t_pp']:.1f} s"
    else:
        legs += f"; Brandes++ oracle not sampled: {ORACLE_PP_SKIPPED[workload]}"
    out["sample"] = f"{legs}; {pool.cores} spawned worker processes, one per host core"
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1406_4173_gb300 import api, gen
    import oracle
    oracle.build()
    g, S = gen.workload(args.workload)
    cores = os.cpu_count() or 1
    if isinstance(g, list):
        graphs = g
        bp = BatchOraclePool(graphs)
        take = graphs[:bp.cores * 8]
        units = float(sum(gi.n * gi.m for gi in take))
        try:
            for _ in range(args.warmup):
                bp.run(take)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                bp.run(take)
            dt = time.perf_counter() - t0
        finally:
            bp.close()
        val = units * args.steps / dt
        sample = (f"first {len(take)} graphs per step, full betweenness each, {bp.cores} spawned worker "
                  "processes, one per host core")
        cfg = {"workload": args.workload, "graphs_per_step": len(take)}
        cores = bp.cores
    else:
        Sall = np.arange(g.n, dtype=np.int32) if S is None else np.asarray(S, np.int32)
        pool = OraclePool(g, Sall)
        try:
            budget = max(1.0, 150.0 / max(1, args.steps + args.warmup))   # the whole run within a few minutes
            per = pool.probe("plain")
            ns = int(max(pool.cores, min(len(Sall), pool.cores * budget / max(per, 1e-6))))
            with_pp = args.workload not in ORACLE_PP_SKIPPED
            ns_pp = 0
            if with_pp:
                per_pp = pool.probe("pp")
                ns_pp = int(max(pool.cores, min(ns, pool.cores * budget / max(per_pp, 1e-6))))

            def step():
                pool.run("plain", 0, ns)
                if with_pp:
                    pool.run("pp", 0, ns_pp)

            for _ in range(args.warmup):
                step()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                step()
            dt = time.perf_counter() - t0
        finally:
            pool.close()
        val = (ns + ns_pp) * g.m * args.steps / dt
        sample = (f"per step: oracle plain Brandes from the first {ns} of {len(Sall)} sources"
                  + (f" and oracle Brandes++ from the first {ns_pp}" if with_pp else
                     f" (Brandes++ oracle not sampled: {ORACLE_PP_SKIPPED[args.workload]})")
                  + f", targets = S; {cores} spawned worker processes")
        cfg = {"workload": args.workload, "n": g.n, "m": g.m, "S": len(Sall), "sample_sources_per_step": ns,
               "sample_sources_pp_per_step": ns_pp}
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- ours
def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, x, dev):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import paper_1406_4173_gb300 as bc
    from paper_1406_4173_gb300 import _build, gen
    _build.build()
    g, S = gen.workload(args.workload)
    # the oracle pool is spawned before the first GPU call of this process
    pool = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not isinstance(g, list):
        pool = OraclePool(g, np.arange(g.n, dtype=np.int32) if S is None else S)
    try:
        dev = torch.device("cuda", torch.cuda.current_device())
        ctx = bc.default_context()
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        if isinstance(g, list):
            line = _run_batched(args, bc, g, ctx, flush, dev, ws, rank)
        else:
            line = _run_single(args, bc, g, S, ctx, flush, dev, ws, rank, pool)
    finally:
        if pool is not None:
            pool.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _timed(args, ws, dev, step):
    """W warm-up steps, then K steps between barriers and device syncs; clock samples."""
    import torch
    for _ in range(args.warmup):
        step()
    clk = Clocks(torch.cuda.current_device())
    _barrier(ws)
    torch.cuda.synchronize()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    logs = []
    e0.record()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        logs.append(step())
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    _barrier(ws)
    clocks = clk.stop()
    dt = _max_over_ranks(ws, e0.elapsed_time(e1) / 1e3, dev)
    return dt, wall, logs, clocks


def _tight_arcs(bc, G, src, ctx):
    """Mean number of tight arcs (d(v) = d(u) + w(u,v)) per source over the given sources, from
    the library's bit-exact distances."""
    dist_s, _ = bc.sssp(G, np.asarray(src, np.int32), ctx=ctx, allow_overflow=True)
    dist_s = dist_s.cpu().numpy().astype(np.int64)
    rp = G.row_ptr.cpu().numpy()
    col = G.col.cpu().numpy()
    wts = 1 if G.w is None else G.w.cpu().numpy().astype(np.int64)
    tails = np.repeat(np.arange(G.n), np.diff(rp))
    tight = []
    for dd in dist_s:
        ok = (dd[tails] < np.iinfo(np.int32).max) & (dd[col] == dd[tails] + wts)
        tight.append(int(ok.sum()))
    return float(np.mean(tight))


def _skeleton_model(bc, g, G, S, part, ctx):
    """Sizes behind the Brandes_SK and Centrality rooflines: skeleton nodes N and arcs, mean
    tight skeleton arcs per source (the library's distances on the skeleton from 32 sampled
    targets), whether weights / multiplicities exceed 1, and the Centrality table entries
    sum_i |F_i| (|V_i| - |F_i|) over the parts with frontiers (V_i without the targets)."""
    nodes, (au, av, aw, amu) = bc.skeleton(G, S, part, ctx=ctx)
    N = len(nodes)
    arcs = len(au)
    in_s = np.zeros(g.n, bool)
    in_s[np.asarray(S)] = True
    k = int(part.max()) + 1
    V = np.bincount(part[~in_s], minlength=k).astype(np.int64)
    fr = nodes[~in_s[nodes]]
    F = np.bincount(part[fr], minlength=k).astype(np.int64)
    interior = int(np.sum(np.where(F > 0, F * (V - F), 0)))
    su = np.searchsorted(nodes, au).astype(np.int32)
    sv = np.searchsorted(nodes, av).astype(np.int32)
    keep = su < sv if not g.directed else np.ones(len(su), bool)
    Gsk = bc.csr_build(N, su[keep], sv[keep], aw[keep].astype(np.uint32), g.directed, ctx)
    sample = np.searchsorted(nodes, np.asarray(S)[np.linspace(0, len(S) - 1, 32).astype(int)]).astype(np.int32)
    D = _tight_arcs(bc, Gsk, sample, ctx)
    return {"N": N, "arcs": arcs, "D": D, "weighted": bool(aw.size and aw.max() > 1),
            "mult": bool(amu.size and amu.max() > 1), "interior_entries": interior}


def _roof(bound, achieved, peak, unit, kernel, traffic, **extra):
    d = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
         "frac": achieved / peak if peak else None, "traffic": traffic, "kernel": kernel}
    d.update(extra)
    return d


def _run_single(args, bc, g, S, ctx, flush, dev, ws, rank, pool):
    import torch
    from paper_1406_4173_gb300 import api, sharded
    n, m = g.n, g.m
    S_order = np.arange(n, dtype=np.int32) if S is None else np.asarray(S, np.int32)
    nS = len(S_order)
    Sarg = None if S is None or len(S) == n else S
    prec = args.precision
    part = torch.as_tensor(g.part, device=dev)
    G = bc.graph_from_edgelist(g)
    A = G.num_arcs
    bc_plain = torch.empty(n, dtype=torch.float64, device=dev)
    bc_pp = torch.empty(n, dtype=torch.float64, device=dev)
    shard = (rank, ws) if ws > 1 else None
    my_sources = api.shard_bounds(nS, rank, ws)
    my_ns = my_sources[1] - my_sources[0]

    def step():
        flush.fill_(1)
        st = {}

        def plain(r, R):
            _, st["plain"] = bc.brandes(G, Sarg, precision=prec, out=bc_plain, stats=True, ctx=ctx, shard=shard)
            return bc_plain

        def pp(r, R):
            _, st["pp"] = bc.brandes_pp(G, Sarg, part, precision=prec, out=bc_pp, stats=True, ctx=ctx, shard=shard)
            return bc_pp

        if ws > 1:
            sharded.sharded_sum(plain)
            sharded.sharded_sum(pp)
        else:
            plain(0, 1)
            pp(0, 1)
        return st["plain"], st["pp"]

    dt, wall, logs, clocks = _timed(args, ws, dev, step)
    units_per_step = 2.0 * nS * m
    value = units_per_step * args.steps / dt
    plain_ms = statistics.mean(s1["ms_total"] for s1, _ in logs)
    pp_ms = statistics.mean(s2["ms_total"] for _, s2 in logs)
    ls_ms = statistics.mean(s1["ms_brandes_sk"] for s1, _ in logs)
    sk_ms = statistics.mean(s2["ms_brandes_sk"] for _, s2 in logs)
    ce_ms = statistics.mean(s2["ms_centrality"] for _, s2 in logs)
    launches = int(sum(s1["kernel_launches"] + s2["kernel_launches"] for s1, s2 in logs)) + args.steps
    s_pp = logs[-1][1]
    a, b = bc_plain.cpu().numpy(), bc_pp.cpu().numpy()
    pp_vs_plain = _rel(b, a)
    line_cfg = {"workload": args.workload, "n": n, "m": m, "arcs": A, "S": nS, "directed": g.directed,
                "weighted": g.w is not None,
                "step": "plain Brandes + Brandes++ (Alg. 1) with the planted partition",
                "l2": "flushed before every step (512 MiB write)", "precision": prec,
                "multi_gpu": ("sources sharded across ranks, FP64 NCCL sum all-reduce of bc[n] per result"
                              if ws > 1 else "one GPU")}

    extra = {}
    if ws == 1:
        # the other precision, measured once after one untimed call (its kernels load lazily and its
        # workspace is allocated on first use)
        other = "fp32" if prec == "fp64" else "fp64"
        bc.brandes(G, Sarg, precision=other, ctx=ctx)
        bc.brandes_pp(G, Sarg, part, precision=other, ctx=ctx)
        flush.fill_(1)
        x1, o1 = bc.brandes(G, Sarg, precision=other, stats=True, ctx=ctx)
        flush.fill_(1)
        x2, o2 = bc.brandes_pp(G, Sarg, part, precision=other, stats=True, ctx=ctx)
        ref64 = a if prec == "fp64" else x1.cpu().numpy()
        got32 = x1.cpu().numpy() if prec == "fp64" else a
        got32_pp = x2.cpu().numpy() if prec == "fp64" else b
        fp32 = {"plain_ms": o1["ms_total"] if prec == "fp64" else plain_ms,
                "pp_ms": o2["ms_total"] if prec == "fp64" else pp_ms,
                "plain_fp64_ms": plain_ms if prec == "fp64" else o1["ms_total"],
                "pp_fp64_ms": pp_ms if prec == "fp64" else o2["ms_total"],
                "max_rel_err_fp32_vs_gpu_fp64": {"plain": _rel(got32, ref64), "brandes_pp": _rel(got32_pp, ref64)}}
        fp32["speedup_fp32_over_fp64_plain"] = fp32["plain_fp64_ms"] / fp32["plain_ms"]
        fp32["speedup_fp32_over_fp64_pp"] = fp32["pp_fp64_ms"] / fp32["pp_ms"]
        extra["fp32_delta"] = fp32

        # Brandes++All (Alg. 3): the k^2 ordered pairs of parts, once, outside the timed region
        if args.pp_all and nS == n:
            flush.fill_(1)
            x3, s3 = bc.brandes_pp_all(G, part, precision=prec, stats=True, ctx=ctx)
            extra["brandes_pp_all"] = {
                "teps": nS * m / (s3["ms_total"] / 1e3), "ms": s3["ms_total"], "pairs": s3["skel_edges"],
                "k": s3["k"], "ms_build_sk": s3["ms_build_sk"], "ms_brandes_sk": s3["ms_brandes_sk"],
                "ms_centrality": s3["ms_centrality"], "max_rel_err_vs_plain": _rel(x3.cpu().numpy(), a),
                "kernel_launches": s3["kernel_launches"]}

        # captured plans (CUDA graphs): plain Brandes replays the whole evaluation; the Brandes++
        # plan replays Brandes_SK + Centrality + combine on the skeleton built at plan creation
        if not args.no_graph:
            pl = bc.plan_brandes(G, Sarg, precision=prec, ctx=ctx)
            pp_plan = bc.plan_brandes_pp(G, Sarg, part, precision=prec, ctx=ctx)
            try:
                tpl, tpp, kpl, kpp = [], [], 0, 0
                for _ in range(2):
                    flush.fill_(1)
                    xg, sg1 = pl.launch(stats=True)
                    flush.fill_(1)
                    xq, sg2 = pp_plan.launch(stats=True)
                    tpl.append(sg1["ms_total"])
                    tpp.append(sg2["ms_total"])
                    kpl, kpp = sg1["kernel_launches"], sg2["kernel_launches"]
                extra["cuda_graph"] = {
                    "plain_ms": min(tpl), "pp_per_source_ms": min(tpp),
                    "kernels_per_replay": {"plain": kpl, "brandes_pp": kpp},
                    "max_rel_err_vs_direct": max(_rel(xg.cpu().numpy(), a), _rel(xq.cpu().numpy(), a)),
                    "note": "Brandes++ replay excludes Build_SK (run once at plan creation)"}
            finally:
                pl.close()
                pp_plan.close()

        # launch-shape autotuner on a sample of the sources
        if not args.no_autotune:
            tuned, times = bc.autotune(G, Sarg, precision=prec, ctx=ctx)
            extra["autotune"] = {"tuned": tuned,
                                 "candidates_ms": {f"batch{b}_cluster{c}": t for (b, c), t in times.items()}}

    # rooflines of the three kernels of the step, per launch of this rank's shard of the sources
    hbm, sm_mhz, peak_kind = measured_peaks()
    peak_src = ("MEASURED_PEAKS.json hbm_gbs (measured)" if peak_kind == "measured" else "fallback 6.8 TB/s")
    delta_bytes = 4 if prec == "fp32" else 8
    rooflines = {}
    if not args.no_roofline_model:
        D_avg = _tight_arcs(bc, G, np.linspace(0, n - 1, 32).astype(np.int32), ctx)
        by_plain = model_bytes_per_source(n, A, D_avg, 32, delta_bytes) * my_ns
        rooflines["plain"] = _roof(
            "hbm", by_plain / (ls_ms / 1e3) / 1e9, hbm, "GB/s", "ls_kernel (plain Brandes, forward + backward)",
            profiled_traffic("ls_kernel", args.workload), peak_source=peak_src,
            algorithmic_bytes_per_launch=by_plain, avg_launch_ms=ls_ms, tight_arcs_per_source=D_avg,
            sources_per_launch=my_ns)
        skm = _skeleton_model(bc, g, G, S_order, np.asarray(g.part), ctx)
        if sk_ms > 0:
            by_sk = model_bytes_per_source_skeleton(skm["N"], skm["arcs"], skm["D"], 32, delta_bytes,
                                                    skm["weighted"], skm["mult"]) * my_ns
            rooflines["brandes_sk"] = _roof(
                "hbm", by_sk / (sk_ms / 1e3) / 1e9, hbm, "GB/s",
                "ls_kernel (Brandes_SK on the weighted skeleton, forward + backward, all chunks)",
                profiled_traffic("ls_kernel_skel", args.workload), peak_source=peak_src,
                algorithmic_bytes_per_launch=by_sk, avg_ms=sk_ms, skeleton_nodes=skm["N"],
                skeleton_arcs=skm["arcs"], tight_arcs_per_source=skm["D"], sources_per_launch=my_ns)
        if ce_ms > 0:
            props = torch.cuda.get_device_properties(dev)
            peak_ops = alu_peak_ops(props.multi_processor_count, sm_mhz)
            ops = centrality_ops_per_source(skm["interior_entries"]) * my_ns
            rooflines["centrality"] = _roof(
                "alu", ops / (ce_ms / 1e3) / 1e12, peak_ops / 1e12, "Tops/s",
                "centrality_tiled_kernel (Eq. 13, forward min-plus + backward tight exits)", None,
                peak_source=f"{props.multi_processor_count} SMs x 4 schedulers x 32 lanes x {sm_mhz:.0f} MHz "
                            "(32-bit integer lane operations)",
                algorithmic_ops_per_launch=ops, avg_ms=ce_ms, interior_table_entries=skm["interior_entries"],
                sources_per_launch=my_ns)
    times = {"plain": ls_ms, "brandes_sk": sk_ms, "centrality": ce_ms}
    dominant = max((k for k in rooflines), key=lambda k: times[k], default=None)
    roofline = dict(rooflines[dominant], dominant_of=sorted(rooflines)) if dominant else None

    # end to end: host buffers through the C ABI (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        H = bc.HostCSR.from_device(G)
        part_h = np.ascontiguousarray(g.part, np.int32)
        out1 = torch.empty(n, dtype=torch.float64).pin_memory()
        out2 = torch.empty(n, dtype=torch.float64).pin_memory()

        def e2e_step():
            bc.brandes_host(H, Sarg, precision=prec, ctx=ctx, out=out1, shard=shard)
            bc.brandes_pp_host(H, Sarg, part_h, precision=prec, ctx=ctx, out=out2, shard=shard)
            if ws > 1:      # the partial sums reach the device for the all-reduce and come back
                for o in (out1, out2):
                    t = o.to(dev, non_blocking=True)
                    sharded.sharded_sum(lambda r, R: t)
                    o.copy_(t)

        e2e_step()
        torch.cuda.synchronize()
        ke = max(1, min(args.steps, args.e2e_steps))
        _barrier(ws)
        t0 = time.perf_counter()
        for _ in range(ke):
            flush.fill_(1)
            e2e_step()
        torch.cuda.synchronize()
        te = _max_over_ranks(ws, time.perf_counter() - t0, dev)
        in_bytes = (H.row_ptr.numel() * 8 + H.col.numel() * 4 + (0 if H.w is None else H.w.numel() * 4)
                    + (0 if Sarg is None else 4 * len(Sarg)))
        e2e = {"value": units_per_step * ke / te, "unit": UNIT, "steps": ke,
               "h2d_bytes_per_step": int(2 * in_bytes + 4 * n + (16 * n if ws > 1 else 0)),
               "d2h_bytes_per_step": int(2 * 8 * n + (16 * n if ws > 1 else 0))}

    # CPU oracle on all host cores over a bounded sample of sources; the same sources' partial
    # sums on the GPU (FP64 and FP32-delta) against it
    cpu, err_oracle = None, None
    if pool is not None:
        smp = oracle_sample(pool, args.workload, args.cpu_seconds, m)
        cpu = {"value": smp["value"], "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": smp["sample"]}
        err_oracle = {"sources": smp["ns"]}
        for p in ("fp64", "fp32"):
            got = bc.brandes(G, Sarg, precision=p, halve=False, shard=(0, smp["count"]), ctx=ctx,
                             order_sources=False).cpu().numpy()
            got_pp = bc.brandes_pp(G, Sarg, part, precision=p, halve=False, shard=(0, smp["count"]), ctx=ctx,
                                   order_sources=False).cpu().numpy()
            err_oracle[p] = {"plain": _rel(got, smp["ref_plain"]), "brandes_pp": _rel(got_pp, smp["ref_plain"])}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32-delta+f64",
        "data": "synthetic", "config": line_cfg,
        "plain": {"teps": nS * m / (plain_ms / 1e3), "ms": plain_ms},
        "brandes_pp": {"teps": nS * m / (pp_ms / 1e3), "ms": pp_ms, "ms_build_sk": s_pp["ms_build_sk"],
                       "ms_brandes_sk": s_pp["ms_brandes_sk"], "ms_centrality": s_pp["ms_centrality"],
                       "N": s_pp["skel_nodes"], "M": s_pp["skel_edges"], "k": s_pp["k"], "LCS": s_pp["lcs"],
                       "table_entries": s_pp["table_entries"]},
        "speedup_pp_over_plain": plain_ms / pp_ms,
        "max_rel_err_pp_vs_plain": pp_vs_plain,
        "rel_err_vs_oracle": err_oracle,
        "wall_s": wall,
        "gpu_launches": launches,
        "roofline": roofline,
        "rooflines": rooflines,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
    }
    line.update(extra)
    return line


def _run_batched(args, bc, graphs, ctx, flush, dev, ws, rank):
    """The batch workload: every graph's full betweenness in one launch.  With N ranks each rank
    takes a contiguous share of the graphs (strong scaling; no exchange is needed, each graph's
    result is complete on its rank)."""
    import torch
    from paper_1406_4173_gb300 import api
    prec = args.precision
    g0, g1 = api.shard_bounds(len(graphs), rank, ws)
    mine = graphs[g0:g1]
    units_total = float(sum(g.n * g.m for g in graphs))
    arena = bc.build_arena(mine)
    out = torch.empty(arena.graph.n, dtype=torch.float64, device=dev)
    tuned = {}
    tune = None
    if not args.no_autotune:
        tuned, times = bc.autotune_batched(arena, precision=prec, ctx=ctx)
        tune = {"tuned": tuned, "candidates_ms": {f"batch{b}_cluster{c}": t for (b, c), t in times.items()}}

    def step():
        flush.fill_(1)
        _, st = bc.brandes_batched(arena, precision=prec, out=out, stats=True, ctx=ctx, **tuned)
        return st

    dt, wall, logs, clocks = _timed(args, ws, dev, step)
    value = units_total * args.steps / dt
    ms = statistics.mean(st["ms_total"] for st in logs)
    launches = int(sum(st["kernel_launches"] for st in logs)) + args.steps
    other = "fp32" if prec == "fp64" else "fp64"
    bc.brandes_batched(arena, precision=other, ctx=ctx, **tuned)      # first use: lazy kernel load, workspace
    flush.fill_(1)
    x, so = bc.brandes_batched(arena, precision=other, stats=True, ctx=ctx, **tuned)
    a, b = out.cpu().numpy(), x.cpu().numpy()
    ref64, got32 = (a, b) if prec == "fp64" else (b, a)
    fp32 = {"ms": so["ms_total"] if prec == "fp64" else ms, "fp64_ms": ms if prec == "fp64" else so["ms_total"],
            "max_rel_err_fp32_vs_gpu_fp64": _rel(got32, ref64)}
    # roofline of the batched lockstep launch: per graph, |V_g| sources of the per-source model
    # bytes, with the tight-arc count D_g from the measured tight fraction of sampled graphs
    # (their distances from 4 sources each, on the GPU)
    rng = np.random.default_rng(0)
    fracs = []
    for gi in rng.choice(len(mine), size=min(32, len(mine)), replace=False):
        gg = mine[int(gi)]
        Gs = bc.graph_from_edgelist(gg, ctx)
        D = _tight_arcs(bc, Gs, np.linspace(0, gg.n - 1, 4).astype(np.int32), ctx)
        fracs.append(D / max(1, Gs.num_arcs))
    tight_frac = float(np.mean(fracs))
    delta_bytes = 4 if prec == "fp32" else 8
    bytes_launch = float(sum(g.n * model_bytes_per_source(g.n, 2 * g.m, tight_frac * 2 * g.m, 32, delta_bytes)
                             for g in mine))
    hbm, _, peak_kind = measured_peaks()
    ls_ms = statistics.mean(st["ms_brandes_sk"] for st in logs)
    achieved = bytes_launch / (ls_ms / 1e3) / 1e9
    roofline = _roof("hbm", achieved, hbm, "GB/s", "ls_kernel (batched plain Brandes, forward + backward)", None,
                     peak_source="MEASURED_PEAKS.json hbm_gbs (measured)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s", algorithmic_bytes_per_launch=bytes_launch, avg_launch_ms=ls_ms,
                     tight_arc_fraction=tight_frac)

    # end to end: arena CSR and offsets from pinned host memory, result back, inside the timing
    e2e = None
    if not args.no_e2e:
        H = bc.HostCSR.from_device(arena.graph)
        hout = torch.empty(arena.graph.n, dtype=torch.float64).pin_memory()
        bc.brandes_batched_host(H, arena.node_ptr_host, precision=prec, ctx=ctx, out=hout)
        torch.cuda.synchronize()
        ke = max(1, min(args.steps, args.e2e_steps))
        _barrier(ws)
        t0 = time.perf_counter()
        for _ in range(ke):
            flush.fill_(1)
            bc.brandes_batched_host(H, arena.node_ptr_host, precision=prec, ctx=ctx, out=hout)
        torch.cuda.synchronize()
        te = _max_over_ranks(ws, time.perf_counter() - t0, dev)
        in_bytes = H.row_ptr.numel() * 8 + H.col.numel() * 4 + 8 * len(arena.node_ptr_host)
        e2e = {"value": units_total * ke / te, "unit": UNIT, "steps": ke, "h2d_bytes_per_step": int(in_bytes),
               "d2h_bytes_per_step": int(8 * arena.graph.n)}

    cpu, err_oracle = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        refs, done, rate, cores = batch_oracle_sample(graphs, args.cpu_seconds)
        off = arena.node_ptr_host
        errs = [_rel(a[off[i]:off[i + 1]], refs[i]) for i in range(done)]
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {done} of {len(graphs)} graphs, full betweenness each, "
                         f"{cores} spawned worker processes, one per host core"}
        err_oracle = {"graphs": done, "max_rel_err": max(errs) if errs else None}
    ns = np.array([g.n for g in graphs])
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32-delta+f64", "data": "synthetic",
        "config": {"workload": args.workload, "graphs": len(graphs), "nodes": int(ns.sum()),
                   "n_median": float(np.median(ns)), "n_max": int(ns.max()),
                   "step": "full betweenness of every graph in one launch (plain Brandes)",
                   "units": "sum over graphs of n_g * m_g", "l2": "flushed before every step (512 MiB write)",
                   "precision": prec,
                   "multi_gpu": "graphs split across ranks" if ws > 1 else "one GPU"},
        "plain": {"teps": value, "ms": ms},
        "rel_err_vs_oracle": err_oracle,
        "fp32_delta": fp32,
        "autotune": tune,
        "wall_s": wall, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "clocks": clocks,
    }


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
