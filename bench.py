#!/usr/bin/env python
"""Benchmark: betweenness TEPS of GPU plain Brandes and GPU Brandes++ on one GB300.

Workload (default): Chung-Lu graph with planted communities, n = 50,000 in 50 power-law
communities, degree exponent 2.3, mean degree 10 (m = 250,000 undirected edges), 90% of the
edges inside communities, S = V, the planted communities given as the partition; FP64.

One step computes the full target-set betweenness twice through the library's C ABI:
plain Brandes (Eq. 5-7) and Brandes++ (Alg. 1) on the same resident inputs.  TEPS counts
|S| * m source-edge pairs per betweenness computation, so a step is 2 * |S| * m units and
Brandes++/plain is the time ratio.  The L2 cache (129 MB) is flushed before every step by
writing a 512 MiB buffer (the graph itself is only a few MB).

--impl reference times the CPU oracle instead (the paper has no GPU implementation to run):
each step runs the oracle's plain Brandes and Brandes++ from a bounded sample of sources.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BC TEPS (sources x edges / s), Brandes++ vs plain GPU Brandes"
UNIT = "TEPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chunglu_50k")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the cpu_baseline leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip the captured-plan (CUDA graph) measurement")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-shape autotuner")
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

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
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


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("lockstep.cu", "lockstep.cuh", "lockstep_kernel.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1406_4173_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per launch of the lockstep kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"ls_kernel_{workload}.md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def model_bytes_per_source(n, A, D, B=32, delta_bytes=8):
    """Algorithmic bytes of one source of plain Brandes (unit weights), per the traffic model:
    forward = A(4 col + 4 d-probe) + D*8 (parent sigma) + n(8 row_ptr + 4 d + 8 sigma),
    backward = A(4 col + 4 d-probe) + D(8 sigma + delta) + n(8 row_ptr + delta + 8 bc),
    with the col and row_ptr terms shared by the B sources of a batch."""
    fwd = A * (4 / B + 4) + D * 8 + n * (8 / B + 4 + 8)
    bwd = A * (4 / B + 4) + D * (8 + delta_bytes) + n * (8 / B + delta_bytes + 8)
    return fwd + bwd


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- cpu baseline (oracle)
def oracle_sample(g, S_order, part, seconds, with_pp=True):
    """Oracle plain Brandes (+ Brandes++) from the first `ns` sources of S_order (targets = all
    of S_order), ns = |S| // count sized to the time budget, so that GPU shard 0 of `count`
    covers the same sources.  Returns (ns, count, t_plain, t_pp, unhalved plain partial
    betweenness of those sources)."""
    import oracle
    oracle.build()
    S = np.ascontiguousarray(S_order, np.int32)
    t0 = time.perf_counter()
    oracle.brandes(g, S, nsrc=8)
    per = (time.perf_counter() - t0) / 8
    if with_pp:
        t0 = time.perf_counter()
        oracle.brandes_pp(g, S, part, nsrc=8)
        per += (time.perf_counter() - t0) / 8
    want = int(max(1, min(len(S), seconds / max(per, 1e-6))))
    count = max(1, len(S) // want)
    ns = len(S) // count                  # shard 0 of `count` covers positions [0, ns)
    t0 = time.perf_counter()
    part_bc, _ = oracle.brandes(g, S, nsrc=ns, halve=False)
    t1 = time.perf_counter()
    if with_pp:
        oracle.brandes_pp(g, S, part, nsrc=ns)
    t2 = time.perf_counter()
    return ns, count, t1 - t0, t2 - t1, part_bc


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1406_4173_gb300 import gen
    import oracle
    oracle.build()
    g, S = gen.workload(args.workload)
    if isinstance(g, list):
        graphs = g
        per = []

        def step():
            t0 = time.perf_counter()
            u = 0.0
            for gi in graphs[:64]:
                oracle.brandes(gi)
                u += gi.n * gi.m
            per.append(u)
            return time.perf_counter() - t0

        for _ in range(args.warmup):
            step()
        per.clear()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        dt = time.perf_counter() - t0
        val = sum(per) / dt
        sample = "first 64 graphs per step, full betweenness each"
        cfg = {"workload": args.workload, "graphs_per_step": 64}
    else:
        Sall = np.arange(g.n, dtype=np.int32) if S is None else np.asarray(S, np.int32)
        t0 = time.perf_counter()
        oracle.brandes(g, Sall, nsrc=4)
        oracle.brandes_pp(g, Sall, g.part, nsrc=4)
        per_src = (time.perf_counter() - t0) / 4
        ns = int(max(4, min(len(Sall), 4.0 / max(per_src, 1e-6))))

        def step():
            oracle.brandes(g, Sall, nsrc=ns)
            oracle.brandes_pp(g, Sall, g.part, nsrc=ns)

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        dt = time.perf_counter() - t0
        val = 2.0 * ns * g.m * args.steps / dt
        sample = f"first {ns} of {len(Sall)} sources per step (targets = S), plain + Brandes++"
        cfg = {"workload": args.workload, "n": g.n, "m": g.m, "S": len(Sall), "sample_sources_per_step": ns}
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0))) if a.size else 0.0


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
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = bc.default_context()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    g, S = gen.workload(args.workload)
    if isinstance(g, list):
        line = _run_batched(args, bc, g, ctx, flush, dev, ws, rank)
    else:
        line = _run_single(args, bc, gen, g, S, ctx, flush, dev, ws, rank)
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


def _run_single(args, bc, gen, g, S, ctx, flush, dev, ws, rank):
    import torch
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

    def step():
        flush.fill_(1)
        _, s1 = bc.brandes(G, Sarg, precision=prec, out=bc_plain, stats=True, ctx=ctx)
        _, s2 = bc.brandes_pp(G, Sarg, part, precision=prec, out=bc_pp, stats=True, ctx=ctx)
        return s1, s2

    dt, wall, logs, clocks = _timed(args, ws, dev, step)
    units_per_step = 2.0 * nS * m
    value = units_per_step * args.steps * ws / dt
    plain_ms = statistics.mean(s1["ms_total"] for s1, _ in logs)
    pp_ms = statistics.mean(s2["ms_total"] for _, s2 in logs)
    ls_ms = statistics.mean(s1["ms_brandes_sk"] for s1, _ in logs)
    launches = int(sum(s1["kernel_launches"] + s2["kernel_launches"] for s1, s2 in logs)) + args.steps
    s_pp = logs[-1][1]
    a, b = bc_plain.cpu().numpy(), bc_pp.cpu().numpy()
    pp_vs_plain = _rel(b, a)

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
    fp32 = {"plain_ms": o1["ms_total"] if prec == "fp64" else plain_ms,
            "pp_ms": o2["ms_total"] if prec == "fp64" else pp_ms,
            "plain_fp64_ms": plain_ms if prec == "fp64" else o1["ms_total"],
            "max_rel_err_fp32_vs_fp64": _rel(got32, ref64)}
    fp32["speedup_fp32_over_fp64_plain"] = fp32["plain_fp64_ms"] / fp32["plain_ms"]

    # Brandes++All (Alg. 3): the k^2 ordered pairs of parts, once, outside the timed region
    pp_all = None
    if args.pp_all and nS == n:
        flush.fill_(1)
        x3, s3 = bc.brandes_pp_all(G, part, precision=prec, stats=True, ctx=ctx)
        pp_all = {"teps": nS * m / (s3["ms_total"] / 1e3), "ms": s3["ms_total"], "pairs": s3["skel_edges"],
                  "k": s3["k"], "ms_build_sk": s3["ms_build_sk"], "ms_brandes_sk": s3["ms_brandes_sk"],
                  "ms_centrality": s3["ms_centrality"], "max_rel_err_vs_plain": _rel(x3.cpu().numpy(), a),
                  "kernel_launches": s3["kernel_launches"]}

    # captured plans (CUDA graphs): plain Brandes replays the whole evaluation; the Brandes++
    # plan replays Brandes_SK + Centrality + combine on the skeleton built at plan creation
    graph = None
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
            graph = {"plain_ms": min(tpl), "pp_per_source_ms": min(tpp),
                     "kernels_per_replay": {"plain": kpl, "brandes_pp": kpp},
                     "max_rel_err_vs_direct": max(_rel(xg.cpu().numpy(), a), _rel(xq.cpu().numpy(), a)),
                     "note": "Brandes++ replay excludes Build_SK (run once at plan creation)"}
        finally:
            pl.close()
            pp_plan.close()

    # launch-shape autotuner on a sample of the sources
    tune = None
    if not args.no_autotune:
        tuned, times = bc.autotune(G, Sarg, precision=prec, ctx=ctx)
        tune = {"tuned": tuned, "candidates_ms": {f"batch{b}_cluster{c}": t for (b, c), t in times.items()}}

    # roofline of the dominant kernel (lockstep forward+backward of plain Brandes)
    sample = np.linspace(0, n - 1, 32).astype(np.int32)
    dist_s, _ = bc.sssp(G, sample, allow_overflow=True)
    dist_s = dist_s.cpu().numpy().astype(np.int64)
    rp = G.row_ptr.cpu().numpy()
    col = G.col.cpu().numpy()
    wts = None if G.w is None else G.w.cpu().numpy().astype(np.int64)
    tails = np.repeat(np.arange(n), np.diff(rp))
    tight = []
    for i in range(len(sample)):
        dd = dist_s[i]
        ok = (dd[tails] < np.iinfo(np.int32).max) & (dd[col] == dd[tails] + (1 if wts is None else wts))
        tight.append(int(ok.sum()))
    D_avg = float(np.mean(tight))
    delta_bytes = 4 if prec == "fp32" else 8
    bytes_launch = model_bytes_per_source(n, A, D_avg, 32, delta_bytes) * nS
    peak, peak_kind = measured_peak_hbm()
    achieved = bytes_launch / (ls_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(args.workload), "kernel": "ls_kernel (plain Brandes, forward + backward)",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "algorithmic_bytes_per_launch": bytes_launch,
                "avg_launch_ms": ls_ms, "tight_arcs_per_source": D_avg}

    # end to end: host buffers through the C ABI (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        H = bc.HostCSR.from_device(G)
        part_h = np.ascontiguousarray(g.part, np.int32)
        out1 = torch.empty(n, dtype=torch.float64).pin_memory()
        out2 = torch.empty(n, dtype=torch.float64).pin_memory()
        bc.brandes_host(H, Sarg, precision=prec, ctx=ctx, out=out1)
        torch.cuda.synchronize()
        _barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1)
            bc.brandes_host(H, Sarg, precision=prec, ctx=ctx, out=out1)
            bc.brandes_pp_host(H, Sarg, part_h, precision=prec, ctx=ctx, out=out2)
        torch.cuda.synchronize()
        te = _max_over_ranks(ws, time.perf_counter() - t0, dev)
        in_bytes = (H.row_ptr.numel() * 8 + H.col.numel() * 4 + (0 if H.w is None else H.w.numel() * 4)
                    + (0 if Sarg is None else 4 * len(Sarg)))
        e2e = {"value": units_per_step * args.steps * ws / te, "unit": UNIT,
               "h2d_bytes_per_step": int(2 * in_bytes + 4 * n), "d2h_bytes_per_step": int(2 * 8 * n)}

    # CPU oracle on a bounded sample of sources; the same sources' partial sums on the GPU
    cpu, err_oracle = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ns_c, count, tp, tpp, ref_part = oracle_sample(g, S_order, g.part, args.cpu_seconds)
        cpu = {"value": 2.0 * ns_c * m / (tp + tpp), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {ns_c} of {nS} sources (targets = S), oracle plain Brandes + Brandes++, "
                         f"{tp:.1f} s + {tpp:.1f} s"}
        got = bc.brandes(G, Sarg, precision=prec, halve=False, shard=(0, count), ctx=ctx,
                         order_sources=False).cpu().numpy()
        err_oracle = {"sources": ns_c, "max_rel_err_plain": _rel(got, ref_part)}

    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32-delta+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "m": m, "arcs": A, "S": nS, "directed": g.directed,
                   "weighted": g.w is not None,
                   "step": "plain Brandes + Brandes++ (Alg. 1) with the planted partition",
                   "l2": "flushed before every step (512 MiB write)", "precision": prec,
                   "multi_gpu": "independent replicas (weak scaling)"},
        "plain": {"teps": nS * m / (plain_ms / 1e3), "ms": plain_ms},
        "brandes_pp": {"teps": nS * m / (pp_ms / 1e3), "ms": pp_ms, "ms_build_sk": s_pp["ms_build_sk"],
                       "ms_brandes_sk": s_pp["ms_brandes_sk"], "ms_centrality": s_pp["ms_centrality"],
                       "N": s_pp["skel_nodes"], "M": s_pp["skel_edges"], "k": s_pp["k"], "LCS": s_pp["lcs"],
                       "table_entries": s_pp["table_entries"]},
        "speedup_pp_over_plain": plain_ms / pp_ms,
        "max_rel_err_pp_vs_plain": pp_vs_plain,
        "rel_err_vs_oracle": err_oracle,
        "fp32_delta": fp32,
        "brandes_pp_all": pp_all,
        "cuda_graph": graph,
        "autotune": tune,
        "wall_s": wall,
        "gpu_launches": launches,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
    }


def _run_batched(args, bc, graphs, ctx, flush, dev, ws, rank):
    import torch
    prec = args.precision
    arena = bc.build_arena(graphs)
    units_per_step = float(sum(g.n * g.m for g in graphs))
    out = torch.empty(arena.graph.n, dtype=torch.float64, device=dev)

    def step():
        flush.fill_(1)
        _, st = bc.brandes_batched(arena, precision=prec, out=out, stats=True, ctx=ctx)
        return st

    dt, wall, logs, clocks = _timed(args, ws, dev, step)
    value = units_per_step * args.steps * ws / dt
    ms = statistics.mean(st["ms_total"] for st in logs)
    launches = int(sum(st["kernel_launches"] for st in logs)) + args.steps
    other = "fp32" if prec == "fp64" else "fp64"
    bc.brandes_batched(arena, precision=other, ctx=ctx)      # first use: lazy kernel load, workspace
    flush.fill_(1)
    x, so = bc.brandes_batched(arena, precision=other, stats=True, ctx=ctx)
    a, b = out.cpu().numpy(), x.cpu().numpy()
    ref64, got32 = (a, b) if prec == "fp64" else (b, a)
    fp32 = {"ms": so["ms_total"] if prec == "fp64" else ms, "fp64_ms": ms if prec == "fp64" else so["ms_total"],
            "max_rel_err_fp32_vs_fp64": _rel(got32, ref64)}
    # roofline of the batched lockstep launch: per graph, |V_g| sources of the per-source model
    # bytes, with the tight-arc count D_g from the measured tight fraction of sampled graphs
    # (their distances from 4 sources each, on the GPU)
    rng = np.random.default_rng(0)
    fracs = []
    for gi in rng.choice(len(graphs), size=min(32, len(graphs)), replace=False):
        gg = graphs[int(gi)]
        Gs = bc.graph_from_edgelist(gg, ctx)
        srcs = np.linspace(0, gg.n - 1, 4).astype(np.int32)
        dist_s, _ = bc.sssp(Gs, srcs, ctx=ctx, allow_overflow=True)
        dist_s = dist_s.cpu().numpy().astype(np.int64)
        rp, col = Gs.row_ptr.cpu().numpy(), Gs.col.cpu().numpy()
        tails = np.repeat(np.arange(gg.n), np.diff(rp))
        for i in range(len(srcs)):
            dd = dist_s[i]
            ok = (dd[tails] < np.iinfo(np.int32).max) & (dd[col] == dd[tails] + 1)
            fracs.append(ok.sum() / max(1, len(col)))
    tight_frac = float(np.mean(fracs))
    delta_bytes = 4 if prec == "fp32" else 8
    bytes_launch = float(sum(g.n * model_bytes_per_source(g.n, 2 * g.m, tight_frac * 2 * g.m, 32, delta_bytes)
                             for g in graphs))
    peak, peak_kind = measured_peak_hbm()
    ls_ms = statistics.mean(st["ms_brandes_sk"] for st in logs)
    achieved = bytes_launch / (ls_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "ls_kernel (batched plain Brandes, forward + backward)",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": ls_ms,
                "tight_arc_fraction": tight_frac}

    # end to end: arena CSR and offsets from pinned host memory, result back, inside the timing
    e2e = None
    if not args.no_e2e:
        H = bc.HostCSR.from_device(arena.graph)
        hout = torch.empty(arena.graph.n, dtype=torch.float64).pin_memory()
        bc.brandes_batched_host(H, arena.node_ptr_host, precision=prec, ctx=ctx, out=hout)
        torch.cuda.synchronize()
        _barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1)
            bc.brandes_batched_host(H, arena.node_ptr_host, precision=prec, ctx=ctx, out=hout)
        torch.cuda.synchronize()
        te = _max_over_ranks(ws, time.perf_counter() - t0, dev)
        in_bytes = H.row_ptr.numel() * 8 + H.col.numel() * 4 + 8 * len(arena.node_ptr_host)
        e2e = {"value": units_per_step * args.steps * ws / te, "unit": UNIT, "h2d_bytes_per_step": int(in_bytes),
               "d2h_bytes_per_step": int(8 * arena.graph.n)}

    cpu, err_oracle = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        errs, done, u = [], 0, 0.0
        off = arena.node_ptr_host
        for i, gi in enumerate(graphs):
            ref, _ = oracle.brandes(gi)
            errs.append(_rel(a[off[i]:off[i + 1]], ref))
            done += 1
            u += gi.n * gi.m
            if time.perf_counter() - t0 > args.cpu_seconds:
                break
        tc = time.perf_counter() - t0
        cpu = {"value": u / tc, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {done} of {len(graphs)} graphs, full betweenness each"}
        err_oracle = {"graphs": done, "max_rel_err": max(errs)}
    ns = np.array([g.n for g in graphs])
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32-delta+f64", "data": "synthetic",
        "config": {"workload": args.workload, "graphs": len(graphs), "nodes": int(ns.sum()),
                   "n_median": float(np.median(ns)), "n_max": int(ns.max()),
                   "step": "full betweenness of every graph in one launch (plain Brandes)",
                   "units": "sum over graphs of n_g * m_g", "l2": "flushed before every step (512 MiB write)",
                   "precision": prec},
        "plain": {"teps": value / ws, "ms": ms},
        "rel_err_vs_oracle": err_oracle,
        "fp32_delta": fp32,
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
