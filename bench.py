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
    for f in ("lockstep.cu", "lockstep.cuh", "common.cuh"):
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
def oracle_sample_rate(g, part, seconds):
    """Oracle plain Brandes + Brandes++ from a bounded sample of sources (targets = V)."""
    import oracle
    oracle.build()
    S = np.arange(g.n, dtype=np.int32)
    # calibrate on 8 sources, then size the sample to the budget
    t0 = time.perf_counter()
    oracle.brandes(g, None, nsrc=8)
    oracle.brandes_pp(g, S, part, nsrc=8)
    per = (time.perf_counter() - t0) / 8
    ns = int(max(8, min(g.n, seconds / max(per, 1e-6))))
    t0 = time.perf_counter()
    oracle.brandes(g, None, nsrc=ns)
    t1 = time.perf_counter()
    oracle.brandes_pp(g, S, part, nsrc=ns)
    t2 = time.perf_counter()
    return ns, t1 - t0, t2 - t1


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1406_4173_gb300 import gen
    g, S = gen.workload(args.workload)
    import oracle
    oracle.build()
    Sall = np.arange(g.n, dtype=np.int32) if S is None else S
    # size each step to ~4 s of oracle work
    t0 = time.perf_counter()
    oracle.brandes(g, Sall, nsrc=4)
    oracle.brandes_pp(g, Sall, g.part, nsrc=4)
    per = (time.perf_counter() - t0) / 4
    ns = int(max(4, min(len(Sall), 4.0 / max(per, 1e-6))))

    def step():
        oracle.brandes(g, Sall, nsrc=ns)
        oracle.brandes_pp(g, Sall, g.part, nsrc=ns)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    units = 2.0 * ns * g.m * args.steps
    val = units / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": g.n, "m": g.m, "S": len(Sall),
                   "sample_sources_per_step": ns},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{ns} of {len(Sall)} sources per step (targets = S), plain + Brandes++"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- ours
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

    g, S = gen.workload(args.workload)
    if isinstance(g, list):
        raise SystemExit("bench: use a single-graph workload")
    n, m = g.n, g.m
    nS = n if S is None else len(S)
    Sarg = None if S is None or len(S) == n else S
    part = torch.as_tensor(g.part, device=dev)
    G = bc.graph_from_edgelist(g)
    A = G.num_arcs
    bc_plain = torch.empty(n, dtype=torch.float64, device=dev)
    bc_pp = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ctx = bc.default_context()

    stats_log = []

    def step():
        flush.fill_(1)
        _, s1 = bc.brandes(G, Sarg, precision=args.precision, out=bc_plain, stats=True, ctx=ctx)
        _, s2 = bc.brandes_pp(G, Sarg, part, precision=args.precision, out=bc_pp, stats=True, ctx=ctx)
        stats_log.append((s1, s2))

    for _ in range(args.warmup):
        step()
    stats_log.clear()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    clk = Clocks(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier()
    clocks = clk.stop()
    dt = e0.elapsed_time(e1) / 1e3
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([dt], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    units_per_step = 2.0 * nS * m
    value = units_per_step * args.steps * ws / dt

    plain_ms = [s1["ms_total"] for s1, _ in stats_log]
    pp_ms = [s2["ms_total"] for _, s2 in stats_log]
    ls_ms = [s1["ms_brandes_sk"] for s1, _ in stats_log]
    launches = int(sum(s1["kernel_launches"] + s2["kernel_launches"] for s1, s2 in stats_log)) + args.steps
    s_pp = stats_log[-1][1]

    # exactness at full size: Brandes++ must equal plain Brandes (both FP64 on the GPU)
    a, b = bc_plain.cpu().numpy(), bc_pp.cpu().numpy()
    pp_vs_plain = float(np.max(np.abs(a - b) / np.maximum(np.abs(a), 1.0)))

    # roofline of the dominant kernel (lockstep forward+backward of plain Brandes)
    sample = np.linspace(0, n - 1, 32).astype(np.int32)
    dist_s, _ = bc.sssp(G, sample, allow_overflow=True)
    dist_s = dist_s.cpu().numpy().astype(np.int64)
    rp = G.row_ptr.cpu().numpy()
    col = G.col.cpu().numpy()
    tails = np.repeat(np.arange(n), np.diff(rp))
    tight = []
    for i in range(len(sample)):
        d = dist_s[i]
        ok = (d[tails] < np.iinfo(np.int32).max) & (d[col] == d[tails] + 1)
        tight.append(int(ok.sum()))
    D_avg = float(np.mean(tight))
    delta_bytes = 4 if args.precision == "fp32" else 8
    bytes_launch = model_bytes_per_source(n, A, D_avg, 32, delta_bytes) * nS
    ls_avg_s = statistics.mean(ls_ms) / 1e3
    peak, peak_kind = measured_peak_hbm()
    achieved = bytes_launch / ls_avg_s / 1e9
    traffic = profiled_traffic(args.workload)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "ls_kernel (plain Brandes, forward + backward)",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "algorithmic_bytes_per_launch": bytes_launch,
                "avg_launch_ms": ls_avg_s * 1e3, "tight_arcs_per_source": D_avg}

    # end to end: host buffers through the C ABI (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        H = bc.HostCSR.from_device(G)
        part_h = np.ascontiguousarray(g.part, np.int32)
        out1 = torch.empty(n, dtype=torch.float64).pin_memory()
        out2 = torch.empty(n, dtype=torch.float64).pin_memory()
        bc.brandes_host(H, Sarg, precision=args.precision, ctx=ctx, out=out1)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1)
            bc.brandes_host(H, Sarg, precision=args.precision, ctx=ctx, out=out1)
            bc.brandes_pp_host(H, Sarg, part_h, precision=args.precision, ctx=ctx, out=out2)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        in_bytes = (H.row_ptr.numel() * 8 + H.col.numel() * 4 + (0 if H.w is None else H.w.numel() * 4)
                    + (0 if Sarg is None else 4 * len(Sarg)))
        e2e = {"value": units_per_step * args.steps * ws / te, "unit": UNIT,
               "h2d_bytes_per_step": int(2 * in_bytes + 4 * n), "d2h_bytes_per_step": int(2 * 8 * n)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ns_c, tp, tpp = oracle_sample_rate(g, g.part, args.cpu_seconds)
        cpu = {"value": 2.0 * ns_c * m / (tp + tpp), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{ns_c} of {nS} sources (targets = S), oracle plain Brandes + Brandes++, "
                         f"{tp:.1f} s + {tpp:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32-delta+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "m": m, "arcs": A, "S": nS,
                       "step": "plain Brandes + Brandes++ (Alg. 1), S = V, planted partition",
                       "l2": "flushed before every step (512 MiB write)",
                       "precision": args.precision, "multi_gpu": "independent replicas (weak scaling)"},
            "plain": {"teps": nS * m / (statistics.mean(plain_ms) / 1e3), "ms": statistics.mean(plain_ms)},
            "brandes_pp": {"teps": nS * m / (statistics.mean(pp_ms) / 1e3), "ms": statistics.mean(pp_ms),
                           "ms_build_sk": s_pp["ms_build_sk"], "ms_brandes_sk": s_pp["ms_brandes_sk"],
                           "ms_centrality": s_pp["ms_centrality"], "N": s_pp["skel_nodes"],
                           "M": s_pp["skel_edges"], "k": s_pp["k"], "LCS": s_pp["lcs"]},
            "speedup_pp_over_plain": statistics.mean(plain_ms) / statistics.mean(pp_ms),
            "max_rel_err_pp_vs_plain": pp_vs_plain,
            "wall_s": wall,
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
