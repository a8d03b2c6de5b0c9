"""CPU checks of bench.py's host logic: the traffic model behind the roofline, the rule that
ties a committed DRAM figure to the kernel source it was measured on, and the JSON line of the
reference arm (the CPU oracle), which needs no GPU."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_model_bytes_chunglu_50k():
    """The per-source traffic model on the default workload (n = 50,000, A = 500,000 arcs, 133,029
    tight arcs per source on average): 8.743 MB per source with FP64 dependencies, 8.011 MB with
    FP32, 437.1 GB for the 50,000 sources of one launch."""
    n, A, D = 50_000, 500_000, 133_029.0625
    f64 = bench.model_bytes_per_source(n, A, D, 32, 8)
    f32 = bench.model_bytes_per_source(n, A, D, 32, 4)
    assert f64 / 1e6 == pytest.approx(8.743, abs=5e-4)
    assert f32 / 1e6 == pytest.approx(8.011, abs=5e-4)
    assert f64 * n / 1e9 == pytest.approx(437.13, abs=5e-3)
    # the FP32 saving is 4 bytes per tight arc and per node of the backward pass
    assert f64 - f32 == pytest.approx(4 * (D + n))


def test_model_bytes_terms():
    """Forward plus backward: arcs cost 2 x (4/B + 4) bytes, tight arcs 8 + 8 + delta, nodes
    2 x 8/B + 4 + 8 + delta + 8; B = 1 charges the CSR reads to every source."""
    assert bench.model_bytes_per_source(0, 1, 0, 32, 8) == pytest.approx(2 * (4 / 32 + 4))
    assert bench.model_bytes_per_source(0, 0, 1, 32, 8) == pytest.approx(24)
    assert bench.model_bytes_per_source(1, 0, 0, 32, 8) == pytest.approx(2 * 8 / 32 + 12 + 16)
    assert bench.model_bytes_per_source(0, 1, 0, 1, 8) == pytest.approx(16)


def test_profiled_traffic_follows_kernel_source(monkeypatch):
    """A committed DRAM figure is reported only while the kernel source hash recorded next to it
    matches the current source."""
    p = os.path.join(ROOT, "profiles", "ls_kernel_chunglu_50k.md")
    rec = {}
    for line in open(p).read().splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            rec[k.strip()] = v.strip()
    assert "kernel_source_hash" in rec and "dram_bytes_per_launch" in rec
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["kernel_source_hash"])
    assert bench.profiled_traffic("chunglu_50k") == float(rec["dram_bytes_per_launch"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic("chunglu_50k") is None
    assert bench.profiled_traffic("no_such_workload") is None


def test_kernel_source_hash_is_stable():
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    assert bench.kernel_source_hash() == h


def _run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                          text=True, cwd=ROOT, env=env, timeout=600)


def test_reference_arm_json_line():
    """--impl reference times the CPU oracle and prints one JSON line with the contract's keys."""
    r = _run_bench(["--impl", "reference", "--workload", "planted_2k", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] == "planted_2k"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    """Under a multi-rank launch only rank 0 runs the oracle and prints; the others exit 0."""
    r = _run_bench(["--impl", "reference", "--workload", "planted_2k", "--steps", "1", "--warmup", "0"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
