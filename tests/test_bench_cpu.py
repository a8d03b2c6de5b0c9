"""CPU checks of bench.py's host logic: the traffic and operation models behind the rooflines,
the rule that ties a committed DRAM figure to the kernel source it was measured on, and the JSON
line of the reference arm (the CPU oracle on all host cores), which needs no GPU."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_model_bytes_chunglu_50k():
    """The per-source traffic model on `chunglu_50k` (n = 50,000, A = 500,000 arcs, 133,029
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


def test_model_bytes_skeleton_terms():
    """Brandes_SK adds, per arc and pass, 4 bytes of weight and 8 of multiplicity shared by the
    batch's B sources; without weights or multiplicities it is the plain model."""
    base = bench.model_bytes_per_source(10, 100, 30, 32, 8)
    assert bench.model_bytes_per_source_skeleton(10, 100, 30, 32, 8, False, False) == pytest.approx(base)
    assert bench.model_bytes_per_source_skeleton(10, 100, 30, 32, 8, True, False) == pytest.approx(
        base + 100 * 2 * 4 / 32)
    assert bench.model_bytes_per_source_skeleton(10, 100, 30, 32, 8, True, True) == pytest.approx(
        base + 100 * 2 * 12 / 32)


def test_centrality_ops_and_alu_peak():
    """Centrality: 4 integer operations per (frontier, non-frontier node) entry and source; the
    ALU peak is SMs x 4 schedulers x 32 lanes x clock (GB300: 152 SMs at 2,070 MHz = 40.3 T/s)."""
    assert bench.centrality_ops_per_source(1000) == 4000
    assert bench.alu_peak_ops(152, 2070.0) == pytest.approx(4.0274e13, rel=1e-4)


def test_profiled_traffic_follows_kernel_source(monkeypatch, tmp_path):
    """A committed DRAM figure (profiles/<kernel>_<workload>.json) is reported only while the
    kernel source hash recorded with it matches the current source."""
    (tmp_path / "profiles").mkdir()
    rec = {"kernel_source_hash": "abcdef0123456789", "dram_bytes_per_launch": 123456789.0}
    (tmp_path / "profiles" / "ls_kernel_w.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["kernel_source_hash"])
    assert bench.profiled_traffic("ls_kernel", "w") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic("ls_kernel", "w") is None
    assert bench.profiled_traffic("ls_kernel", "no_such_workload") is None


def test_committed_traffic_records_are_well_formed():
    pdir = os.path.join(ROOT, "profiles")
    for f in os.listdir(pdir):
        if f.endswith(".json"):
            rec = json.load(open(os.path.join(pdir, f)))
            assert len(rec["kernel_source_hash"]) == 16 and float(rec["dram_bytes_per_launch"]) > 0, f


def _fake_smi(tmp_path, lines, period=0.05):
    """An nvidia-smi stand-in on PATH that prints the given CSV lines in a loop."""
    script = tmp_path / "nvidia-smi"
    body = "".join(f'  echo "{l}"; sleep {period}\n' for l in lines)
    script.write_text("#!/bin/bash\nwhile true; do\n" + body + "done\n")
    script.chmod(0o755)
    return str(tmp_path)


def test_clock_sampler_waits_for_first_sample(monkeypatch, tmp_path):
    """The sampler starts nvidia-smi and returns only after its first sample (its start-up must
    not overlap the timed steps); the median SM clock and the active throttle reasons are read
    from the samples taken after that."""
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, [ok, capped, ok]) + os.pathsep + os.environ["PATH"])
    c = bench.Clocks(0)
    c.start()
    assert c.first >= 1 and len(c.lines) >= 1
    import time
    time.sleep(0.4)
    r = c.stop()
    assert r["sm_max_mhz"] == 2070.0
    assert r["sm_mhz"] in (2070.0, 1980.0)
    assert r["reasons"] == ["sw_power_cap"]
    assert r["samples"] >= 2


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    """No nvidia-smi on PATH: no clock record, and no error."""
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.Clocks(0)
    c.start()
    assert c.stop() is None


def test_batch_oracle_sample_on_all_cores():
    """The batch workload's CPU baseline: a spawned pool over the graphs in order gives the same
    per-graph results as the oracle called directly, and reports the host's core count."""
    import numpy as np
    import oracle
    from paper_1406_4173_gb300 import gen
    graphs = [gen.erdos_renyi(40 + 7 * i, 0.1, seed=i) for i in range(12)]
    refs, done, rate, cores = bench.batch_oracle_sample(graphs, seconds=0.0, chunk=2)
    assert cores == (os.cpu_count() or 1)
    assert done == min(len(graphs), 2 * cores) and rate > 0
    for gi, r in zip(graphs[:done], refs):
        np.testing.assert_array_equal(r, oracle.brandes(gi)[0])


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
    assert d["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    """Under a multi-rank launch only rank 0 runs the oracle and prints; the others exit 0."""
    r = _run_bench(["--impl", "reference", "--workload", "planted_2k", "--steps", "1", "--warmup", "0"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
