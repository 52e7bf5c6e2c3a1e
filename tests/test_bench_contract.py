"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU: its one JSON line carries the keys the benchmark contract
asks for, with the GPU arm's config."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_complete_line():
    import time
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["grid"] == 512 and "workload" in d["config"]
    # the line reports what this run measured: its K timed steps fit in the
    # wall time of the whole command, and each step is the stated sample
    assert d["steps"] * d["ms_per_step"] / 1e3 < wall
    assert d["value"] == pytest.approx(d["sample"]["cells_per_step"] / (d["ms_per_step"] / 1e3), rel=1e-9)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_bench_rejects_too_few_warmup_steps():
    r = subprocess.run([sys.executable, "bench.py", "--warmup", "2"], cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode != 0 and "warmup" in r.stderr


def test_ncu_records_are_used_only_for_the_sources_they_were_taken_from():
    """The DRAM-traffic and flop records under profiles/ carry the hash of
    the substep kernel's sources they were captured from: the bench line
    reports them while the hash matches and null once the kernel changed."""
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_source_hash()
    for name, get in (("substep_traffic.json", lambda: bench.ncu_traffic(512, "f32")),
                      ("substep_flops.json", lambda: bench.ncu_flops("f32"))):
        with open(os.path.join(ROOT, "profiles", name)) as f:
            rec = json.load(f)
        assert rec["source_hash"]
        if rec["source_hash"] == h:
            assert get() is not None
        else:
            assert get() is None
