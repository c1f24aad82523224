"""The reference arm of bench.py (the oracle on the host cores) prints one JSON line with the
keys of the benchmark contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--ref-L", "64"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["unit"] == d["e2e"]["unit"] == d["cpu_baseline"]["unit"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_cpu_baseline_reports_all_cores_and_one_core():
    sys.path.insert(0, ROOT)
    import bench
    cb = bench.cpu_baseline(sample_L=32, mcs=1, single_L=16, single_mcs=1)
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    one = cb["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == cb["unit"]
    import oracle
    assert oracle.set_threads(cb["cores"]) == cb["cores"]  # the thread count is put back
