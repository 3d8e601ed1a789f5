"""bench.py's output contract, run at a small scale on the GPU: one JSON line
with the keys the benchmark promises (metric, throughput, roofline, CPU
baseline, end-to-end figure, launch count, clocks), and the batch-only
profiling mode."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=900):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


SMALL = ["--scale", "18", "--steps", "3", "--warmup", "3", "--no-served", "--no-side-graphs",
         "--batch-graphs", "48", "--batch-reps", "3", "--edge-list-steps", "2", "--symmetric-steps", "2",
         "--layout-steps", "2", "--e2e-steps", "1", "--cpu-seconds", "0.5"]


def test_bench_line_carries_the_contract_keys():
    d = run_bench(*SMALL)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "rmat18_ef16"
    rf = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert rf["bound"] == "hbm" and 0 < rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert rf["traffic"] is None          # the committed capture is for scale 27 only
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] == 4 * d["config"]["n"]
    assert d["gpu_launches"] == 2 * d["steps"]           # prepare + sweep per step
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    b = d["batched"]
    assert b["graphs"] == 48 and b["p50_ms"] > 0 and b["roofline"]["frac"] > 0
    assert d["edge_list"]["gedges_s"] > 0


def test_batched_only_profiling_mode():
    d = run_bench("--batched-only", "--batch-graphs", "48", "--batch-opts", "2048,8,0,1,0",
                  "--batch-reps", "2")
    b = d["batched"]
    assert b["tuned"]["grain"] == 2048 and b["tuned"]["searched"] == "fixed by --batch-opts"
    assert b["p50_ms"] > 0 and b["roofline"]["traffic"] is None
    assert "plain_p50_ms" not in b           # the one-call-per-graph arm is skipped
