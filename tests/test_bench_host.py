"""The benchmark's host-side contract on CPU: the reference arm's JSON line
(the oracle timed on the host) and the compiled-CPU context."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--n", "256"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "impl", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 1 and line["warmup"] == 0
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "256^2" in line["config"]["workload"]


def test_compiled_cpu_context_reports_every_tile():
    sys.path.insert(0, ROOT)
    import bench
    out = bench.compiled_cpu_context(64, seconds=0.01, rows=(8, 16))
    assert out["untiled"]["value"] > 0 and set(out["tiled"]) == {"8", "16"}
    assert out["best_tile_rows"] in (8, 16) and out["speedup_tiled_vs_untiled"] > 0
