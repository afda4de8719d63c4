"""The benchmark's reference arm (the FP64 oracle on the host cores) runs without a GPU and
prints one JSON line with the contract's fields."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    # the driver divides the two arms only when metric, unit and direction are identical
    import importlib.util
    spec = importlib.util.spec_from_file_location("_bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert line["metric"] == bench.METRIC
    assert "whole matrix" in line["cpu_baseline"]["sample"]
    st = line["cpu_baseline"]["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and line["cpu_baseline"]["cpu_model"]
    assert line["unit"] == "GFLOP/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0 and line["n_gpus"] == 1
    assert line["config"]["workload"].startswith("powerlaw-rmat-2^20")
    # the power-law configuration at its full size: 2^20 x 2^20, 2^24 distinct edges, K = 128
    cfg = line["config"]
    assert cfg["m"] == cfg["n"] == 1 << 20 and cfg["nnz"] == 1 << 24 and cfg["K"] == 128
    assert cfg["b_dtype"] == "f32"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
