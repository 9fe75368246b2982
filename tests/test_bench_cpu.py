"""bench.py's reference arm (the oracle on the host cores) runs without a GPU:
its JSON line carries the keys of the benchmark contract, with the oracle
named as the baseline kind and the workload named from the sizes it ran."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--boundary-nodes", "64", "--count", "8"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["higher_is_better"] is False and line["unit"] == "s"
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["config"]["workload"].startswith("8 ellipses, unbounded, n=64 (512 unknowns)")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert cb["pair_evals_per_s"] > 0 and "OpenMP" in cb["pair_sample"]
    assert cb["measured"]["N"] == 512 and cb["measured"]["lu_solve_s"] > 0
    # the GPU arm's config dict for the same arguments (same_config)
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(precision="fmm")
    assert line["config"] == bench.bench_config(args, 512, 8, 64, 1)
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
