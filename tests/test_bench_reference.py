"""The benchmark's reference arm (the FP64 CPU oracle timed on bounded
samples of the batched workload) runs on the CPU: one JSON line with the
benchmark contract's keys, and nothing from ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra, env=None):
    e = dict(os.environ, OMP_NUM_THREADS="2")
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--problems", "64", *extra], cwd=ROOT, env=e, capture_output=True,
                          text=True, timeout=600)


def test_reference_line_has_the_contract_keys():
    pr = _run("--steps", "2", "--warmup", "1", "--L", "3")
    assert pr.returncode == 0, pr.stderr[-2000:]
    lines = [ln for ln in pr.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "fits/s" and d["higher_is_better"] is True
    assert d["dtype"] == "f64" and d["vs_baseline"] is None
    assert "64 problems" in d["config"]["workload"] and "L=3" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "fits/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # fits per step / time per step
    per_step = int(cb["sample"].split()[0])
    assert abs(d["value"] - per_step * 3 / (d["ms_per_step"] / 1e3)) <= 1e-6 * d["value"]


def test_reference_single_lambda_path():
    pr = _run("--steps", "1", "--warmup", "1", "--L", "1")
    assert pr.returncode == 0, pr.stderr[-2000:]
    d = json.loads([ln for ln in pr.stdout.splitlines() if ln.startswith("{")][0])
    assert d["value"] > 0


def test_reference_other_ranks_print_nothing():
    pr = _run("--steps", "1", "--warmup", "1", "--L", "2",
              env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert pr.returncode == 0, pr.stderr[-2000:]
    assert not [ln for ln in pr.stdout.splitlines() if ln.startswith("{")]


def test_bench_arguments_parse():
    pr = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], cwd=ROOT,
                        capture_output=True, text=True, timeout=300)
    assert pr.returncode == 0, pr.stderr[-2000:]
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--no-variants", "--no-cv",
                 "--no-large", "--no-diff", "--no-serve", "--launch"):
        assert flag in pr.stdout, flag
