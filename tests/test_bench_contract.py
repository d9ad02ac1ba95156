"""The benchmark's command-line contract, checked on the CPU.

- `bench.py --impl reference` times the FP64 oracle on a sample of the workload and prints
  one JSON line with the keys the benchmark's consumers read: the metric and unit of the
  GPU arm, `ms_per_step` as the time of the sample that actually ran (the extrapolation is a
  separate field), a `cpu_baseline` describing the run and an `e2e` entry with no host
  transfers.
- Without a GPU the library's own arm fails with a non-zero exit and prints no result: there
  is no CPU fallback behind the benchmark.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--nx", "101", "--nz", "51", "--nt", "200", "--shots", "2"]


def _run(args, timeout=300):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def _json_lines(out):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_complete_line():
    p = _run(["--impl", "reference", "--steps", "2", "--warmup", "1", "--cpu-steps", "8", "--r", "8",
              *SMALL])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _json_lines(p.stdout)
    assert len(lines) == 1
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["unit"] == "shot-gradients/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["sample_steps"] == 8
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # the sample is 8 of 200 steps: the extrapolated shot-gradient time is 25 samples long
    assert abs(d["extrapolated_ms_per_shot_gradient"] / d["ms_per_step"] - 25.0) < 1e-6
    assert abs(d["value"] - 1e3 / d["extrapolated_ms_per_shot_gradient"]) < 1e-9 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_gpu_arm_fails_without_a_gpu():
    p = _run(["--steps", "1", "--warmup", "3", "--no-cpu", *SMALL])
    assert p.returncode != 0
    assert not [d for d in _json_lines(p.stdout) if "value" in d]
