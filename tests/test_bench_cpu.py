"""CPU checks of bench.py's reference arm (the float64 oracle timed on the host
cores) and of its command-line contract: one JSON line with the keys the
GPU arm prints, `unavailable` lines where the oracle has nothing to time, and
the minimum warm-up. The GPU arm itself runs only on a GB300."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    return r


def _last_json(r):
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert lines, r.stdout[-2000:]
    return [json.loads(ln) for ln in lines]


def _check_reference_line(d, unit):
    assert d["impl"] == "reference"
    assert d["unit"] == unit and d["higher_is_better"] is True and d["value"] > 0
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == unit
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_default_workload():
    (d,) = _last_json(_bench("--impl", "reference", "--steps", "1", "--warmup", "3"))
    _check_reference_line(d, "sweeps/s")
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["N"] == 1_000_000 and d["config"]["M"] == 1_000_000 and d["config"]["d"] == 64
    # the oracle does 2 N M pair evaluations per sweep
    assert d["gpair_evals_per_s"] == pytest.approx(d["value"] * 2e12 / 1e9, rel=1e-9)


def test_reference_arm_times_the_sigma_override():
    """--sigma changes the fused workload's exponent range (0.01 makes it wide,
    the running-maximum half-sweep); the reference arm times that same market."""
    (d,) = _last_json(_bench("--impl", "reference", "--sigma", "0.01", "--steps", "1", "--warmup", "3"))
    _check_reference_line(d, "sweeps/s")
    assert d["config"]["sigma"] == 0.01 and "sigma=0.01" in d["config"]["workload"]
    assert d["config"]["N"] == 1_000_000 and d["config"]["d"] == 64


def test_reference_arm_batched_workload():
    (d,) = _last_json(_bench("--impl", "reference", "--workload", "batched", "--steps", "1", "--warmup", "3"))
    _check_reference_line(d, "Gpair-evals/s")
    assert d["config"]["markets"] == 512


@pytest.mark.parametrize("workload", ["ranking", "serving"])
def test_reference_arm_unavailable_for_library_loops(workload):
    (d,) = _last_json(_bench("--impl", "reference", "--workload", workload))
    assert d["impl"] == "reference" and "unavailable" in d


def test_reference_arm_only_rank0_prints():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_warmup_minimum_is_enforced():
    r = _bench("--impl", "reference", "--warmup", "2", timeout=120)
    assert r.returncode != 0 and "warmup" in (r.stderr + r.stdout)


def test_reference_arm_dimension_sweep():
    lines = _last_json(_bench("--impl", "reference", "--workload", "dims"))
    assert [d["D"] for d in lines] == [8, 16, 32, 50, 64, 100, 128]
    for d in lines:
        assert d["impl"] == "reference" and d["N"] == d["M"] == 10_000 and d["ms_per_sweep"] > 0
        assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


@pytest.mark.parametrize("workload", ["paper", "batched", "ranking", "serving", "dims"])
def test_single_gpu_workloads_leave_other_ranks_idle(workload):
    """Under torchrun the single-GPU workloads run on rank 0 only: another
    rank exits 0 at once, without touching a device or printing a line."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", workload, "--gpus", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
