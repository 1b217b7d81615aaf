"""The benchmark's command-line contract, checked on the CPU.

* `bench.py --impl reference` times the FP64 oracle on the host cores and
  prints one JSON line with the GPU arm's metric, unit and workload, its
  `cpu_baseline` and an `e2e` object with no host<->device bytes.
* `bench.py` itself (the GPU arm) needs a GPU and exits non-zero without one:
  there is no CPU fallback.
"""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=600, cwd=ROOT)


def test_reference_arm_prints_the_contract_line():
    r = _run("--impl", "reference", "--steps", "2", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["n_gpus"] == 1
    assert line["config"]["workload"].startswith("jet_c3")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_gpu_arm_fails_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        import pytest
        pytest.skip("a GPU is present")
    r = _run("--steps", "2", "--warmup", "3")
    assert r.returncode != 0
    assert not r.stdout.strip(), "no bench line without a GPU"


def test_pool_peaks_fall_back_when_the_measured_file_is_absent(monkeypatch, tmp_path):
    # the roofline denominators come from MEASURED_PEAKS.json when present
    # ("of measured"), else from the documented fallback ("of fallback")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.pool_peak("hbm_gbs") == (6800.0, "of fallback")
    assert bench.pool_peak("bf16_tflops") == (1900.0, "of fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6805.1}))
    assert bench.pool_peak("hbm_gbs") == (6805.1, "of measured")
    assert bench.pool_peak("bf16_tflops") == (1900.0, "of fallback")


def test_step_bytes_lower_bound_itemised():
    # FP32 with surface tension: 2 x (28 + 8 + 16) + 56 + 28 = 188 B, the
    # method's ~190 B per particle-step, plus 100 B per cell sort
    assert bench.step_bytes_lower(False, True, 0.0) == 188.0
    assert bench.step_bytes_lower(False, True, 0.13) == pytest.approx(201.0)
    assert bench.step_bytes_lower(False, False, 0.0) == 2 * 28 + 56 + 28
    assert bench.step_bytes_lower(True, False, 0.0) == 2 * 40 + 80 + 40
