"""bench.py's JSON line on a GPU: a short run of the default workload (the
8192 x 8192 grid, one step = one whole pass) carries every key of the bench
contract, with consistent values, and the other forms in the same line."""
from __future__ import annotations

import json
import subprocess
import sys
from pathlib import Path

import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = Path(__file__).resolve().parent.parent


def test_default_bench_line():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "bench.py", "--steps", "4", "--warmup", "3", "--cpu-seconds", "1",
                        "--serve-scale", "18"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks"):
        assert key in d, key
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 4 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["unit"] == "edges/s"
    assert d["config"]["n"] == 1 << 26 and d["config"]["minibatches_per_pass"] == 32
    per_pass = d["config"]["edges_per_pass"]
    assert per_pass == 134201344
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - per_pass) / per_pass < 0.01
    rf = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in rf, key
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0 < rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"], rel=1e-3)
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0 and cpu["sample"]
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] >= 2 * 32 * d["steps"]     # an update and a query per minibatch
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert rf["timing_basis"] and 0 < rf["in_step_share"] <= 1
    lat = d["latency_ms"]
    assert 0 < lat["batch_p50"] <= lat["batch_p99"] and 0 < lat["pass_p50"] <= lat["pass_p99"]
    forms = d["forms"]
    assert set(forms) == {"rmat", "uniform", "segmented", "serving"}
    assert forms["rmat"]["value"] > 0 and forms["rmat"]["config"]["edges_per_pass"] == 1 << 27
    assert forms["segmented"]["speedup_vs_plain"] > 0 and forms["segmented"]["plain_form"]["edges_per_s"] > 0
    sv = forms["serving"]
    assert sv["saturation"]["edges_per_s"] > 0 and len(sv["saturation"]["runs_edges_per_s"]) == 3
    assert set(sv["latency_at_load"]) == {"0.5", "0.8", "0.95"}
    assert sv["served_labels_equal_plain"] is True


def test_stream_runner_for_profilers():
    # the command the ncu summaries name: a few minibatches with the tuned
    # options, and with an option given over them
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for extra in ([], ["--opt", "big_filter=0", "--opt", "compress_every=4"]):
        r = subprocess.run([sys.executable, "-m", "paper_1602_05232_gb300.stream_run", "--workload", "rmat",
                            "--minibatches", "3", *extra],
                           cwd=ROOT, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        assert "rmat: 3 minibatches" in r.stdout
    r = subprocess.run([sys.executable, "-m", "paper_1602_05232_gb300.stream_run", "--opt", "no_such=1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0 and "unknown option" in r.stderr
