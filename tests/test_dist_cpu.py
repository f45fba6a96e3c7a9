"""bench.py's multi-rank logic on CPU with two gloo ranks: the max/sum
reductions used for the timing (no data-path collective), and the reference
arm running on rank 0 only."""
from __future__ import annotations

import os
import socket
import sys
from pathlib import Path

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = Path(__file__).resolve().parent.parent


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    sys.path.insert(0, str(ROOT))
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, lr = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    bench.dist_barrier(dist)
    mx = bench.dist_max(dist, float(10 + rank))
    sm = bench.dist_sum(dist, float(1 + rank))
    import argparse
    ns = argparse.Namespace(workload="uniform", steps=4, warmup=3, ref_fraction=64)
    ref = bench.run_reference(ns, r, w)
    q.put((r, mx, sm, ref is None, None if ref is None else ref.get("impl")))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [11.0, 11.0]          # max over ranks
    assert [x[2] for x in res] == [3.0, 3.0]            # sum over ranks
    assert res[0][3] is False and res[0][4] == "reference"   # rank 0 runs the reference arm
    assert res[1][3] is True                             # rank 1 does no work


def test_reference_arm_line_has_the_contract_keys():
    """The --impl reference line (the oracle on the host) carries the keys the
    bench contract asks for, with the GPU arm's metric and unit."""
    sys.path.insert(0, str(ROOT))
    import argparse
    import bench
    ns = argparse.Namespace(workload="uniform", steps=3, warmup=3, ref_fraction=64)
    d = bench.run_reference(ns, 0, 1)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "edges/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 3
    assert "workload" in d["config"]
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["value"] == d["value"] and cpu["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_on_the_headline_workload():
    """With no --workload the reference arm times the oracle on the headline
    workload (the 8192 x 8192 grid), one step being a pass over a sample of
    every minibatch, and reports it on the GPU arm's metric and unit."""
    sys.path.insert(0, str(ROOT))
    import bench
    ns = bench.argparse.Namespace(workload=bench.HEADLINE, steps=1, warmup=3, ref_fraction=256)
    d = bench.run_reference(ns, 0, 1)
    assert bench.HEADLINE == "grid"
    assert d["impl"] == "reference" and d["unit"] == "edges/s" and d["value"] > 0
    assert "8192x8192" in d["config"]["workload"] and "pass" in d["config"]["step"]
    assert d["cpu_baseline"]["value"] == d["value"]


def test_paper_compression_interval_scales_with_the_batch():
    # the interval tuned at the largest paper batch, kept in edges at the
    # smaller ones; never compressing stays never
    sys.path.insert(0, str(ROOT))
    import bench
    big = bench.PAPER_BATCHES[-1]
    assert bench.paper_compress_every(6, big) == 6
    assert bench.paper_compress_every(6, big // 20) == 120
    assert bench.paper_compress_every(8, big // 2) == 16
    assert bench.paper_compress_every(0, big // 20) == 0
    assert bench.paper_compress_every(1, 2 * big) == 1          # never below one
    for b in bench.PAPER_BATCHES:
        e = bench.paper_compress_every(6, b)
        assert abs(e * b - 6 * big) <= b                       # edges between compressions kept


def test_ncu_traffic_is_withheld_under_option_overrides(monkeypatch):
    # measured DRAM bytes belong to the tuned configuration they were taken with
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setattr(bench, "OPTION_OVERRIDES", {"big_filter": 0})
    assert bench.ncu_traffic("update", "grid") == (None, None)
    monkeypatch.setattr(bench, "OPTION_OVERRIDES", {})
    t, k = bench.ncu_traffic("update", "grid")
    assert t is None or (t > 0 and k)
