"""Autotuner search logic on a synthetic cost surface (no GPU)."""
from __future__ import annotations

import pytest

torch = pytest.importorskip("torch")
from paper_1602_05232_gb300 import tune  # noqa: E402


def test_coordinate_descent_finds_separable_minimum():
    space = {"a": [1, 2, 3, 4], "b": [10, 20, 30], "c": [0, 1]}
    target = {"a": 3, "b": 20, "c": 1}
    calls = []

    def cost(o):
        calls.append(o)
        return sum((o[k] - target[k]) ** 2 for k in target) + 1.0

    best, t, table = tune.coordinate_descent(space, {"a": 1, "b": 10, "c": 0}, cost)
    assert best == target and t == 1.0
    assert len(table) < 4 * 3 * 2            # fewer evaluations than the full grid


def test_coordinate_descent_retimes_finalists():
    noise = {"n": 0}

    def cost(o):
        noise["n"] += 1
        return {1: 5.0, 2: 1.0, 3: 3.0}[o["x"]]

    best, t, _ = tune.coordinate_descent({"x": [1, 2, 3]}, {"x": 1}, cost)
    assert best == {"x": 2}


def test_tuned_options_missing_device_is_none():
    assert tune.tuned_options("rmat", device="no such device") is None
