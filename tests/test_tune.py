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


def test_coordinate_descent_from_several_starts_escapes_a_local_optimum():
    # two basins: from the default start, one-coordinate moves stop at
    # (a=1, b=1) with cost 2; the global minimum (a=4, b=4) needs a second start
    space = {"a": [1, 2, 3, 4], "b": [1, 2, 3, 4]}
    cost_table = {(1, 1): 2.0, (4, 4): 1.0}

    def cost(o):
        return cost_table.get((o["a"], o["b"]), 10.0)

    best, t, _ = tune.coordinate_descent(space, {"a": 1, "b": 1}, cost)
    assert best == {"a": 1, "b": 1}
    best, t, _ = tune.coordinate_descent(space, [{"a": 1, "b": 1}, {"a": 4, "b": 3}], cost)
    assert best == {"a": 4, "b": 4} and t == 1.0


def test_starts_include_the_stored_result(monkeypatch):
    space = {"x": [1, 2, 3], "y": [0, 1]}
    default = {"x": 1, "y": 0, "fixed": 7}
    monkeypatch.setattr(tune, "tuned_options", lambda wl, device=None: {"x": 3})
    starts = tune.starts_for("w", space, default)
    assert starts == [default, {"x": 3, "y": 0, "fixed": 7}]   # completed with the defaults
    monkeypatch.setattr(tune, "tuned_options", lambda wl, device=None: {"x": 9})
    assert tune.starts_for("w", space, default) == [default]     # value no longer in the space
    monkeypatch.setattr(tune, "tuned_options", lambda wl, device=None: None)
    assert tune.starts_for("w", space, default) == [default]


def test_canonical_plain_drops_a_filter_nothing_builds():
    o = {"compress_every": 0, "compress_scope": 0, "big_filter": 896, "block": 128}
    assert tune.canonical_plain(o) == {"compress_every": 0, "compress_scope": 0, "big_filter": 0, "block": 128}
    o = {"compress_every": 4, "compress_scope": 1, "big_filter": 640}
    assert tune.canonical_plain(o)["big_filter"] == 0
    o = {"compress_every": 6, "compress_scope": 0, "big_filter": 640}
    assert tune.canonical_plain(o) == o


def test_coordinate_descent_pairs_find_options_that_only_act_together():
    # b does nothing while a is 0 and a costs time while b is 0: from (0, 0)
    # no single move improves, the joint move (2, 1) does
    space = {"a": [0, 1, 2], "b": [0, 1], "c": [0, 1]}

    def cost(o):
        if o["a"] and o["b"]:
            return 1.0 + 0.1 * o["c"]
        return 3.0 + (1.0 if o["a"] else 0.0) + 0.1 * o["c"]

    best, t, _ = tune.coordinate_descent(space, {"a": 0, "b": 0, "c": 0}, cost)
    assert best == {"a": 0, "b": 0, "c": 0}
    best, t, _ = tune.coordinate_descent(space, {"a": 0, "b": 0, "c": 0}, cost, pairs=(("a", "b"),))
    assert best["a"] > 0 and best["b"] == 1 and t == 1.0
