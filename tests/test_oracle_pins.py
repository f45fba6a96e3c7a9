"""The CPU oracle against its pins, and the pins against planted mistakes.

Each planted mistake is applied to a copy of ``oracle/cc_oracle.c`` in a temp
directory and compiled there; the real oracle source is never changed.
"""
from __future__ import annotations

import subprocess

import pytest

import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(lib, pin):
    assert pin(lib) == []


# (description, exact text in cc_oracle.c, replacement, occurrence index)
MUTANTS = [
    ("drops the last edge of every minibatch",
     "int64_t made = 0;\n    for (int64_t i = 0; i < k; i++) {",
     "int64_t made = 0;\n    for (int64_t i = 0; i + 1 < k; i++) {"),
    ("unions already-connected roots instead of distinct ones",
     "if (ra == rb) continue;", "if (ra != rb) continue;"),
    ("query compares an endpoint with itself",
     "out[i] = (uint8_t)(find(u, a) == find(u, b));",
     "out[i] = (uint8_t)(find(u, a) == find(u, a));"),
    ("reads the first endpoint twice",
     "int32_t a = edges[2 * i], b = edges[2 * i + 1];\n        if (!in_range(u, a) || !in_range(u, b)) { u->errors++;",
     "int32_t a = edges[2 * i], b = edges[2 * i];\n        if (!in_range(u, a) || !in_range(u, b)) { u->errors++;"),
    ("labels keep the maximum id",
     "if (v < mn[r]) mn[r] = (int32_t)v;", "if (mn[r] == INT32_MAX || v > mn[r]) mn[r] = (int32_t)v;"),
    ("compression cuts a node loose",
     "u->p[x] = r;", "u->p[x] = x;"),
    ("vertex 0 treated as out of range",
     "return x >= 0 && x < u->n;", "return x > 0 && x < u->n;"),
    ("component count ignores unions",
     "return u->n - u->unions;", "return u->n;"),
    ("forgets the link when ranks are equal",
     "u->p[rb] = ra;\n            u->rank[ra]++;", "u->rank[ra]++;"),
    ("relabel keeps self-loops",
     "if (lab[a] == lab[b]) continue;", "if (lab[a] == lab[b] && a < 0) continue;"),
    ("relabel writes the endpoint instead of its identifier",
     "out[2 * m + 1] = lab[b];", "out[2 * m + 1] = b;"),
    ("bulk find compresses only the query node",
     "seen[x] = 1;\n            parent_out[x] = r;", "seen[x] = 1;\n            if (x == S[i]) parent_out[x] = r;"),
    ("bulk find points at the parent instead of the root",
     "parent_out[x] = r;\n            traversed++;", "parent_out[x] = parent_in[parent_in[x]];\n            traversed++;"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, desc, old, new):
    src = oracle.SRC.read_text()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    r = subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", str(mutant), "-o", str(so)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    fails = P.run_all(oracle.load(so))
    assert fails, f"no pin caught the planted mistake: {desc}"
