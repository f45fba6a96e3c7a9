"""Bulk-Find (Algorithm 4, with the Response Distributor) against the CPU
oracle: on forests the test builds (the Figure 1 tree and seeded random
forests), the whole parent array after the call, the roots it returns and the
number of traversed vertices must match exactly; and Bulk-Query / the paper's
relabel step run through Bulk-Find must answer as the oracle does."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from oracle_pins import GOLDEN, random_forest
from paper_1602_05232_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05232_gb300 import _build, cc as ccmod
    _build.build_cc()
    ccmod.load()
    return ccmod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def check_forest(cc, par: np.ndarray, S: np.ndarray):
    want_par, want_res, want_t = oracle.bulk_find(par, S)
    f = cc.Forest(len(par))
    f.load_forest(dev(par))
    res = f.bulk_find(dev(S)).cpu().numpy()
    got_par = f.parent().cpu().numpy()
    t, up, down = f.bulk_find_stats()
    f.sync()
    assert np.array_equal(res, want_res)
    assert np.array_equal(got_par, want_par)
    assert t == want_t
    return up, down


def test_figure1_tree(cc):
    g = {"parent": []}
    for line in (GOLDEN / "figure1_bulk_find.txt").read_text().splitlines():
        line = line.split("#")[0].strip()
        if line:
            key, *vals = line.split()
            if key == "parent":
                g["parent"].append([int(x) for x in vals])
            elif key in ("n", "query", "expect_traversed"):
                g[key] = [int(x) for x in vals]
    n = g["n"][0]
    # renumber so that every parent has a smaller id (the GPU forest's
    # invariant): breadth-first from the root 19, then the untouched vertices
    children = {}
    for c, p in g["parent"]:
        children.setdefault(p, []).append(c)
    order, queue = [], [19]
    while queue:
        x = queue.pop(0)
        order.append(x)
        queue += sorted(children.get(x, []))
    order += [v for v in range(n) if v not in order]
    new = {old: i for i, old in enumerate(order)}
    par = np.arange(n, dtype=np.int32)
    for c, p in g["parent"]:
        par[new[c]] = new[p]
    S = np.array([new[q] for q in g["query"]], dtype=np.int32)
    up, down = check_forest(cc, par, S)
    # Phase I, all flows at once: F1 = {2, 10, 8} (3's flow merges into 1's at
    # 2), F2 = {19, 9} (2's flow stops at the visited 4), then 9's flow stops at
    # 4 and 19 is a root: 3 levels. Phase II goes down 19, 10, 4, {2, 9},
    # {1, 3, 8}, 7: 6 levels.
    assert (up, down) == (3, 6)


@pytest.mark.parametrize("seed", range(6))
def test_random_forests(cc, seed):
    r = np.random.default_rng(100 + seed)
    n = int(r.integers(1000, 200_000))
    par = random_forest(r, n, "index")
    S = r.integers(0, n, size=int(r.integers(1, 3 * n))).astype(np.int32)
    check_forest(cc, par, S)


def test_long_chains_and_duplicates(cc):
    # a few chains of 300 vertices (ids decreasing towards the roots) and a
    # query set made of many copies of the chain ends
    n = 3000
    par = np.arange(n, dtype=np.int32)
    for v in range(n):
        if v % 300:
            par[v] = v - 1
    S = np.array([v for v in range(299, n, 300)] * 50 + [0, 5, 5], dtype=np.int32)
    up, down = check_forest(cc, par, S)
    assert up == 300


def test_bulk_query_and_relabel_through_bulk_find(cc):
    for s, opts in [(I.uniform_stream(), {"compress_every": 0}),
                    (I.rmat_stream(scale=16, m=1 << 19, batch=1 << 15, q=1 << 14, seed=8),
                     {"compress_every": 0}),
                    (I.grid_stream(256, 256, batch=4001, q=4096, seed=9),
                     {"compress_every": 0, "update_schedule": 1})]:
        f = cc.Forest(s.n, bulk_find=1, **opts)
        ref = oracle.OracleUF(s.n)
        for i, (e, q) in enumerate(s):
            if opts.get("update_schedule") == 1:
                want_a2 = ref.relabel(e)
            f.bulk_update(dev(e))
            ref.bulk_update(e)
            if opts.get("update_schedule") == 1:
                assert f.schedule_stats()[0] == len(want_a2), i
            assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q)), i
        assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
        f.sync()


def test_load_forest_rejects_bad_arrays(cc):
    f = cc.Forest(10)
    bad = np.arange(10, dtype=np.int32)
    bad[3] = 7                      # a parent above the vertex
    with pytest.raises(cc.CCError) as ex:
        f.load_forest(dev(bad))
    assert ex.value.status == cc.CC_ERR_LABELS
    assert f.components() == 10
