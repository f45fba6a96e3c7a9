"""Pins for the CPU oracle: checks against things other than the oracle.

Each ``pin_*`` function runs the oracle library ``lib`` (a loaded build of
``oracle/cc_oracle.c``) and returns a list of failure messages (empty = pass).
They are run on the real oracle (all must pass) and on copies of it with a
planted mistake (at least one must fail), so a plausible slip anywhere in the
oracle -- a dropped edge, a wrong comparison, a swapped operand -- is caught.

What they pin to:
  * breadth-first search over an adjacency list (textbook connected
    components) on tiny random streams, every pair and every label;
  * scipy.sparse.csgraph.connected_components on mid-size graphs;
  * closed forms: the paper's star minibatch (Section 3.2, golden fixture),
    full and partial grids, a descending path, a perfect matching, the empty
    stream;
  * set semantics (Section 1, "Model"): the answers depend only on the edge
    set, not on order or batch split;
  * invariants: components = n - successful unions; answers reflexive,
    symmetric and transitive; labels idempotent with label[v] <= v;
    component count non-increasing along the stream;
  * the out-of-range rule: such edges are skipped and counted.
"""
from __future__ import annotations

from pathlib import Path

import numpy as np

import oracle

GOLDEN = Path(__file__).resolve().parent / "golden"


def bfs_labels(n: int, edges) -> list[int]:
    """Minimum-id component labels by iterative DFS/BFS over adjacency lists.
    Starting points are taken in increasing id order, so the first vertex of
    each component reached is its minimum."""
    adj: list[list[int]] = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    lab = [-1] * n
    for s in range(n):
        if lab[s] >= 0:
            continue
        lab[s] = s
        stack = [s]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if lab[y] < 0:
                    lab[y] = s
                    stack.append(y)
    return lab


def _uf(lib, n):
    return oracle.OracleUF(n, lib=lib)


def _rng(seed):
    return np.random.default_rng(seed)


def pin_bfs_tiny(lib, seeds=range(200)) -> list[str]:
    fails = []
    for seed in seeds:
        r = _rng(seed)
        n = int(r.integers(1, 40))
        uf = _uf(lib, n)
        seen: list[tuple[int, int]] = []
        for b in range(int(r.integers(1, 6))):
            k = int(r.integers(0, 2 * n + 1))
            e = r.integers(0, n, size=(k, 2)).astype(np.int32)
            uf.bulk_update(e)
            seen += [tuple(x) for x in e.tolist()]
            lab = bfs_labels(n, seen)
            got = uf.labels().tolist()
            if got != lab:
                fails.append(f"bfs labels seed={seed} batch={b}")
                break
            uu, vv = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
            pairs = np.stack([uu.ravel(), vv.ravel()], 1).astype(np.int32)
            ans = uf.bulk_query(pairs)
            lab_a = np.asarray(lab)
            want = (lab_a[pairs[:, 0]] == lab_a[pairs[:, 1]]).astype(np.uint8)
            if not np.array_equal(ans, want):
                fails.append(f"bfs answers seed={seed} batch={b}")
                break
            ncomp = len(set(lab))
            if uf.components != ncomp:
                fails.append(f"components seed={seed}: {uf.components} vs bfs {ncomp}")
                break
    return fails


def pin_scipy(lib) -> list[str]:
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    fails = []
    for seed, (n, m) in enumerate([(4096, 3000), (4096, 6000), (1 << 14, 1 << 14)]):
        r = _rng(1000 + seed)
        e = r.integers(0, n, size=(m, 2)).astype(np.int32)
        uf = _uf(lib, n)
        for part in np.array_split(e, 7):
            uf.bulk_update(part)
        g = coo_matrix((np.ones(m), (e[:, 0], e[:, 1])), shape=(n, n))
        ncomp, comp = connected_components(g, directed=False)
        first = np.full(ncomp, n, dtype=np.int64)
        np.minimum.at(first, comp, np.arange(n))
        want = first[comp].astype(np.int32)
        if not np.array_equal(uf.labels(), want):
            fails.append(f"scipy labels n={n} m={m}")
        if uf.components != ncomp:
            fails.append(f"scipy components n={n} m={m}")
    return fails


def load_golden(name: str) -> dict:
    d: dict = {"edges": []}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "edge":
            d["edges"].append(tuple(int(x) for x in vals))
        elif key in ("n", "expect_components"):
            d[key] = int(vals[0])
        else:
            d[key] = [int(x) for x in vals]
    return d


def pin_star(lib) -> list[str]:
    g = load_golden("star_minibatch.txt")
    uf = _uf(lib, g["n"])
    uf.bulk_update(np.array(g["edges"], dtype=np.int32))
    fails = []
    if uf.labels().tolist() != g["expect_labels"]:
        fails.append("star labels")
    if uf.components != g["expect_components"]:
        fails.append("star components")
    q = np.array([[1, 8], [8, 1], [2, 7], [0, 1], [0, 0]], dtype=np.int32)
    if uf.bulk_query(q).tolist() != [1, 1, 1, 0, 1]:
        fails.append("star answers")
    # high-id hub: the same star mirrored so the centre is the largest id
    uf2 = _uf(lib, 9)
    uf2.bulk_update(np.array([[8, i] for i in range(1, 8)], dtype=np.int32))
    if uf2.labels().tolist() != [0] + [1] * 8:
        fails.append("mirrored star labels")
    return fails


def pin_closed_forms(lib) -> list[str]:
    from paper_1602_05232_gb300 import inputs as I
    fails = []
    # full grid: one component, every label 0
    rows, cols = 48, 37
    e = I.shuffle_pairs(I.grid_edges(rows, cols), seed=3)
    uf = _uf(lib, rows * cols)
    for part in np.array_split(e, 5):
        uf.bulk_update(part)
    lab = uf.labels()
    if uf.components != 1 or lab.max() != 0:
        fails.append("grid: not one component labelled 0")
    # horizontal edges only: one component per row, labelled r*cols
    h = e[e[:, 1] == e[:, 0] + 1]
    uf = _uf(lib, rows * cols)
    uf.bulk_update(h)
    want = (np.arange(rows * cols) // cols) * cols
    if uf.components != rows or not np.array_equal(uf.labels(), want):
        fails.append("row grid")
    # path with ids in descending order
    n = 1000
    p = np.stack([np.arange(n - 1, 0, -1), np.arange(n - 2, -1, -1)], 1).astype(np.int32)
    uf = _uf(lib, n)
    uf.bulk_update(p)
    if uf.components != 1 or uf.labels().max() != 0:
        fails.append("descending path")
    # perfect matching in random order: n/2 components, label of 2i+1 is 2i
    n = 2000
    mt = np.stack([np.arange(0, n, 2), np.arange(1, n, 2)], 1).astype(np.int32)
    mt = mt[_rng(5).permutation(n // 2)][:, ::-1].copy()
    uf = _uf(lib, n)
    uf.bulk_update(mt)
    if uf.components != n // 2 or not np.array_equal(uf.labels(), np.arange(n) & ~1):
        fails.append("perfect matching")
    # empty stream: identity labels, n components, only reflexive pairs connected
    uf = _uf(lib, 77)
    uf.bulk_update(np.zeros((0, 2), dtype=np.int32))
    q = np.array([[3, 3], [3, 4], [76, 0]], dtype=np.int32)
    if (uf.components != 77 or not np.array_equal(uf.labels(), np.arange(77))
            or uf.bulk_query(q).tolist() != [1, 0, 0]):
        fails.append("empty stream")
    # self-loops and duplicates change nothing
    uf = _uf(lib, 10)
    uf.bulk_update(np.array([[4, 4], [2, 2], [1, 3], [3, 1], [1, 3]], dtype=np.int32))
    if uf.components != 9 or uf.unions != 1:
        fails.append("self-loops/duplicates")
    return fails


def pin_order_independence(lib) -> list[str]:
    fails = []
    r = _rng(77)
    n, m = 3000, 2500
    e = r.integers(0, n, size=(m, 2)).astype(np.int32)
    q = r.integers(0, n, size=(5000, 2)).astype(np.int32)
    results = []
    for trial in range(3):
        perm = r.permutation(m)
        cuts = np.sort(r.choice(np.arange(1, m), size=trial * 3, replace=False))
        uf = _uf(lib, n)
        for part in np.split(e[perm], cuts):
            uf.bulk_update(part)
        results.append((uf.labels(), uf.bulk_query(q), uf.components))
    for lab, ans, c in results[1:]:
        if not (np.array_equal(lab, results[0][0]) and np.array_equal(ans, results[0][1])
                and c == results[0][2]):
            fails.append("order/split dependence")
    return fails


def pin_invariants(lib) -> list[str]:
    from paper_1602_05232_gb300 import inputs as I
    fails = []
    s = I.rmat_stream(scale=12, m=1 << 14, batch=1 << 11, q=1 << 11, seed=9)
    uf = _uf(lib, s.n)
    prev = s.n
    r = _rng(3)
    for i, (e, q) in enumerate(s):
        made = uf.bulk_update(e)
        if uf.components != prev - made:
            fails.append(f"unions/components mismatch at batch {i}")
        if uf.components > prev:
            fails.append("components increased")
        prev = uf.components
        lab = uf.labels()
        if not np.array_equal(lab[lab], lab) or np.any(lab > np.arange(s.n)):
            fails.append(f"labels not idempotent/minimal at batch {i}")
        # reflexive, symmetric, transitive on sampled triples
        x, y, z = (r.integers(0, s.n, 4000).astype(np.int32) for _ in range(3))
        a_xy = uf.bulk_query(np.stack([x, y], 1))
        a_yx = uf.bulk_query(np.stack([y, x], 1))
        a_yz = uf.bulk_query(np.stack([y, z], 1))
        a_xz = uf.bulk_query(np.stack([x, z], 1))
        if not np.array_equal(a_xy, a_yx):
            fails.append("not symmetric")
        if np.any((a_xy & a_yz) > a_xz):
            fails.append("not transitive")
        if not np.all(uf.bulk_query(np.stack([x, x], 1)) == 1):
            fails.append("not reflexive")
        # answers agree with the labels
        if not np.array_equal(a_xy, (lab[x] == lab[y]).astype(np.uint8)):
            fails.append("answers disagree with labels")
        # lab[v] is in v's component, and no smaller id is
        a_lab = uf.bulk_query(np.stack([x, lab[x]], 1))
        if not np.all(a_lab == 1):
            fails.append("label not connected to its vertex")
    return fails


def pin_range_rule(lib) -> list[str]:
    fails = []
    uf = _uf(lib, 6)
    e = np.array([[0, 1], [-1, 2], [2, 6], [3, 4], [5, 7]], dtype=np.int32)
    made = uf.bulk_update(e)
    if made != 2 or uf.errors != 3 or uf.labels().tolist() != [0, 0, 2, 3, 3, 5]:
        fails.append("out-of-range edges not skipped and counted")
    ans = uf.bulk_query(np.array([[0, 1], [6, 6], [3, 4]], dtype=np.int32))
    if ans.tolist() != [1, 0, 1] or uf.errors != 4:
        fails.append("out-of-range query not answered 0 and counted")
    return fails


def pin_relabel(lib) -> list[str]:
    """A'' (Algorithm 2's relabel + self-loop filter) against BFS labels on
    tiny streams, and the star minibatch closed form (Section 3.2)."""
    fails = []
    for seed in range(120):
        r = _rng(5000 + seed)
        n = int(r.integers(1, 30))
        uf = _uf(lib, n)
        seen = []
        for b in range(4):
            e = r.integers(0, n, size=(int(r.integers(0, 2 * n + 1)), 2)).astype(np.int32)
            lab = bfs_labels(n, seen)
            want = [(lab[u], lab[v]) for u, v in e.tolist() if lab[u] != lab[v]]
            got = [tuple(x) for x in uf.relabel(e).tolist()]
            if got != want:
                fails.append(f"relabel seed={seed} batch={b}")
                break
            uf.bulk_update(e)
            seen += [tuple(x) for x in e.tolist()]
    g = load_golden("star_minibatch.txt")
    star = np.array(g["edges"], dtype=np.int32)
    uf = _uf(lib, g["n"])
    if uf.relabel(star).tolist() != star.tolist():
        fails.append("star: on the empty graph A'' is the minibatch itself")
    uf.bulk_update(star)
    if len(uf.relabel(star)) != 0:
        fails.append("star: repeating the minibatch leaves only self-loops")
    if uf.relabel(np.array([[0, 8]], dtype=np.int32)).tolist() != [[0, 1]]:
        fails.append("star: an edge into the star relabels to the star's smallest id")
    # the range rule: an edge with an id outside [0, n) is dropped from A''
    # (as Bulk-Update skips it); ids 0 and n - 1 are in range
    n = 10
    uf = _uf(lib, n)
    uf.bulk_update(np.array([[1, 2]], dtype=np.int32))
    e = np.array([[0, 9], [-1, 3], [2, 3], [4, n], [2**31 - 1, 0], [9, 1]], dtype=np.int32)
    if uf.relabel(e).tolist() != [[0, 9], [1, 3], [9, 1]]:
        fails.append("relabel: out-of-range edges dropped, boundary ids kept")
    return fails


def serial_finds(parent, order):
    """Textbook serial find with full path compression, applied in `order`."""
    p = list(parent)
    for s in order:
        r = s
        while p[r] != r:
            r = p[r]
        x = s
        while p[x] != r and x != r:
            nxt = p[x]
            p[x] = r
            x = nxt
    return p


def random_forest(rng, n, shape):
    """Seeded random forest on 0..n-1. 'index': parent[v] <= v (the GPU
    path's invariant); 'any': parents point anywhere, no cycles."""
    if shape == "index":
        par = np.arange(n)
        for v in range(1, n):
            if rng.random() < 0.8:
                par[v] = int(rng.integers(0, v))
        return par.astype(np.int32)
    order = rng.permutation(n)
    par = np.arange(n)
    for i in range(1, n):
        if rng.random() < 0.8:
            par[order[i]] = order[int(rng.integers(0, i))]
    return par.astype(np.int32)


def pin_bulk_find(lib) -> list[str]:
    """Bulk-Find against the Figure 1 example (golden fixture) and against
    serial finds with full path compression in several orders, including the
    dependency order the paper derives (Section 4.2)."""
    fails = []
    g = {"parent": [], "expect_parent": []}
    for line in (GOLDEN / "figure1_bulk_find.txt").read_text().splitlines():
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        vals = [int(x) for x in vals]
        if key in ("parent", "expect_parent"):
            g[key].append(vals)
        else:
            g[key] = vals
    n = g["n"][0]
    par = np.arange(n, dtype=np.int32)
    for c, p in g["parent"]:
        par[c] = p
    want = par.copy()
    for c, p in g["expect_parent"]:
        want[c] = p
    out, res, t = oracle.bulk_find(par, g["query"], lib=lib)
    if not np.array_equal(out, want):
        fails.append("figure 1: forest after Bulk-Find")
    if res.tolist() != g["expect_res"] or t != g["expect_traversed"][0]:
        fails.append("figure 1: roots or traversal count")
    if serial_finds(par.tolist(), g["serial_order"]) != out.tolist():
        fails.append("figure 1: serial finds in the paper's order")
    r = _rng(4242)
    for trial in range(60):
        n = int(r.integers(2, 80))
        par = random_forest(r, n, "any" if trial % 2 else "index")
        S = r.integers(0, n, size=int(r.integers(1, 2 * n))).astype(np.int32)
        out, res, t = oracle.bulk_find(par, S, lib=lib)
        for order in (S.tolist(), S[::-1].tolist(), r.permutation(S).tolist()):
            if serial_finds(par.tolist(), order) != out.tolist():
                fails.append(f"bulk find vs serial finds, trial {trial}")
                break
        roots = []
        path_nodes = set()
        for s in S.tolist():
            x = s
            while par[x] != x:
                path_nodes.add(x)
                x = int(par[x])
            roots.append(x)
        if res.tolist() != roots or t != len(path_nodes):
            fails.append(f"bulk find roots / traversal count, trial {trial}")
    return fails


ALL_PINS = [pin_bfs_tiny, pin_scipy, pin_star, pin_closed_forms,
            pin_order_independence, pin_invariants, pin_range_rule, pin_relabel,
            pin_bulk_find]


def run_all(lib) -> list[str]:
    out = []
    for p in ALL_PINS:
        try:
            out += [f"{p.__name__}: {m}" for m in p(lib)]
        except Exception as ex:  # a mutant may also crash a pin's bookkeeping
            out.append(f"{p.__name__}: raised {type(ex).__name__}: {ex}")
    return out
