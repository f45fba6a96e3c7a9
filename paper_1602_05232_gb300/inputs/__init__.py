"""Seeded synthetic graph streams (host side, numpy arrays).

Holds no connectivity arithmetic: it draws vertex ids and nothing else, and
both the CUDA path and the CPU oracle consume the arrays it returns. The
native generator ``gen.c`` is counter-based (SplitMix64 evaluated at a
position), so any batch can be regenerated on its own and the bytes do not
depend on the thread count.

Stream model (Section 1, "Model"): a graph stream on V = {0..n-1} is a
sequence of minibatches of edges, not necessarily equal in size; after each
Bulk-Update the workloads here issue one Bulk-Query minibatch of vertex pairs.
Edges and pairs are ``int32`` arrays of shape ``(k, 2)`` (flat AoS
``u0, v0, u1, v1, ...``).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import Iterator

import numpy as np

from .._build import build_gen

# Stream tags: every purpose draws from its own SplitMix64 key.
TAG_EDGES = 1
TAG_QUERIES = 2
TAG_PERM = 3
TAG_SHUFFLE = 4
TAG_GRAPH_SIZES = 5
TAG_BATCH_SIZES = 6
TAG_TRACE = 7

_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build_gen()))
        u64, i64, i32, dbl, p = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_void_p)
        L.gen_stream_key.argtypes = [u64, u64]
        L.gen_stream_key.restype = u64
        L.gen_uniform_pairs.argtypes = [u64, u64, i64, i64, i64, p]
        L.gen_rmat_edges.argtypes = [u64, u64, i32, dbl, dbl, dbl, i64, i64, p, p]
        L.gen_permutation.argtypes = [u64, u64, i64, p]
        L.gen_shuffle_pairs.argtypes = [u64, u64, i64, p]
        L.gen_grid_edges.argtypes = [i64, i64, p]
        L.gen_grid_edges.restype = i64
        L.gen_grid3d_edges.argtypes = [i64, i64, i64, p]
        L.gen_grid3d_edges.restype = i64
        L.gen_unit.argtypes = [u64, u64, i64, i64, p]
        L.gen_u64.argtypes = [u64, u64, i64, i64, p]
        L.gen_set_threads.argtypes = [i32]
        for f in ("gen_uniform_pairs", "gen_rmat_edges", "gen_permutation",
                  "gen_shuffle_pairs", "gen_unit", "gen_u64", "gen_set_threads"):
            getattr(L, f).restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _out(k: int, out: np.ndarray | None) -> np.ndarray:
    if out is None:
        return np.empty((k, 2), dtype=np.int32)
    assert out.dtype == np.int32 and out.flags.c_contiguous and out.size >= 2 * k
    return out


def uniform_pairs(n: int, k: int, seed: int, tag: int, offset: int = 0,
                  out: np.ndarray | None = None) -> np.ndarray:
    """k pairs with both ids i.i.d. uniform over [0, n)."""
    out = _out(k, out)
    if k:
        lib().gen_uniform_pairs(seed, tag, n, k, offset, _ptr(out))
    return out


def permutation(n: int, seed: int, tag: int = TAG_PERM) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    lib().gen_permutation(seed, tag, n, _ptr(out))
    return out


def rmat_edges(scale: int, k: int, a: float, b: float, c: float, seed: int,
               tag: int = TAG_EDGES, offset: int = 0, perm: np.ndarray | None = None,
               out: np.ndarray | None = None) -> np.ndarray:
    """k R-MAT edges on 2^scale vertices, ids mapped through ``perm``."""
    if perm is not None:
        assert perm.dtype == np.int32 and perm.size == (1 << scale)
    out = _out(k, out)
    if k:
        lib().gen_rmat_edges(seed, tag, scale, a, b, c, k, offset, _ptr(perm), _ptr(out))
    return out


def grid_edges(rows: int, cols: int) -> np.ndarray:
    m = rows * (cols - 1) + (rows - 1) * cols
    out = np.empty((m, 2), dtype=np.int32)
    got = lib().gen_grid_edges(rows, cols, _ptr(out))
    assert got == m
    return out


def grid3d_edges(a: int, b: int, c: int) -> np.ndarray:
    m = a * b * (c - 1) + a * (b - 1) * c + (a - 1) * b * c
    out = np.empty((m, 2), dtype=np.int32)
    got = lib().gen_grid3d_edges(a, b, c, _ptr(out))
    assert got == m
    return out


def shuffle_pairs(pairs: np.ndarray, seed: int, tag: int = TAG_SHUFFLE) -> np.ndarray:
    assert pairs.dtype == np.int32 and pairs.flags.c_contiguous
    lib().gen_shuffle_pairs(seed, tag, pairs.shape[0], _ptr(pairs))
    return pairs


def unit(count: int, seed: int, tag: int, offset: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    if count:
        lib().gen_unit(seed, tag, count, offset, _ptr(out))
    return out


# ------------------------------------------------------------------ streams

@dataclass
class PlainStream:
    """One forest on n vertices fed by a sequence of (update, query) minibatch
    pairs. ``kind`` selects the edge source: 'uniform', 'rmat' or 'grid'."""
    name: str
    kind: str
    n: int
    update_sizes: list[int]
    query_sizes: list[int]
    seed: int = 0
    scale: int = 0
    abc: tuple[float, float, float] = (0.57, 0.19, 0.19)
    rows: int = 0
    cols: int = 0
    depth: int = 0
    hub: int = -1
    _perm: np.ndarray | None = field(default=None, repr=False)
    _grid: np.ndarray | None = field(default=None, repr=False)

    def __post_init__(self):
        self._eoff = np.concatenate([[0], np.cumsum(self.update_sizes, dtype=np.int64)])
        self._qoff = np.concatenate([[0], np.cumsum(self.query_sizes, dtype=np.int64)])

    @property
    def batches(self) -> int:
        return len(self.update_sizes)

    @property
    def m(self) -> int:
        return int(self._eoff[-1])

    @property
    def q(self) -> int:
        return int(self._qoff[-1])

    def perm(self) -> np.ndarray:
        if self._perm is None:
            self._perm = permutation(self.n, self.seed, TAG_PERM)
        return self._perm

    def grid(self) -> np.ndarray:
        if self._grid is None:
            g = (grid3d_edges(self.rows, self.cols, self.depth) if self.depth
                 else grid_edges(self.rows, self.cols))
            self._grid = shuffle_pairs(g, self.seed, TAG_SHUFFLE)
        return self._grid

    def edges_range(self, lo: int, hi: int, out: np.ndarray | None = None) -> np.ndarray:
        """Edges lo..hi-1 of the whole stream (global edge positions)."""
        k = hi - lo
        if self.kind == "uniform":
            return uniform_pairs(self.n, k, self.seed, TAG_EDGES, lo, out)
        if self.kind == "rmat":
            a, b, c = self.abc
            return rmat_edges(self.scale, k, a, b, c, self.seed, TAG_EDGES, lo,
                              self.perm(), out)
        if self.kind == "hub":
            out = uniform_pairs(self.n, k, self.seed, TAG_EDGES, lo, out)
            out[:k, 0] = self.hub
            return out
        if self.kind == "grid":
            src = self.grid()[lo:hi]
            if out is None:
                return src.copy()
            out[:k] = src
            return out[:k]
        raise ValueError(self.kind)

    def edges(self, i: int) -> np.ndarray:
        return self.edges_range(int(self._eoff[i]), int(self._eoff[i + 1]))

    def queries(self, i: int) -> np.ndarray:
        return uniform_pairs(self.n, self.query_sizes[i], self.seed, TAG_QUERIES,
                             int(self._qoff[i]))

    def all_edges(self, out: np.ndarray | None = None) -> np.ndarray:
        return self.edges_range(0, self.m, out)

    def all_queries(self, out: np.ndarray | None = None) -> np.ndarray:
        return uniform_pairs(self.n, self.q, self.seed, TAG_QUERIES, 0, out)

    def edge_offsets(self) -> np.ndarray:
        return self._eoff.copy()

    def query_offsets(self) -> np.ndarray:
        return self._qoff.copy()

    def __iter__(self) -> Iterator[tuple[np.ndarray, np.ndarray]]:
        for i in range(self.batches):
            yield self.edges(i), self.queries(i)


def uniform_stream(n: int = 1 << 16, m: int = 1 << 20, batch: int = 1 << 16,
                   q: int = 1 << 16, seed: int = 0) -> PlainStream:
    """Uniform random edges, endpoints i.i.d. over [0, n), self-loops kept
    (a stand-in for the paper's 'random' graph, Table 1). Defaults: n = 2^16,
    2^20 edges in 16 minibatches of 2^16, 2^16 query pairs after each."""
    nb = -(-m // batch)
    ups = [min(batch, m - i * batch) for i in range(nb)]
    return PlainStream(f"uniform n={n} m={m} b={batch}", "uniform", n, ups, [q] * nb, seed)


def rmat_stream(scale: int = 24, m: int = 1 << 27, batch: int = 1 << 20,
                q: int = 1 << 20, seed: int = 0,
                abc: tuple[float, float, float] = (0.57, 0.19, 0.19)) -> PlainStream:
    """R-MAT edges (a, b, c, d) = (0.57, 0.19, 0.19, 0.05) on 2^scale vertices
    with randomly permuted ids (stand-in for the paper's rMat graphs,
    Table 1). Defaults: scale 24, 2^27 edges in minibatches of 2^20, 2^20
    uniform query pairs after each."""
    nb = -(-m // batch)
    ups = [min(batch, m - i * batch) for i in range(nb)]
    return PlainStream(f"rmat scale={scale} m={m} b={batch}", "rmat", 1 << scale, ups,
                       [q] * nb, seed, scale=scale, abc=abc)


def hub_stream(n: int = 1 << 24, m: int = 1 << 27, batch: int = 1 << 20, q: int = 1 << 20,
               hub: int | None = None, seed: int = 0) -> PlainStream:
    """Every edge joins one hub vertex (default the largest id) to a uniform
    random vertex: the star of Section 3.2 at scale, the worst case for
    concurrent hooking onto one root."""
    nb = -(-m // batch)
    ups = [min(batch, m - i * batch) for i in range(nb)]
    h = n - 1 if hub is None else hub
    return PlainStream(f"hub n={n} m={m} b={batch} hub={h}", "hub", n, ups, [q] * nb, seed, hub=h)


def grid_stream(rows: int = 8192, cols: int = 8192, batch: int = 1 << 22,
                q: int = 1 << 22, seed: int = 0) -> PlainStream:
    """4-neighbour rows x cols grid, ids r*cols + c, edges Fisher-Yates shuffled
    (a 2-D stand-in for the paper's 3Dgrid, Table 1). Defaults: 8192 x 8192,
    134,201,344 edges in minibatches of 2^22 (the last one shorter), 2^22
    uniform query pairs after each."""
    m = rows * (cols - 1) + (rows - 1) * cols
    nb = -(-m // batch)
    ups = [min(batch, m - i * batch) for i in range(nb)]
    return PlainStream(f"grid {rows}x{cols} b={batch}", "grid", rows * cols, ups, [q] * nb,
                       seed, rows=rows, cols=cols)


def grid3d_stream(a: int = 464, b: int = 464, c: int = 464, batch: int = 10_000_000,
                  q: int = 1 << 20, seed: int = 0) -> PlainStream:
    """6-neighbour a x b x c mesh, edges Fisher-Yates shuffled. Default
    464^3: 99.9 M vertices and 299 M edges, the size of the paper's 3Dgrid
    (Table 1)."""
    m = a * b * (c - 1) + a * (b - 1) * c + (a - 1) * b * c
    nb = -(-m // batch)
    ups = [min(batch, m - i * batch) for i in range(nb)]
    return PlainStream(f"grid3d {a}x{b}x{c} b={batch}", "grid", a * b * c, ups, [q] * nb,
                       seed, rows=a, cols=b, depth=c)


# Paper-scale stand-ins for Table 1 (the paper's own generators are not
# available): sizes match, structure follows the named generator family.
def paper_stream(name: str, batch: int, q: int = 0, seed: int = 0) -> PlainStream:
    """'random': 10^8 vertices, 5x10^8 edges with i.i.d. uniform endpoints
    (the paper's random graph has 5 random neighbours per vertex);
    'rmat5': R-MAT scale 27 (134 M vertices), 5x10^8 edges; 'rmat16': the
    same with 1.6x10^9 edges; '3dgrid': the 464^3 mesh (99.9 M vertices,
    299 M edges)."""
    if name == "random":
        return uniform_stream(n=100_000_000, m=500_000_000, batch=batch, q=q, seed=seed)
    if name == "rmat5":
        return rmat_stream(scale=27, m=500_000_000, batch=batch, q=q, seed=seed)
    if name == "rmat16":
        return rmat_stream(scale=27, m=1_600_000_000, batch=batch, q=q, seed=seed)
    if name == "3dgrid":
        return grid3d_stream(batch=batch, q=q, seed=seed)
    raise ValueError(name)


# --------------------------------------------------------- segmented graphs

@dataclass
class SegmentedWorkload:
    """Many independent graphs, each with its own stream of uneven minibatches.

    Graph g has n_g = floor(2^(lo + (hi-lo) U)) vertices, U uniform in [0,1),
    and m_g = deg * n_g uniform local edges; its stream is cut into
    minibatches of floor(2^(blo + (bhi-blo) U)) edges (the last one
    truncated), each followed by a query minibatch of the same size with
    uniform local pairs. Ids in edges and pairs are LOCAL to the graph.
    """
    G: int
    n: np.ndarray                # int64[G]
    update_sizes: list[list[int]]
    seed: int
    deg: int

    def m(self, g: int) -> int:
        return self.deg * int(self.n[g])

    def edges(self, g: int) -> np.ndarray:
        return uniform_pairs(int(self.n[g]), self.m(g), self.seed, 256 * (g + 1) + TAG_EDGES)

    def queries(self, g: int) -> np.ndarray:
        return uniform_pairs(int(self.n[g]), self.m(g), self.seed, 256 * (g + 1) + TAG_QUERIES)

    def ops(self, g: int) -> list[tuple[int, int, int]]:
        """(kind, offset, size) in stream order; kind 0 = update, 1 = query;
        offset indexes edges(g) for updates and queries(g) for queries."""
        out, off = [], 0
        for s in self.update_sizes[g]:
            out.append((0, off, s))
            out.append((1, off, s))
            off += s
        return out

    @property
    def total_vertices(self) -> int:
        return int(self.n.sum())

    @property
    def total_edges(self) -> int:
        return self.deg * self.total_vertices


def segmented_workload(G: int = 1024, seed: int = 0, nlo: float = 8, nhi: float = 16,
                       blo: float = 6, bhi: float = 14, deg: int = 4) -> SegmentedWorkload:
    """Defaults: 1024 graphs, n log-uniform in [2^8, 2^16), m = 4n, minibatch
    sizes log-uniform in [2^6, 2^14)."""
    u = unit(G, seed, TAG_GRAPH_SIZES)
    n = np.floor(np.exp2(nlo + (nhi - nlo) * u)).astype(np.int64)
    sizes = []
    for g in range(G):
        m = deg * int(n[g])
        tag = 256 * (g + 1) + TAG_BATCH_SIZES
        out, left, j = [], m, 0
        while left > 0:
            need = max(8, 2 * left // (1 << int(blo)) + 8)
            draws = unit(need, seed, tag, j)
            for d in draws:
                s = int(math.floor(2.0 ** (blo + (bhi - blo) * d)))
                s = min(s, left)
                out.append(s)
                left -= s
                j += 1
                if left == 0:
                    break
        sizes.append(out)
    return SegmentedWorkload(G, n, sizes, seed, deg)


# ----------------------------------------------------------- request trace

@dataclass
class Request:
    t: float          # arrival time, seconds from trace start
    kind: int         # 0 = Bulk-Update, 1 = Bulk-Query
    offset: int       # position in the edge stream (updates) or pair stream (queries)
    size: int


def request_trace(stream_m: int, rate_hz: float, seed: int = 0, p_update: float = 0.75,
                  ulo: float = 8, uhi: float = 20, qlo: float = 8, qhi: float = 18,
                  max_requests: int | None = None) -> list[Request]:
    """Poisson arrivals at ``rate_hz``; each request is a Bulk-Update with
    probability p_update, taking the next floor(2^U(ulo,uhi)) edges of the
    stream, else a Bulk-Query of floor(2^U(qlo,qhi)) uniform pairs. The trace
    ends when the edge stream is used up (the last update truncated)."""
    reqs: list[Request] = []
    t, eoff, qoff, i = 0.0, 0, 0, 0
    chunk = 4096
    while eoff < stream_m and (max_requests is None or len(reqs) < max_requests):
        d = unit(4 * chunk, seed, TAG_TRACE, 4 * i)
        for j in range(chunk):
            gap, kind, size = d[4 * j], d[4 * j + 1], d[4 * j + 2]
            t += -math.log1p(-gap) / rate_hz
            if kind < p_update:
                s = min(int(math.floor(2.0 ** (ulo + (uhi - ulo) * size))), stream_m - eoff)
                reqs.append(Request(t, 0, eoff, s))
                eoff += s
            else:
                s = int(math.floor(2.0 ** (qlo + (qhi - qlo) * size)))
                reqs.append(Request(t, 1, qoff, s))
                qoff += s
            if eoff >= stream_m or (max_requests is not None and len(reqs) >= max_requests):
                break
        i += chunk
    return reqs
