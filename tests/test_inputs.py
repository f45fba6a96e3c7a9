"""Seeded input generators: determinism, shapes, ranges and distributions."""
from __future__ import annotations

import numpy as np

from paper_1602_05232_gb300 import inputs as I


def test_uniform_deterministic_and_offset_consistent():
    a = I.uniform_pairs(1000, 5000, seed=0, tag=I.TAG_EDGES)
    b = I.uniform_pairs(1000, 5000, seed=0, tag=I.TAG_EDGES)
    assert np.array_equal(a, b)
    part = I.uniform_pairs(1000, 100, seed=0, tag=I.TAG_EDGES, offset=1234)
    assert np.array_equal(part, a[1234:1334])
    assert a.min() >= 0 and a.max() < 1000
    c = I.uniform_pairs(1000, 5000, seed=1, tag=I.TAG_EDGES)
    assert not np.array_equal(a, c)


def test_thread_count_does_not_change_bytes():
    L = I.lib()
    L.gen_set_threads(1)
    a = I.rmat_edges(16, 200_000, 0.57, 0.19, 0.19, seed=4)
    L.gen_set_threads(7)
    b = I.rmat_edges(16, 200_000, 0.57, 0.19, 0.19, seed=4)
    L.gen_set_threads(0)
    assert np.array_equal(a, b)


def test_rmat_quadrant_frequencies():
    # without a permutation, the top bit of (u, v) picks the first quadrant
    e = I.rmat_edges(10, 200_000, 0.57, 0.19, 0.19, seed=2)
    top_u, top_v = e[:, 0] >> 9, e[:, 1] >> 9
    freq = [np.mean((top_u == i) & (top_v == j)) for i, j in ((0, 0), (0, 1), (1, 0), (1, 1))]
    assert np.allclose(freq, [0.57, 0.19, 0.19, 0.05], atol=0.005)


def test_permutation_is_a_permutation():
    p = I.permutation(100_003, seed=0)
    assert np.array_equal(np.sort(p), np.arange(100_003))


def test_grid_edges_and_shuffle():
    g = I.grid_edges(5, 7)
    assert g.shape == (5 * 6 + 4 * 7, 2)
    assert set(np.unique(g[:, 1] - g[:, 0])) == {1, 7}
    s = I.shuffle_pairs(g.copy(), seed=0)
    assert sorted(map(tuple, s.tolist())) == sorted(map(tuple, g.tolist()))
    assert not np.array_equal(s, g)


def test_stream_shapes():
    s = I.uniform_stream()
    assert (s.n, s.batches, s.m, s.q) == (1 << 16, 16, 1 << 20, 1 << 20)
    r = I.rmat_stream(scale=12, m=10_000, batch=3000, q=100)
    assert r.update_sizes == [3000, 3000, 3000, 1000]
    assert np.array_equal(r.all_edges()[3000:6000], r.edges(1))
    g = I.grid_stream(16, 16, batch=100, q=10)
    assert g.m == 2 * 16 * 15 and g.update_sizes[-1] == 480 - 400


def test_segmented_workload_shape():
    w = I.segmented_workload(G=64, seed=0)
    assert w.n.min() >= 256 and w.n.max() < 65536
    for g in range(w.G):
        sz = w.update_sizes[g]
        assert sum(sz) == w.m(g)
        assert all(1 <= s < (1 << 14) for s in sz)
        assert all(s >= 64 for s in sz[:-1])


def test_request_trace():
    t = I.request_trace(1 << 22, rate_hz=1000.0, seed=0)
    kinds = np.array([r.kind for r in t])
    assert abs(kinds.mean() - 0.25) < 0.05
    assert sum(r.size for r in t if r.kind == 0) == 1 << 22
    times = np.array([r.t for r in t])
    assert np.all(np.diff(times) > 0)
