"""The paper's Bulk-Update schedule (Algorithm 2 as written: relabel and
filter, connected components of A'', join) against the CPU oracle: A'' itself
as a multiset after every minibatch, the answers and the labels."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1602_05232_gb300 import inputs as I
from oracle_pins import load_golden

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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def sorted_pairs(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.int64).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def run(cc, s, options, check_a2=True):
    f = cc.Forest(s.n, update_schedule=1, **options)
    ref = oracle.OracleUF(s.n)
    for i, (e, q) in enumerate(s):
        want_a2 = ref.relabel(e) if check_a2 else None
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        m, rounds = f.schedule_stats()
        if check_a2:
            assert m == len(want_a2), f"|A''| at minibatch {i}"
            assert np.array_equal(sorted_pairs(f.nonloop_edges().cpu().numpy()),
                                  sorted_pairs(want_a2)), f"A'' at minibatch {i}"
        assert (rounds >= 1) == (m > 0)
        assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q)), i
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    assert f.components() == ref.components
    f.sync()


@pytest.mark.parametrize("opts", [{}, {"compress_every": 0}, {"compress_every": 3, "query_halving": 1},
                                  {"sv_graph": 0}, {"sv_graph": 0, "compress_every": 0}])
def test_paper_schedule_uniform(cc, opts):
    run(cc, I.uniform_stream(), opts)


@pytest.mark.parametrize("sv_graph", [1, 0], ids=["rounds_as_graph", "rounds_from_host"])
def test_paper_schedule_rmat_and_grid(cc, sv_graph):
    run(cc, I.rmat_stream(scale=16, m=1 << 19, batch=1 << 15, q=1 << 14, seed=3), {"sv_graph": sv_graph})
    run(cc, I.grid_stream(256, 256, batch=4001, q=4096, seed=4), {"compress_every": 2, "sv_graph": sv_graph})


@pytest.mark.parametrize("sv_graph", [1, 0], ids=["rounds_as_graph", "rounds_from_host"])
def test_paper_schedule_star_minibatch(cc, sv_graph):
    # the star of Section 3.2: on an empty graph A'' is the minibatch itself,
    # and one round of hooking joins v1..v8 under v1
    g = load_golden("star_minibatch.txt")
    f = cc.Forest(g["n"], update_schedule=1, sv_graph=sv_graph)
    f.bulk_update(dev(np.array(g["edges"], dtype=np.int32)))
    m, rounds = f.schedule_stats()
    assert m == 7 and rounds == 2           # one round hooks, the next finds nothing
    assert f.labels().cpu().tolist() == g["expect_labels"]
    assert f.components() == g["expect_components"]


def test_paper_schedule_hub_and_descending_path(cc):
    run(cc, I.hub_stream(n=1 << 16, m=1 << 19, batch=1 << 15, q=1 << 13), {})
    run(cc, I.hub_stream(n=1 << 16, m=1 << 18, batch=1 << 15, q=1 << 13, hub=0), {})
    n = 5000
    path = np.stack([np.arange(n - 1, 0, -1), np.arange(n - 2, -1, -1)], 1).astype(np.int32)
    for sv_graph in (1, 0):
        f = cc.Forest(n, update_schedule=1, sv_graph=sv_graph)
        f.bulk_update(dev(path))
        assert f.components() == 1 and int(f.labels().max()) == 0
        m, rounds = f.schedule_stats()
        assert m == n - 1 and rounds >= 2


def test_paper_schedule_full_size_rmat(cc):
    # the R-MAT n=2^24 stream (2^27 edges, minibatches of 2^20): every answer
    # and the final labels
    s = I.rmat_stream()
    f = cc.Forest(s.n, update_schedule=1)
    ref = oracle.OracleUF(s.n)
    for i in range(s.batches):
        e, q = s.edges(i), s.queries(i)
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q)), i
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())


def test_paper_schedule_unaligned_ragged_and_out_of_range(cc):
    # edge arrays 8 and 4 bytes past a 16-byte boundary, odd lengths (a ragged
    # last thread), and ids outside [0, n) that are skipped and reported
    s = I.uniform_stream(n=5000, m=3 * 12001, batch=12001, q=7001, seed=9)
    for shift in (2, 1):
        f = cc.Forest(s.n, update_schedule=1)
        ref = oracle.OracleUF(s.n)
        for i, (e, q) in enumerate(s):
            e = e.copy()
            e[::997, i % 2] = -1 - i          # negative ids
            e[5::1009, 1 - i % 2] = s.n + i   # ids >= n
            want_a2 = ref.relabel(e)
            buf = torch.zeros(e.size + 4, dtype=torch.int32, device="cuda")
            buf[shift:shift + e.size] = dev(e.ravel())
            f.bulk_update(buf[shift:shift + e.size])
            ref.bulk_update(e)
            m, _ = f.schedule_stats()
            assert m == len(want_a2), (shift, i)
            assert np.array_equal(sorted_pairs(f.nonloop_edges().cpu().numpy()), sorted_pairs(want_a2))
            with pytest.raises(cc.CCError) as ex:
                f.sync()
            assert ex.value.status == cc.CC_ERR_RANGE
            assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q)), (shift, i)
        assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
        f.sync()
