"""The largest-component filter (CC_OPT_BIG_FILTER) against the oracle.

The filter must never change an answer or a label (the parity option sets in
test_parity_gpu.py run whole streams with it). These tests check what it
records: the root it picks is a component minimum, the vertices it marks are
exactly that component, the sampled-share threshold is honoured, and a reset
or a loaded forest turns it off so that stale marks cannot answer a query.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
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


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def component_sizes(labels: np.ndarray) -> np.ndarray:
    return np.bincount(labels, minlength=len(labels))


def test_marks_exactly_the_picked_component_along_a_grid_stream(cc):
    # 512 x 512 grid, 32 minibatches: the largest component appears near the
    # percolation point and grows to the whole grid. After every minibatch
    # (each followed by a compression), the picked root is a component
    # minimum, the marked count is that component's size, and once one
    # component holds more than half the vertices it is the one picked.
    s = I.grid_stream(512, 512, batch=(2 * 512 * 511) // 32 + 1, q=1 << 12, seed=3)
    f = cc.Forest(s.n, big_filter=1, compress_every=1)
    ref = oracle.OracleUF(s.n)
    picked_largest = 0
    for i, (e, q) in enumerate(s):
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        root, members = f.big_filter_stats()
        lab = ref.labels()
        size = component_sizes(lab)
        assert root >= 0, f"minibatch {i}: a share of 1 always picks a root"
        assert lab[root] == root, f"minibatch {i}: root {root} is not a component minimum"
        assert members == size[root], f"minibatch {i}: marked {members}, component has {size[root]}"
        if size.max() * 2 > s.n:
            assert size[root] == size.max(), f"minibatch {i}: the majority component was not picked"
            picked_largest += 1
        got = f.bulk_query(dev(q)).cpu().numpy()
        assert np.array_equal(got, ref.bulk_query(q)), f"answers differ at minibatch {i}"
    assert picked_largest >= 8
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    f.sync()


@pytest.mark.parametrize("share", [1, 300, 700, 1024])
def test_sampled_share_threshold(cc, share):
    # one component of about half the vertices (ids spread over [0, n)), the
    # rest singletons: the filter turns on only when its sampled share is at
    # least the threshold; the answers are the oracle's either way
    n = 1 << 16
    rng = np.random.default_rng(7)
    members = np.sort(rng.choice(n, size=n // 2, replace=False)).astype(np.int32)
    path = np.stack([members[:-1], members[1:]], axis=1)
    f = cc.Forest(n, big_filter=share, compress_every=1)
    ref = oracle.OracleUF(n)
    f.bulk_update(dev(path))
    ref.bulk_update(path)
    root, marked = f.big_filter_stats()
    if share <= 300:
        assert root == int(members[0]) and marked == n // 2
    elif share >= 700:
        assert root == -1 and marked == 0
    q = rng.integers(0, n, size=(1 << 16, 2)).astype(np.int32)
    q[: 1 << 12] = members[rng.integers(0, n // 2, size=(1 << 12, 2))]
    assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q))
    f.sync()


def _connected_then(cc, n, after):
    """Connect all n vertices with the filter on, then call after(f)."""
    f = cc.Forest(n, big_filter=1, compress_every=1)
    chain = np.stack([np.arange(1, n), np.arange(n - 1)], axis=1).astype(np.int32)
    f.bulk_update(dev(chain))
    root, marked = f.big_filter_stats()
    assert (root, marked) == (0, n)
    after(f)
    return f


def test_reset_turns_the_filter_off(cc):
    # a forest of one component, marked in full; after cc_reset the marks
    # must not answer: with no compression since, every pair of distinct
    # vertices is disconnected
    n = 5000
    f = _connected_then(cc, n, lambda f: f.reset())
    assert f.big_filter_stats() == (-1, 0)
    f.set_option("compress_every", 0)
    f.bulk_update(dev(np.array([[10, 20]])))
    q = np.array([[1, 2], [10, 20], [0, n - 1], [7, 7], [20, 4999]], dtype=np.int32)
    assert f.bulk_query(dev(q)).cpu().tolist() == [0, 1, 0, 1, 0]
    f.sync()


def test_loaded_labels_and_forest_turn_the_filter_off(cc):
    n = 3000
    q = np.array([[1, 2], [0, n - 1], [5, 5], [100, 200]], dtype=np.int32)
    ident = torch.arange(n, dtype=torch.int32, device="cuda")
    f = _connected_then(cc, n, lambda f: f.load_labels(ident))
    assert f.big_filter_stats() == (-1, 0)
    assert f.bulk_query(dev(q)).cpu().tolist() == [0, 0, 1, 0]
    f.sync()
    g = _connected_then(cc, n, lambda g: g.load_forest(ident))
    assert g.big_filter_stats() == (-1, 0)
    g.set_option("compress_every", 0)
    g.bulk_update(dev(np.array([[100, 200]])))
    assert g.bulk_query(dev(q)).cpu().tolist() == [0, 0, 1, 1]
    g.sync()


@pytest.mark.parametrize("n", [1, 5, 31, 32, 33, 127, 129, 1000, 1023, 4097, 100_003])
def test_ragged_vertex_counts(cc, n):
    # bitmap words and the warp grouping at sizes that do not fill them,
    # including fewer vertices than samples
    rng = np.random.default_rng(n)
    f = cc.Forest(n, big_filter=1, compress_every=1, block=64)
    ref = oracle.OracleUF(n)
    for _ in range(3):
        e = rng.integers(0, n, size=(max(1, n // 2), 2)).astype(np.int32)
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        root, marked = f.big_filter_stats()
        lab = ref.labels()
        assert root >= 0 and lab[root] == root and marked == int((lab == root).sum())
        q = rng.integers(0, n, size=(4 * n + 7, 2)).astype(np.int32)
        assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q))
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    f.sync()


def test_explicit_compress_and_labels_keep_the_marks(cc):
    # cc_compress(ALL) builds the bitmap with automatic compression off; a
    # labels call (which flattens the forest) leaves it valid
    n = 1 << 14
    rng = np.random.default_rng(11)
    f = cc.Forest(n, big_filter=1, compress_every=0)
    ref = oracle.OracleUF(n)
    e = rng.integers(0, n, size=(n, 2)).astype(np.int32)
    f.bulk_update(dev(e))
    ref.bulk_update(e)
    assert f.big_filter_stats() == (-1, 0)
    f.compress()
    root, marked = f.big_filter_stats()
    lab = ref.labels()
    assert marked == int((lab == root).sum()) and marked > n // 2
    assert np.array_equal(f.labels().cpu().numpy(), lab)
    e2 = rng.integers(0, n, size=(n // 4, 2)).astype(np.int32)
    f.bulk_update(dev(e2))
    ref.bulk_update(e2)
    q = rng.integers(0, n, size=(1 << 16, 2)).astype(np.int32)
    assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q))
    assert f.kernel_stats()["big_pick"] == 1
    f.sync()


def test_segmented_handle_rejects_the_filter(cc):
    f = cc.Forest.segmented([100, 200])
    with pytest.raises(cc.CCError) as ex:
        f.set_option("big_filter", 1)
    assert ex.value.status == cc.CC_ERR_UNSUPPORTED
    assert f.get_option("big_filter") == 0
    f.close()


@pytest.mark.parametrize("offset", [0, 1, 2], ids=["16B", "4B", "8B"])
def test_ordered_update_reads_the_callers_edges_while_the_filter_is_on(cc, offset):
    # edge order + filter: once the bitmap marks a tree, the order kernels do
    # nothing and the update reads the caller's array, here starting 0, 4 or 8
    # bytes past a 16-byte boundary; compared with the oracle after every
    # minibatch of a 512 x 512 grid stream, through the point where the filter
    # turns on
    s = I.grid_stream(512, 512, batch=(1 << 14) + 1, q=1 << 13, seed=5)
    f = cc.Forest(s.n, big_filter=128, edge_order=7, compress_every=2, update_variant=5, block=128)
    ref = oracle.OracleUF(s.n)
    on = 0
    for i, (e, q) in enumerate(s):
        buf = torch.empty(2 * len(e) + 4, dtype=torch.int32, device="cuda")
        view = buf[offset:offset + 2 * len(e)].view(-1, 2)
        view.copy_(dev(e))
        f.bulk_update(view)
        ref.bulk_update(e)
        got = f.bulk_query(dev(q)).cpu().numpy()
        assert np.array_equal(got, ref.bulk_query(q)), f"answers differ at minibatch {i}"
        on += f.big_filter_stats()[0] >= 0
    assert on >= 4, "the filter never turned on"
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    assert f.kernel_stats()["order"] == 2 * s.batches
    f.sync()
