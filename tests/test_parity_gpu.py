"""CUDA path (through the C-ABI) against the CPU oracle: bit-exact answers,
minimum-id labels and component counts, on seeded streams, edge cases, and
the full-size R-MAT and grid streams in the benchmark's launch configuration.

Parent forests are not unique (link rules differ), so parity is checked on
what is: every query answer and every canonical label. Forest invariants
(parent[v] <= v, entries never increase, roots are component minima) are
checked on the raw parent array.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1602_05232_gb300 import inputs as I

pytestmark = pytest.mark.gpu

OPTION_SETS = {
    "default": {},
    "ept1_b64": {"edges_per_thread": 1, "block": 64},
    "ept4_b1024": {"edges_per_thread": 4, "block": 1024},
    "no_compress": {"compress_every": 0},
    "no_compress_halving_query": {"compress_every": 0, "query_halving": 1},
    "touched_compress": {"compress_scope": 1},
    "compress_every3": {"compress_every": 3},
    "lockstep": {"update_variant": 1},
    "lockstep_ept4_nocompress": {"update_variant": 1, "edges_per_thread": 4, "compress_every": 0},
    "persistent_ept4": {"update_variant": 2, "edges_per_thread": 4},
    "persistent_ept1_b1024": {"update_variant": 2, "edges_per_thread": 1, "block": 1024},
    "l2_persist": {"l2_persist": 1, "update_variant": 2, "edges_per_thread": 2},
    "persistent_query": {"query_variant": 1, "compress_every": 0, "edges_per_thread": 4},
    "persistent_query_halving": {"query_variant": 1, "compress_every": 0, "query_halving": 1},
    "persistent_query_flat": {"query_variant": 1, "compress_every": 1, "block": 1024},
    "splitting_query": {"query_halving": 2, "compress_every": 0, "edges_per_thread": 4},
    "splitting_query_persistent": {"query_halving": 2, "compress_every": 0, "query_variant": 1},
    "pdl_off": {"pdl": 0},
    "min_hook": {"hook": 1},
    "min_hook_persistent": {"hook": 1, "update_variant": 2, "edges_per_thread": 4, "compress_every": 0},
    "min_hook_deep": {"hook": 1, "update_variant": 3, "edges_per_thread": 2, "block": 128, "compress_every": 0,
                      "query_pairs_per_thread": 2, "l2_persist": 1},
    "min_hook_two_pass": {"hook": 1, "update_variant": 4, "edges_per_thread": 1, "compress_every": 3},
    "min_hook_first_only": {"hook": 2, "update_variant": 3, "edges_per_thread": 2, "compress_every": 0},
    "min_hook_first_only_two_pass": {"hook": 2, "update_variant": 4, "edges_per_thread": 2, "compress_every": 0},
    "two_pass_ept4": {"update_variant": 4, "edges_per_thread": 4, "compress_every": 0},
    "two_pass_ept1_pdl0": {"update_variant": 4, "edges_per_thread": 1, "pdl": 0, "compress_every": 2},
    "two_pass_ept2_pdl2_b1024": {"update_variant": 4, "edges_per_thread": 2, "pdl": 2, "block": 1024,
                                 "compress_every": 0, "query_pairs_per_thread": 4},
    "query_ept2_update_ept4": {"edges_per_thread": 4, "query_pairs_per_thread": 2, "compress_every": 0,
                               "update_variant": 2, "pdl": 2},
    "query_ept1_halving": {"query_pairs_per_thread": 1, "query_halving": 1, "compress_every": 0},
    "deep_prefetch_ept4": {"update_variant": 3, "edges_per_thread": 4, "compress_every": 0},
    "deep_prefetch_ept2_pdl2": {"update_variant": 3, "edges_per_thread": 2, "compress_every": 0, "pdl": 2},
    "deep_prefetch_ept1_b1024": {"update_variant": 3, "edges_per_thread": 1, "block": 1024, "compress_every": 3},
    "pdl_early_persistent": {"pdl": 2, "update_variant": 2, "edges_per_thread": 4, "compress_every": 0,
                             "query_halving": 1},
    "pdl_early_query_persistent": {"pdl": 2, "query_variant": 1, "compress_every": 0, "l2_persist": 1},
    "pdl_early_ept1": {"pdl": 2, "update_variant": 1, "edges_per_thread": 1, "compress_every": 2},
    "order8": {"edge_order": 8},
    "order6": {"edge_order": 6, "pdl": 2, "compress_every": 0},
    "order9_persistent_pdl2": {"edge_order": 9, "update_variant": 2, "edges_per_thread": 1, "block": 128,
                                "pdl": 2, "compress_every": 2},
    "order7_deep_min_hook": {"edge_order": 7, "update_variant": 3, "edges_per_thread": 2, "hook": 2,
                              "pdl": 2, "compress_every": 0},
    "order9_two_pass": {"edge_order": 9, "update_variant": 4, "edges_per_thread": 2, "pdl": 2,
                         "compress_every": 4},
    "order8_paper_schedule": {"edge_order": 8, "update_schedule": 1},
    "warp_hook_lockstep": {"hook_warp": 1, "update_variant": 1, "edges_per_thread": 2, "block": 96},
    "warp_hook_persistent_min": {"hook_warp": 1, "hook": 1, "update_variant": 2, "edges_per_thread": 4,
                                 "compress_every": 0},
    "warp_hook_deep_first_min": {"hook_warp": 1, "hook": 2, "update_variant": 3, "edges_per_thread": 2,
                                 "block": 512, "compress_every": 0, "pdl": 2},
    "warp_hook_deep_ept1": {"hook_warp": 1, "update_variant": 3, "edges_per_thread": 1, "block": 128,
                            "compress_every": 2},
    "warp_hook_two_pass": {"hook_warp": 1, "update_variant": 4, "edges_per_thread": 2, "compress_every": 0},
    "warp_hook_two_pass_min": {"hook_warp": 1, "hook": 1, "update_variant": 4, "edges_per_thread": 1},
    "warp_hook_ordered": {"hook_warp": 1, "edge_order": 8, "update_variant": 2, "edges_per_thread": 1,
                          "block": 128, "compress_every": 4},
    "warp_hook_per_edge_ignored": {"hook_warp": 1, "update_variant": 0},
    "cta_list_ept1_b128": {"update_variant": 5, "edges_per_thread": 1, "block": 128, "compress_every": 0},
    "cta_list_ept2_min": {"update_variant": 5, "edges_per_thread": 2, "hook": 1, "pdl": 2, "compress_every": 2},
    "cta_list_ept4_b1024": {"update_variant": 5, "edges_per_thread": 4, "block": 1024, "hook": 2,
                            "compress_every": 0},
    "cta_list_ordered": {"update_variant": 5, "edges_per_thread": 2, "edge_order": 9, "compress_every": 4},
    "warp_query": {"query_variant": 2, "compress_every": 0},
    "warp_query_flat_b1024": {"query_variant": 2, "compress_every": 1, "block": 1024},
    "warp_query_halving_ignored_pdl2": {"query_variant": 2, "query_halving": 1, "compress_every": 3, "pdl": 2,
                                        "block": 64},
    # largest-component filter: the bitmap written by full compressions
    "big_default": {"big_filter": 256},
    "big_every1_flat_query": {"big_filter": 1, "compress_every": 1},
    "big_cta_list_ordered_min": {"big_filter": 128, "update_variant": 5, "edges_per_thread": 2, "edge_order": 7,
                                 "compress_every": 2, "hook": 1, "pdl": 2},
    "big_cta_list_ept1": {"big_filter": 1, "update_variant": 5, "edges_per_thread": 1, "block": 128,
                          "compress_every": 3},
    "big_persistent_query_halving": {"big_filter": 64, "query_variant": 1, "query_halving": 1, "compress_every": 3},
    "big_splitting_query": {"big_filter": 64, "query_halving": 2, "compress_every": 2, "update_variant": 2,
                            "edges_per_thread": 1},
    "big_deep_pdl2": {"big_filter": 32, "update_variant": 3, "edges_per_thread": 4, "pdl": 2, "compress_every": 2},
    "big_two_pass": {"big_filter": 16, "update_variant": 4, "edges_per_thread": 2, "compress_every": 2},
    "big_lockstep_warp_hook": {"big_filter": 1, "update_variant": 1, "hook_warp": 1, "compress_every": 1,
                               "edges_per_thread": 4},
    "big_per_edge_query_ept4": {"big_filter": 1, "update_variant": 0, "compress_every": 2,
                                "query_pairs_per_thread": 4},
    "big_warp_query": {"big_filter": 1, "query_variant": 2, "compress_every": 1},
    "big_all_samples": {"big_filter": 1024, "compress_every": 1},
    "big_touched_scope_never_built": {"big_filter": 1, "compress_scope": 1},
    # with the edge order: the order is skipped and the caller's edges read while the bitmap is in use
    "big_ordered_lockstep_every1": {"big_filter": 1, "edge_order": 6, "update_variant": 1, "compress_every": 1},
    "big_ordered_two_pass": {"big_filter": 1, "edge_order": 9, "update_variant": 4, "compress_every": 2},
    "big_ordered_deep_pdl2": {"big_filter": 1, "edge_order": 8, "update_variant": 3, "edges_per_thread": 2,
                              "pdl": 2, "compress_every": 2},
    "big_ordered_persistent_ept1": {"big_filter": 64, "edge_order": 7, "update_variant": 2, "edges_per_thread": 1,
                                    "block": 512, "compress_every": 3, "pdl": 2},
    "big_ordered_paper_schedule": {"big_filter": 1, "edge_order": 8, "update_schedule": 1, "compress_every": 2},
    "big_ordered_touched_scope": {"big_filter": 1, "edge_order": 7, "compress_scope": 1, "compress_every": 2},
}


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05232_gb300 import _build, cc as ccmod
    _build.build_cc()
    ccmod.load()
    return ccmod


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_stream(cc, stream, options, label_every=1, check_invariants=False):
    f = cc.Forest(stream.n, **options)
    ref = oracle.OracleUF(stream.n)
    prev_parent = None
    for i, (e, q) in enumerate(stream):
        f.bulk_update(dev(e))
        got = f.bulk_query(dev(q)).cpu().numpy()
        ref.bulk_update(e)
        want = ref.bulk_query(q)
        assert np.array_equal(got, want), f"answers differ at batch {i}: " \
            f"{int((got != want).sum())} of {len(want)}"
        if check_invariants:
            par = f.parent().cpu().numpy()
            assert np.all(par <= np.arange(stream.n)), "parent[v] > v"
            if prev_parent is not None:
                assert np.all(par <= prev_parent), "a parent entry increased"
            prev_parent = par
        if label_every and (i % label_every == 0 or i == stream.batches - 1):
            lab = f.labels().cpu().numpy()
            assert np.array_equal(lab, ref.labels()), f"labels differ at batch {i}"
            assert f.components() == ref.components, f"components differ at batch {i}"
            if check_invariants:
                par = f.parent().cpu().numpy()
                roots = np.flatnonzero(par == np.arange(stream.n))
                assert np.array_equal(lab[roots], roots), "a root is not its component minimum"
    f.sync()
    f.close()
    return ref


@pytest.mark.parametrize("opts", list(OPTION_SETS), ids=list(OPTION_SETS))
def test_uniform_small_every_batch(cc, opts):
    # n = 2^16, 16 minibatches of 2^16 uniform edges, 2^16 queries after each
    run_stream(cc, I.uniform_stream(), OPTION_SETS[opts], label_every=1,
               check_invariants=(opts == "default"))


@pytest.mark.parametrize("opts", ["default", "ept1_b64", "no_compress", "touched_compress",
                                  "lockstep_ept4_nocompress", "persistent_ept4",
                                  "persistent_query_halving", "splitting_query", "deep_prefetch_ept2_pdl2",
                                  "two_pass_ept4", "query_ept2_update_ept4", "min_hook", "min_hook_persistent",
                                  "min_hook_deep", "min_hook_two_pass", "min_hook_first_only", "order8",
                                  "order6", "order7_deep_min_hook", "order8_paper_schedule",
                                  "warp_hook_lockstep", "warp_hook_persistent_min", "warp_hook_deep_first_min",
                                  "warp_hook_two_pass", "warp_hook_ordered", "warp_query", "cta_list_ept1_b128",
                                  "cta_list_ept2_min", "cta_list_ept4_b1024",
                                  "warp_query_halving_ignored_pdl2", "big_default", "big_every1_flat_query",
                                  "big_cta_list_ordered_min", "big_persistent_query_halving", "big_deep_pdl2",
                                  "big_two_pass", "big_lockstep_warp_hook", "big_ordered_two_pass",
                                  "big_ordered_paper_schedule"])
def test_rmat_small(cc, opts):
    s = I.rmat_stream(scale=16, m=1 << 20, batch=(1 << 16) + 3, q=(1 << 16) - 5, seed=1)
    run_stream(cc, s, OPTION_SETS[opts], label_every=4, check_invariants=True)


@pytest.mark.parametrize("opts", ["default", "no_compress", "ept4_b1024", "compress_every3",
                                  "lockstep", "persistent_ept1_b1024", "splitting_query",
                                  "deep_prefetch_ept1_b1024", "two_pass_ept1_pdl0", "min_hook",
                                  "min_hook_deep", "order8", "order9_persistent_pdl2", "order9_two_pass",
                                  "warp_hook_deep_ept1", "warp_hook_two_pass_min", "warp_hook_ordered",
                                  "warp_query", "warp_query_flat_b1024", "cta_list_ept1_b128", "cta_list_ordered",
                                  "big_default", "big_every1_flat_query", "big_cta_list_ordered_min",
                                  "big_cta_list_ept1", "big_splitting_query", "big_per_edge_query_ept4",
                                  "big_warp_query", "big_all_samples", "big_ordered_lockstep_every1",
                                  "big_ordered_two_pass", "big_ordered_deep_pdl2", "big_ordered_persistent_ept1",
                                  "big_ordered_paper_schedule", "big_ordered_touched_scope"])
def test_grid_small(cc, opts):
    s = I.grid_stream(512, 512, batch=(1 << 14) + 1, q=1 << 14, seed=2)
    ref = run_stream(cc, s, OPTION_SETS[opts], label_every=8, check_invariants=True)
    assert ref.components == 1


def test_edge_cases(cc):
    n = 1000
    f = cc.Forest(n)
    ref = oracle.OracleUF(n)

    def both(e):
        e = np.asarray(e, dtype=np.int32).reshape(-1, 2)
        f.bulk_update(dev(e))
        ref.bulk_update(e)

    both(np.zeros((0, 2)))                       # empty minibatch
    both([[5, 9]])                               # k = 1
    both([[1, 2], [3, 4], [5, 6]])               # odd k
    both([[7, 7]] * 17)                          # only self-loops
    both([[10, 11]] * 33 + [[11, 10]] * 31)      # duplicates both ways
    both([[999, i] for i in range(100, 400)])    # star into a high-id hub
    both([[0, i] for i in range(400, 700)])      # star into a low-id hub
    both([[i, i - 1] for i in range(999, 900, -1)])  # descending path
    q = np.random.default_rng(0).integers(0, n, size=(20000, 2)).astype(np.int32)
    assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q))
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    assert f.components() == ref.components
    empty = f.bulk_query(dev(np.zeros((0, 2), dtype=np.int32)))
    assert empty.numel() == 0
    f.sync()


def test_unaligned_arrays(cc):
    # pair arrays starting 8 and 4 bytes past a 16-byte boundary, odd lengths
    s = I.uniform_stream(n=5000, m=40001, batch=40001, q=30001, seed=3)
    e, q = s.edges(0), s.queries(0)
    ref = oracle.OracleUF(s.n)
    ref.bulk_update(e)
    want = ref.bulk_query(q)
    for shift in (2, 1):   # in int32 elements: 8 bytes, 4 bytes
        for ept in (1, 2, 4):
            f = cc.Forest(s.n, edges_per_thread=ept)
            buf = torch.zeros(e.size + 4, dtype=torch.int32, device="cuda")
            buf[shift:shift + e.size] = dev(e.ravel())
            f.bulk_update(buf[shift:shift + e.size])
            qb = torch.zeros(q.size + 4, dtype=torch.int32, device="cuda")
            qb[shift:shift + q.size] = dev(q.ravel())
            out = torch.zeros(len(q) + 3, dtype=torch.uint8, device="cuda")
            f.bulk_query(qb[shift:shift + q.size], out=out[1:1 + len(q)])
            assert np.array_equal(out[1:1 + len(q)].cpu().numpy(), want), (shift, ept)
            lab = torch.zeros(s.n + 1, dtype=torch.int32, device="cuda")
            f.labels(out=lab[1:])
            assert np.array_equal(lab[1:].cpu().numpy(), ref.labels())
            f.sync()


def test_out_of_range_ids(cc):
    n = 100
    f = cc.Forest(n)
    ref = oracle.OracleUF(n)
    e = np.array([[0, 1], [-1, 2], [2, n], [3, 4], [2**31 - 1, 5], [5, 6]], dtype=np.int32)
    f.bulk_update(dev(e))
    ref.bulk_update(e)
    with pytest.raises(cc.CCError) as ex:
        f.sync()
    assert ex.value.status == cc.CC_ERR_RANGE
    f.sync()  # the status word was cleared
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    q = np.array([[0, 1], [n, n], [-5, 0], [3, 4]], dtype=np.int32)
    assert f.bulk_query(dev(q)).cpu().numpy().tolist() == ref.bulk_query(q).tolist() == [1, 0, 0, 1]
    with pytest.raises(cc.CCError):
        f.sync()


@pytest.mark.parametrize("log_buckets", [6, 8, 9])
def test_edge_order_ragged_sizes_and_bad_ids(cc, log_buckets):
    # minibatch sizes around the ordering threshold (4096 edges) and around
    # the per-CTA chunk granularity, with ids outside [0, n) among the edges:
    # the ordered copy holds every edge once, bad ones are skipped and
    # reported, and answers and labels match the oracle
    n = 70001
    rng = np.random.default_rng(log_buckets)
    f = cc.Forest(n, edge_order=log_buckets, compress_every=0)
    ref = oracle.OracleUF(n)
    launches0 = f.kernel_stats()["order"]
    ordered = 0
    for k in (4095, 4096, 4097, 2047 * 4 + 3, 100003, 262145):
        e = rng.integers(0, n, size=(k, 2)).astype(np.int32)
        e[rng.integers(0, k, size=5), rng.integers(0, 2, size=5)] = [-1, n, 2**31 - 1, -7, n + 5]
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        ordered += k >= 4096
        with pytest.raises(cc.CCError) as ex:
            f.sync()
        assert ex.value.status == cc.CC_ERR_RANGE
        q = rng.integers(0, n, size=(30011, 2)).astype(np.int32)
        assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q)), k
    assert f.kernel_stats()["order"] - launches0 == 2 * ordered      # count, scatter
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    assert f.components() == ref.components
    f.sync()


@pytest.mark.parametrize("hub", ["first", "last"])
def test_edge_order_with_every_edge_in_one_bucket(cc, hub):
    # a star minibatch whose smaller endpoints all fall into one bucket (hub 0:
    # every edge in bucket 0; hub n-1: the other endpoints spread, then a
    # second star with every edge inside the last bucket's id range)
    n = 1 << 20
    rng = np.random.default_rng(7)
    f = cc.Forest(n, edge_order=9, update_variant=2, edges_per_thread=1, block=128, hook=1,
                  compress_every=0)
    ref = oracle.OracleUF(n)
    h = 0 if hub == "first" else n - 1
    others = rng.integers(0, n, size=300000).astype(np.int32)
    e1 = np.stack([np.full_like(others, h), others], 1)
    lo = n - (n >> 9)                                      # the last bucket's first id
    tail = rng.integers(lo, n, size=50000).astype(np.int32)
    e2 = np.stack([tail, np.roll(tail, 1)], 1)
    for e in (e1, e2):
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        q = rng.integers(0, n, size=(100000, 2)).astype(np.int32)
        assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q))
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    f.sync()


def test_argument_errors_leave_state(cc):
    f = cc.Forest(10)
    with pytest.raises(TypeError):
        f.bulk_update(torch.zeros(4, dtype=torch.int64, device="cuda"))
    with pytest.raises(cc.CCError) as ex:
        f.set_option("block", 100)
    assert ex.value.status == cc.CC_ERR_ARG
    with pytest.raises(cc.CCError):
        f.set_option("edges_per_thread", 3)
    assert f.get_option("block") == 256
    assert f.components() == 10


# (option, rejected values, accepted values): include/cc.h gives the ranges
OPTION_RANGES = [
    ("block", [0, 63, 100, 1056], [64, 1024]),
    ("edges_per_thread", [0, 3, 8], [1, 2, 4]),
    ("compress_every", [-1], [0, 16]),
    ("compress_scope", [2, -1], [0, 1]),
    ("query_halving", [-1, 3], [0, 1, 2]),
    ("profile", [2], [0, 1]),
    ("update_variant", [-1, 6], [0, 1, 2, 3, 4, 5]),
    ("query_variant", [-1, 3], [0, 1, 2]),
    ("pdl", [-1, 3], [0, 1, 2]),
    ("query_pairs_per_thread", [3, 8], [0, 1, 2, 4]),
    ("hook", [-1, 3], [0, 1, 2]),
    ("bulk_find", [2], [0, 1]),
    ("update_schedule", [2], [0, 1]),
    ("sv_graph", [-1, 2], [0, 1]),
    ("edge_order", [-1, 1, 5, 10], [0, 6, 9]),
    ("hook_warp", [-1, 2], [0, 1]),
    ("big_filter", [-1, 1025], [0, 1, 1024]),
]


@pytest.mark.parametrize("name,bad,good", OPTION_RANGES, ids=[o[0] for o in OPTION_RANGES])
def test_option_ranges(cc, name, bad, good):
    f = cc.Forest(100)
    before = f.get_option(name)
    for v in bad:
        with pytest.raises(cc.CCError) as ex:
            f.set_option(name, v)
        assert ex.value.status == cc.CC_ERR_ARG
        assert f.get_option(name) == before          # a rejected value changes nothing
    for v in good:
        f.set_option(name, v)
        assert f.get_option(name) == v
    f.close()


def _cudart():
    import ctypes
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("no CUDA runtime library to query the limit with")


def test_l2_persist_gives_back_the_limit_and_lines(cc):
    # handles with l2_persist raise the context's persisting-L2 limit (to their
    # forest size, capped by the device maximum); when the last one leaves
    # (option off or destroyed) the limit found before is back, so later
    # kernels of the process get the whole L2 again
    import ctypes
    rt = _cudart()
    PERSISTING_L2 = 6            # cudaLimitPersistingL2CacheSize
    ATTR_MAX_PERSISTING = 108    # cudaDevAttrMaxPersistingL2CacheSize

    def limit():
        v = ctypes.c_size_t()
        assert rt.cudaDeviceGetLimit(ctypes.byref(v), PERSISTING_L2) == 0
        return v.value

    torch.zeros(1, device="cuda")
    mx = ctypes.c_int()
    assert rt.cudaDeviceGetAttribute(ctypes.byref(mx), ATTR_MAX_PERSISTING, torch.cuda.current_device()) == 0
    before = limit()
    can_raise = mx.value > before
    f = cc.Forest(1 << 25, l2_persist=1)         # 128 MiB forest: asks for the device maximum
    g = cc.Forest(1 << 18, l2_persist=1)
    raised = limit()
    assert raised >= before and (raised > before) == can_raise
    f.bulk_update(dev(I.uniform_pairs(1 << 25, 1 << 16, seed=1, tag=I.TAG_EDGES)))
    f.sync()
    f.close()
    assert limit() == raised                     # g still has its window
    g.set_option("l2_persist", 1)                # already on: no second claim
    g.set_option("l2_persist", 0)
    assert limit() == before
    h = cc.Forest(1 << 25, l2_persist=1)
    assert limit() == raised
    h.close()
    g.close()
    assert limit() == before


def test_checkpoint_resume(cc):
    s = I.rmat_stream(scale=14, m=1 << 17, batch=1 << 13, q=1 << 12, seed=4)
    whole = cc.Forest(s.n)
    first = cc.Forest(s.n)
    cut = 7
    for i, (e, q) in enumerate(s):
        whole.bulk_update(dev(e))
        if i < cut:
            first.bulk_update(dev(e))
    saved = first.labels()
    resumed = cc.Forest(s.n)
    resumed.load_labels(saved)
    assert resumed.components() == first.components()
    for i in range(cut, s.batches):
        resumed.bulk_update(dev(s.edges(i)))
    assert torch.equal(resumed.labels(), whole.labels())
    assert resumed.components() == whole.components()
    q = dev(s.all_queries())
    assert torch.equal(resumed.bulk_query(q), whole.bulk_query(q))
    # an invalid labelling is refused and the forest is left as it was
    before = resumed.labels().clone()
    bad = before.clone()
    bad[5] = 7   # label above the vertex id
    with pytest.raises(cc.CCError) as ex:
        resumed.load_labels(bad)
    assert ex.value.status == cc.CC_ERR_LABELS
    assert torch.equal(resumed.labels(), before)


def test_non_default_stream_and_touched_compress_api(cc):
    st = torch.cuda.Stream()
    s = I.uniform_stream(n=1 << 14, m=1 << 16, batch=1 << 13, q=1 << 13, seed=5)
    ref = oracle.OracleUF(s.n)
    with torch.cuda.stream(st):
        f = cc.Forest(s.n, compress_every=0)
        for e, q in s:
            de, dq = dev(e), dev(q)
            f.bulk_update(de)
            f.compress("touched", de)
            got = f.bulk_query(dq)
            ref.bulk_update(e)
            assert np.array_equal(got.cpu().numpy(), ref.bulk_query(q))
        f.compress("all")
        assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    st.synchronize()


def test_kernel_counters_and_profile(cc):
    f = cc.Forest(1 << 12, profile=1)
    e = dev(I.uniform_pairs(1 << 12, 5000, seed=0, tag=1))
    f.bulk_update(e)
    f.bulk_query(e)
    st = f.kernel_stats(timing=True)
    assert st["update"][0] == 1 and st["compress_all"][0] == 1 and st["query"][0] == 1
    assert st["update"][1] > 0 and st["query"][1] > 0


# ----------------------------------------------------------- full sizes

def _full_stream(cc, s, options, label_batches):
    """Whole stream through the GPU and the oracle; every answer compared."""
    f = cc.Forest(s.n, **options)
    ref = oracle.OracleUF(s.n)
    for i in range(s.batches):
        e, q = s.edges(i), s.queries(i)
        f.bulk_update(dev(e))
        got = f.bulk_query(dev(q))
        ref.bulk_update(e)
        want = ref.bulk_query(q)
        assert np.array_equal(got.cpu().numpy(), want), f"answers differ at batch {i}"
        if i in label_batches:
            assert np.array_equal(f.labels().cpu().numpy(), ref.labels()), f"labels at {i}"
    f.sync()
    return f, ref


def test_full_size_rmat_stream(cc):
    # R-MAT scale 24 (n = 2^24), 2^27 edges in 128 minibatches of 2^20, 2^20
    # queries after each: every answer and the final labels against the oracle
    from bench import launch_options
    s = I.rmat_stream()
    f, ref = _full_stream(cc, s, launch_options("rmat"), label_batches={0, 63, s.batches - 1})
    assert f.components() == ref.components


def test_full_size_grid_stream(cc):
    # 8192 x 8192 grid, shuffled, minibatches of 2^22 with 2^22 queries each
    from bench import launch_options
    s = I.grid_stream()
    f, ref = _full_stream(cc, s, launch_options("grid"), label_batches={0, s.batches // 2})
    lab = f.labels()
    assert int(lab.max()) == 0 and f.components() == 1 == ref.components


def test_uniform_stream_at_the_benchmarked_options(cc):
    # n = 2^16, 16 minibatches of 2^16 uniform edges, 2^16 queries after each,
    # at the options the benchmark's uniform form times: every answer and the
    # labels after every minibatch
    from bench import launch_options
    run_stream(cc, I.uniform_stream(), launch_options("uniform"), label_every=1)


def test_paper_scale_random_stream_component_curve(cc):
    # 10^8 vertices, 5x10^8 uniform edges in minibatches of 10^7 (the paper's
    # largest batch, Table 3): component count after every minibatch (the
    # Figure 2 curve) and the final labels against the oracle
    from bench import launch_options
    s = I.paper_stream("random", batch=10_000_000, q=1)
    f = cc.Forest(s.n, **launch_options("paper-random"))
    ref = oracle.OracleUF(s.n)
    for i in range(s.batches):
        e = s.edges(i)
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        assert f.components() == ref.components, f"component count at minibatch {i}"
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    f.sync()


def test_paper_scale_3dgrid_stream_component_curve(cc):
    # the 464^3 mesh (99.9 M vertices, 299 M edges) in minibatches of 10^7 at
    # its tuned options: edge order, update variant 5, the largest-component
    # filter, which turns the order off once it marks a tree. Component count
    # after every minibatch and the final labels against the oracle
    from bench import launch_options
    s = I.paper_stream("3dgrid", batch=10_000_000, q=1)
    opts = launch_options("paper-3dgrid")
    f = cc.Forest(s.n, **opts)
    ref = oracle.OracleUF(s.n)
    on = 0
    for i in range(s.batches):
        e = s.edges(i)
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        assert f.components() == ref.components, f"component count at minibatch {i}"
        on += opts.get("big_filter", 0) > 0 and f.big_filter_stats()[0] >= 0
    assert np.array_equal(f.labels().cpu().numpy(), ref.labels())
    if opts.get("big_filter", 0) > 0:
        assert on > 0, "the filter never turned on"
    f.sync()


def test_single_vertex_forest(cc):
    f = cc.Forest(1)
    f.bulk_update(dev(np.array([[0, 0]], dtype=np.int32)))
    assert f.bulk_query(dev(np.array([[0, 0]], dtype=np.int32))).cpu().tolist() == [1]
    assert f.labels().cpu().tolist() == [0] and f.components() == 1
    f.sync()


def test_maximum_vertex_count(cc):
    # n = 2^31 - 1, the largest the int32 ids allow: an 8 GiB forest; edges at
    # both ends of the id range, checked through answers and component counts
    n = 2**31 - 1
    f = cc.Forest(n, **{"compress_every": 1})
    e = np.array([[n - 1, n - 2], [0, n - 1], [1 << 30, (1 << 30) + 1], [n - 3, n - 3]], dtype=np.int32)
    f.bulk_update(dev(e))
    assert f.components() == n - 3
    q = np.array([[0, n - 2], [n - 2, n - 1], [1, n - 1], [1 << 30, (1 << 30) + 1], [n - 3, n - 3]],
                 dtype=np.int32)
    assert f.bulk_query(dev(q)).cpu().tolist() == [1, 1, 0, 1, 1]
    par = f.parent()
    assert int(par[n - 1]) == 0 and int(par[n - 2]) == 0
    f.sync()
    f.close()
