"""Serving form (cc_server_*): requests enqueued as they arrive, merged and
overlapped on the device, must give every query the same answers as running
each request alone, in arrival order, on the CPU oracle and on the plain GPU
path. Also: admission when the staging ring is small, and argument errors."""
from __future__ import annotations

import threading
import time

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


def make_trace(scale, m, seed, ulo=4, uhi=12, qlo=4, qhi=11):
    s = I.rmat_stream(scale=scale, m=m, batch=m, q=1, seed=seed)
    edges = s.all_edges()
    reqs = I.request_trace(m, rate_hz=2000.0, seed=seed, ulo=ulo, uhi=uhi, qlo=qlo, qhi=qhi)
    qtot = sum(r.size for r in reqs if r.kind == 1)
    pairs = I.uniform_pairs(s.n, qtot, seed, I.TAG_QUERIES)
    data = []
    for r in reqs:
        src = edges if r.kind == 0 else pairs
        data.append(torch.from_numpy(src[r.offset:r.offset + r.size].copy()).pin_memory())
    return s.n, reqs, data


def alone_answers(n, reqs, data):
    """Each request alone, in arrival order, on the oracle."""
    uf = oracle.OracleUF(n)
    want = {}
    for i, (r, d) in enumerate(zip(reqs, data)):
        if r.kind == 0:
            uf.bulk_update(d.numpy())
        else:
            want[i] = uf.bulk_query(d.numpy())
    return want, uf.labels()


def serve(cc, n, reqs, data, paced=False, batch=0, forest_opts=None, **cfg):
    """batch > 0: hand the requests over `batch` at a time (cc_server_enqueue_many)."""
    f = cc.Forest(n, **(forest_opts or {}))
    outs = {}
    with cc.Server(f, **cfg) as srv:
        t0 = time.perf_counter()
        pending = []
        for i, (r, d) in enumerate(zip(reqs, data)):
            if paced:
                while time.perf_counter() - t0 < r.t:
                    pass
            out = None
            if r.kind == 1:
                out = torch.zeros(r.size, dtype=torch.uint8).pin_memory()
                outs[i] = out
            if batch:
                pending.append((r.kind, d, out))
                if len(pending) == batch:
                    assert srv.enqueue_list(pending) == i + 1 - batch   # consecutive tickets
                    pending = []
            else:
                srv.enqueue(r.kind, d, out)
        if pending:
            srv.enqueue_list(pending)
        srv.drain()
        lat = srv.latencies()
        st = srv.stats()
    labels = f.labels().cpu().numpy()
    f.sync()
    return {i: o.numpy() for i, o in outs.items()}, labels, lat, st


@pytest.mark.parametrize("mode", ["burst", "paced", "no_merge", "tiny_ring", "batched_enqueue",
                                  "early_pairs_tiny_ring"])
def test_served_equals_alone(cc, mode):
    n, reqs, data = make_trace(scale=16, m=1 << 19, seed=7)
    want, want_labels = alone_answers(n, reqs, data)
    cfg = {}
    if mode == "no_merge":
        cfg = {"merge": False}
    forest_opts = None
    if mode in ("tiny_ring", "early_pairs_tiny_ring"):
        cfg = {"ring_pairs": 1 << 12, "max_group_pairs": 1 << 11}
    if mode == "early_pairs_tiny_ring":
        # the kernels read their first pairs before waiting for the previous
        # kernel (pdl 2); the ring is small, so its slots are reused constantly
        # and a read that overtook its staging copy would see another
        # request's pairs
        forest_opts = {"pdl": 2, "update_variant": 3, "edges_per_thread": 2, "compress_every": 0}
    got, labels, lat, st = serve(cc, n, reqs, data, paced=(mode == "paced"),
                                 batch=(97 if mode == "batched_enqueue" else 0), forest_opts=forest_opts,
                                 **cfg)
    for i, w in want.items():
        assert np.array_equal(got[i], w), f"request {i} differs from running it alone"
    assert np.array_equal(labels, want_labels)
    assert st["completed"] == st["requests"] == len(reqs)
    assert np.all(lat >= 0)
    if mode == "burst":
        assert st["groups"] < len(reqs)     # requests were merged
    if mode == "no_merge":
        assert st["groups"] == len(reqs)


@pytest.mark.parametrize("ring,group,merge", [(1 << 13, 1 << 11, True), (1 << 12, 1 << 9, True),
                                              (3000, 1 << 12, False), (1 << 20, 1 << 22, True)])
def test_contiguous_requests_share_copies(cc, ring, group, merge):
    # the requests' data are consecutive views of one pinned edge buffer and
    # one pinned pair buffer, and the answers consecutive views of one pinned
    # output buffer, as in a caller that keeps its stream in one place: copies
    # then run across requests and groups, in both rings, and wrap round the
    # small rings; every query answers as it would alone, in arrival order
    n, reqs, data = make_trace(scale=15, m=1 << 18, seed=12, ulo=4, uhi=10, qlo=4, qhi=10)
    e_all = torch.cat([d for r, d in zip(reqs, data) if r.kind == 0]).pin_memory()
    q_all = torch.cat([d for r, d in zip(reqs, data) if r.kind == 1]).pin_memory()
    o_all = torch.zeros(q_all.shape[0], dtype=torch.uint8).pin_memory()
    views, eo, qo = [], 0, 0
    for r in reqs:
        if r.kind == 0:
            views.append((0, e_all[eo:eo + r.size], None))
            eo += r.size
        else:
            views.append((1, q_all[qo:qo + r.size], o_all[qo:qo + r.size]))
            qo += r.size
    want, want_labels = alone_answers(n, reqs, [v[1] for v in views])
    f = cc.Forest(n)
    with cc.Server(f, ring_pairs=ring, max_group_pairs=group, merge=merge) as srv:
        srv.enqueue_list(views)
        srv.drain()
        st = srv.stats()
    for i, (kind, d, o) in enumerate(views):
        if kind == 1:
            assert np.array_equal(o.numpy(), want[i]), f"request {i}"
    assert np.array_equal(f.labels().cpu().numpy(), want_labels)
    assert st["completed"] == len(reqs) and st["groups"] >= (len(reqs) if not merge else 2)
    f.sync()


def test_empty_requests_do_not_hide_a_full_ring(cc):
    # A request of zero pairs becomes a group that sits at the ring's head
    # without occupying it. With no merging (one group per request) and a
    # ring a few groups long, such a group is often the oldest in flight
    # while later groups wrap all the way round to its position; the ring is
    # then full, not empty, and a new group must wait. Every answer and the
    # final labels must still match the oracle run request by request.
    n, reqs, data = make_trace(scale=14, m=1 << 17, seed=10, ulo=4, uhi=9, qlo=4, qhi=9)
    rng = np.random.default_rng(10)
    Req = type(reqs[0])
    reqs2, data2 = [], []
    for r, d in zip(reqs, data):
        if rng.random() < 0.3:
            kind = int(rng.integers(0, 2))
            reqs2.append(Req(r.t, kind, 0, 0))
            data2.append(torch.zeros((0, 2), dtype=torch.int32).pin_memory())
        reqs2.append(r)
        data2.append(d)
    want, want_labels = alone_answers(n, reqs2, data2)
    for ring in (1 << 10, 1536):
        got, labels, _, st = serve(cc, n, reqs2, data2, merge=False, ring_pairs=ring,
                                   max_group_pairs=1 << 9)
        for i, w in want.items():
            assert np.array_equal(got[i], w), f"ring {ring}: request {i} differs from running it alone"
        assert np.array_equal(labels, want_labels)
        assert st["completed"] == st["requests"] == len(reqs2)


def test_served_equals_plain_gpu_alone(cc):
    n, reqs, data = make_trace(scale=14, m=1 << 16, seed=8)
    got, labels, _, _ = serve(cc, n, reqs, data)
    f = cc.Forest(n)
    for i, (r, d) in enumerate(zip(reqs, data)):
        if r.kind == 0:
            f.bulk_update(d.cuda())
        else:
            assert np.array_equal(f.bulk_query(d.cuda()).cpu().numpy(), got[i]), i
    assert np.array_equal(f.labels().cpu().numpy(), labels)


def test_concurrent_producers_keep_each_thread_order(cc):
    # two client threads enqueue interleaved; the server's ticket order is the
    # arrival order, and the answers match the oracle run in that order
    n, reqs, data = make_trace(scale=14, m=1 << 17, seed=9)
    f = cc.Forest(n)
    tickets = [None] * len(reqs)
    outs = {}
    lock = threading.Lock()
    with cc.Server(f) as srv:
        def producer(idx):
            for i in idx:
                r, d = reqs[i], data[i]
                out = torch.zeros(r.size, dtype=torch.uint8).pin_memory() if r.kind else None
                with lock:
                    tickets[i] = srv.enqueue(r.kind, d, out)
                    if out is not None:
                        outs[i] = out
        th = [threading.Thread(target=producer, args=(list(range(j, len(reqs), 2)),)) for j in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        srv.drain()
    order = sorted(range(len(reqs)), key=lambda i: tickets[i])
    uf = oracle.OracleUF(n)
    for i in order:
        if reqs[i].kind == 0:
            uf.bulk_update(data[i].numpy())
        else:
            assert np.array_equal(outs[i].numpy(), uf.bulk_query(data[i].numpy())), i


def test_server_errors(cc):
    f = cc.Forest(100)
    with cc.Server(f, ring_pairs=64) as srv:
        big = torch.zeros((65, 2), dtype=torch.int32)
        with pytest.raises(cc.CCError) as ex:
            srv.enqueue(cc.OP_UPDATE, big)
        assert ex.value.status == cc.CC_ERR_ARG
        with pytest.raises(TypeError):
            srv.enqueue(cc.OP_QUERY, torch.zeros((3, 2), dtype=torch.int32), None)
        t = srv.enqueue(cc.OP_UPDATE, torch.zeros((0, 2), dtype=torch.int32))
        assert srv.wait(t) >= 0
    # the handle is usable again after the server is gone
    f.bulk_update(torch.tensor([[1, 2]], dtype=torch.int32, device="cuda"))
    assert f.components() == 99


def test_enqueue_many_checks_everything_first(cc):
    f = cc.Forest(100)
    e = torch.tensor([[1, 2], [3, 4]], dtype=torch.int32).pin_memory()
    q = torch.tensor([[1, 2]], dtype=torch.int32).pin_memory()
    o = torch.zeros(1, dtype=torch.uint8).pin_memory()
    with cc.Server(f) as srv:
        kinds = np.array([cc.OP_UPDATE, cc.OP_QUERY, 7], dtype=np.int32)     # request 2: bad kind
        ptrs = np.array([e.data_ptr(), q.data_ptr(), e.data_ptr()], dtype=np.uint64)
        ks = np.array([2, 1, 2], dtype=np.int64)
        outs = np.array([0, o.data_ptr(), 0], dtype=np.uint64)
        with pytest.raises(cc.CCError) as ex:
            srv.enqueue_many(kinds, ptrs, ks, outs)
        assert ex.value.status == cc.CC_ERR_ARG and "request 2" in str(ex.value)
        assert srv.stats()["requests"] == 0                    # nothing was accepted
        with pytest.raises(cc.CCError):                        # a query without an output
            srv.enqueue_many(kinds[:2], ptrs[:2], ks[:2], None)
        assert srv.stats()["requests"] == 0
        first = srv.enqueue_many(kinds[:2], ptrs[:2], ks[:2], outs[:2], keep=(e, q, o))
        assert first == 0
        srv.drain()
        assert srv.stats()["completed"] == 2 and o[0] == 1     # 1-2 joined by the update before it
    f.close()


def test_full_size_served_trace_equals_oracle(cc):
    # The served workload exactly as the benchmark serves it: R-MAT n = 2^26,
    # 2^30 edges, Poisson request trace (updates of log-uniform [2^8, 2^20]
    # edges, queries of log-uniform [2^8, 2^18] pairs, 3:1), all requests handed
    # over in one call, the tuned serving options and the default staging ring
    # and group sizes. Every query request's answers, and the final labels,
    # must equal the oracle's with the requests applied one by one in arrival
    # order (a query sees exactly the updates before it).
    from bench import ServingTrace, launch_options
    tr = ServingTrace(26, seed=0)
    f = cc.Forest(tr.n, **launch_options("serving"))
    with cc.Server(f) as srv:
        srv.enqueue_many(*tr.many)
        srv.drain()
        st = srv.stats()
    labels = f.labels().cpu().numpy()
    f.sync()
    f.close()
    assert st["completed"] == st["requests"] == len(tr.reqs)
    assert st["groups"] < len(tr.reqs)
    uf = oracle.OracleUF(tr.n)
    edges, pairs, got = tr.h_edges.numpy(), tr.h_pairs.numpy(), tr.h_out.numpy()
    for i, r in enumerate(tr.reqs):
        if r.kind == 0:
            uf.bulk_update(edges[r.offset:r.offset + r.size])
        else:
            want = uf.bulk_query(pairs[r.offset:r.offset + r.size])
            assert np.array_equal(got[r.offset:r.offset + r.size], want), f"request {i} differs"
    assert np.array_equal(labels, uf.labels())
