"""Union by size (CC_OPT_LINK = 1, the paper's link rule, with the paper's
schedule) against the CPU oracle, and Lemma 1's height bound: every tree of
a union-by-size forest is at most floor(log2 n) high."""
from __future__ import annotations

import math

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(cc, s, options, label_every=1):
    f = cc.Forest(s.n, update_schedule=1, link=1, **options)
    ref = oracle.OracleUF(s.n)
    height_bound = int(math.floor(math.log2(s.n)))
    for i, (e, q) in enumerate(s):
        f.bulk_update(dev(e))
        ref.bulk_update(e)
        assert np.array_equal(f.bulk_query(dev(q)).cpu().numpy(), ref.bulk_query(q)), i
        mx, _ = f.depth()
        assert mx <= height_bound, f"height {mx} above log2 n at minibatch {i}"
        if i % label_every == 0 or i == s.batches - 1:
            assert np.array_equal(f.labels().cpu().numpy(), ref.labels()), i
            assert f.components() == ref.components
    f.sync()
    return f


@pytest.mark.parametrize("opts", [{"compress_every": 0}, {"compress_every": 1}, {"compress_every": 4}])
def test_size_uniform(cc, opts):
    run(cc, I.uniform_stream(), opts)


def test_size_rmat_grid_hub(cc):
    run(cc, I.rmat_stream(scale=16, m=1 << 19, batch=1 << 15, q=1 << 14, seed=5), {"compress_every": 0}, 4)
    run(cc, I.grid_stream(256, 256, batch=4001, q=4096, seed=6), {"compress_every": 0}, 4)
    run(cc, I.hub_stream(n=1 << 16, m=1 << 18, batch=1 << 15, q=1 << 13), {"compress_every": 0}, 4)


def test_size_full_grid_height(cc):
    # the 8192 x 8192 grid in minibatches of 2^22 without any compression pass:
    # union by size keeps every tree within floor(log2 n) = 26, link by index
    # does not have that bound
    s = I.grid_stream()
    f = cc.Forest(s.n, update_schedule=1, link=1, compress_every=0)
    g = cc.Forest(s.n, update_schedule=1, link=0, compress_every=0)
    for i in range(s.batches):
        e = dev(s.edges(i))
        f.bulk_update(e)
        g.bulk_update(e)
    mx_size, _ = f.depth()
    assert mx_size <= 26
    assert f.components() == g.components() == 1
    assert int(f.labels().max()) == 0


def test_size_checkpoint_and_errors(cc):
    s = I.rmat_stream(scale=14, m=1 << 16, batch=1 << 12, q=1 << 10, seed=7)
    ref = oracle.OracleUF(s.n)
    f = cc.Forest(s.n, update_schedule=1, link=1)
    for i in range(8):
        f.bulk_update(dev(s.edges(i)))
        ref.bulk_update(s.edges(i))
    with pytest.raises(cc.CCError) as ex:
        f.set_option("link", 0)          # not while the forest has edges
    assert ex.value.status == cc.CC_ERR_ARG
    saved = f.labels()
    h = cc.Forest(s.n, update_schedule=1, link=1)
    h.load_labels(saved)                 # sizes are recounted from the labels
    for i in range(8, s.batches):
        h.bulk_update(dev(s.edges(i)))
        ref.bulk_update(s.edges(i))
    assert np.array_equal(h.labels().cpu().numpy(), ref.labels())
    assert h.depth()[0] <= 14
    z = cc.Forest(100, link=1)           # union by size needs the paper's schedule
    with pytest.raises(cc.CCError) as ex:
        z.bulk_update(torch.tensor([[1, 2]], dtype=torch.int32, device="cuda"))
    assert ex.value.status == cc.CC_ERR_UNSUPPORTED
    z.reset()
    z.set_option("update_schedule", 1)
    z.bulk_update(torch.tensor([[1, 2]], dtype=torch.int32, device="cuda"))
    assert z.components() == 99
