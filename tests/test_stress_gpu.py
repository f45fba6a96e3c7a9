"""Randomised stress of the concurrent Bulk-Update paths against the oracle.

Every update variant, with compare-and-swap hooks and with the atomicMin hook
(whose correctness rests on an argument about concurrent displacement and
repair), each also with the hooks of a warp grouped by target root, runs
many small seeded streams of varied shape -- hub-heavy,
uniform, long descending paths, many duplicate edges -- cut into minibatches
of random, ragged sizes. After every minibatch the labels (minimum vertex id
per component) and a batch of query answers must equal the oracle's exactly.
Small forests and hub-heavy batches make many threads contend for the same
roots within one launch, which is where a wrong interleaving would show."""
from __future__ import annotations

import zlib

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05232_gb300 import _build, cc as ccmod
    _build.build_cc()
    ccmod.load()
    return ccmod


def random_stream(rng: np.random.Generator):
    """(n, edges, cut points) for one random stream shape."""
    n = int(rng.choice([7, 33, 257, 1000, 4099, 20000]))
    m = int(rng.integers(1, 6 * n + 2))
    kind = rng.integers(0, 4)
    if kind == 0:    # hubs: most edges touch a few vertices
        hubs = rng.integers(0, n, size=max(1, n // 100))
        u = rng.choice(hubs, size=m)
        v = rng.integers(0, n, size=m)
    elif kind == 1:  # uniform
        u = rng.integers(0, n, size=m)
        v = rng.integers(0, n, size=m)
    elif kind == 2:  # a descending path, shuffled, plus noise
        p = np.arange(n - 1, 0, -1)
        u = np.concatenate([p, rng.integers(0, n, size=m // 4)])
        v = np.concatenate([p - 1, rng.integers(0, n, size=m // 4)])
        perm = rng.permutation(len(u))
        u, v = u[perm], v[perm]
    else:            # few distinct edges, many duplicates
        base_u = rng.integers(0, n, size=max(1, m // 20))
        base_v = rng.integers(0, n, size=len(base_u))
        idx = rng.integers(0, len(base_u), size=m)
        u, v = base_u[idx], base_v[idx]
    edges = np.stack([u, v], 1).astype(np.int32)
    cuts = np.unique(np.concatenate([[0, len(edges)], rng.integers(0, len(edges) + 1, size=rng.integers(1, 8))]))
    return n, edges, cuts


CONFIGS = {
    "v0_cas": {"update_variant": 0, "edges_per_thread": 2},
    "v1_cas": {"update_variant": 1, "edges_per_thread": 4, "block": 64},
    "v2_cas": {"update_variant": 2, "edges_per_thread": 1, "compress_every": 0},
    "v3_cas": {"update_variant": 3, "edges_per_thread": 2, "compress_every": 0, "pdl": 2},
    "v4_cas": {"update_variant": 4, "edges_per_thread": 4, "compress_every": 0},
    "v0_min": {"update_variant": 0, "edges_per_thread": 1, "hook": 1},
    "v1_min": {"update_variant": 1, "edges_per_thread": 2, "hook": 1, "compress_every": 0},
    "v2_min": {"update_variant": 2, "edges_per_thread": 4, "hook": 1, "compress_every": 0},
    "v3_min": {"update_variant": 3, "edges_per_thread": 1, "hook": 1, "compress_every": 0, "block": 1024},
    "v4_min": {"update_variant": 4, "edges_per_thread": 2, "hook": 1, "compress_every": 2},
    "v3_min_first": {"update_variant": 3, "edges_per_thread": 2, "hook": 2, "compress_every": 0, "pdl": 2},
    "v5_cas": {"update_variant": 5, "edges_per_thread": 2, "block": 64, "compress_every": 0},
    "v5_min": {"update_variant": 5, "edges_per_thread": 4, "hook": 1, "compress_every": 0},
    # hooks grouped per warp by target root (hook_warp), both link primitives
    "v1_cas_warp": {"update_variant": 1, "edges_per_thread": 2, "block": 64, "hook_warp": 1},
    "v2_min_warp": {"update_variant": 2, "edges_per_thread": 1, "hook": 1, "compress_every": 0, "hook_warp": 1},
    "v3_cas_warp": {"update_variant": 3, "edges_per_thread": 4, "compress_every": 0, "hook_warp": 1},
    "v3_min_warp": {"update_variant": 3, "edges_per_thread": 2, "hook": 1, "compress_every": 0, "hook_warp": 1,
                    "pdl": 2},
    "v4_cas_warp": {"update_variant": 4, "edges_per_thread": 1, "compress_every": 0, "hook_warp": 1},
    "v4_min_warp": {"update_variant": 4, "edges_per_thread": 4, "hook": 1, "compress_every": 3, "hook_warp": 1},
}


@pytest.mark.parametrize("name", list(CONFIGS), ids=list(CONFIGS))
def test_random_streams_match_oracle(cc, name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))   # the same streams in every run
    for trial in range(150):
        n, edges, cuts = random_stream(rng)
        f = cc.Forest(n, **CONFIGS[name])
        ref = oracle.OracleUF(n)
        pairs = rng.integers(0, n, size=(512, 2)).astype(np.int32)
        d_pairs = torch.from_numpy(pairs).cuda()
        for a, b in zip(cuts[:-1], cuts[1:]):
            e = edges[a:b]
            if len(e):
                f.bulk_update(torch.from_numpy(np.ascontiguousarray(e)).cuda())
                ref.bulk_update(e)
            assert np.array_equal(f.labels().cpu().numpy(), ref.labels()), (name, trial, int(a))
            assert np.array_equal(f.bulk_query(d_pairs).cpu().numpy(), ref.bulk_query(pairs)), (name, trial)
        assert f.components() == ref.components
        f.sync()
        f.close()
