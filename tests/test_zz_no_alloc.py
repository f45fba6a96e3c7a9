"""cc_components_static: labelling without any device allocation.

Some callers cannot allocate device memory: code whose stream is being
captured into a CUDA graph, real-time loops that cannot take cudaMalloc's
implicit synchronisation, plugins whose host framework owns all device memory.
cc_components_static serves them from a static array inside libcc. This test
calls it through the C-ABI twice in a row, on two different graphs (the second
smaller, so anything left over from the first call would show), and checks
each result bit for bit against the regular path (cc_create + cc_bulk_update
+ cc_labels) on the same edges. It also checks the size limit.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MAX_VERTICES = 1 << 22


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05232_gb300 import _build, cc
    _build.build_cc()
    L = cc.load()
    f = L.cc_components_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L


def test_static_labels_match_regular_path(lib):
    from paper_1602_05232_gb300 import cc, inputs as I
    stream = torch.cuda.current_stream()
    cases = [
        ("R-MAT scale 20", 1 << 20, I.rmat_edges(20, 3 << 19, 0.57, 0.19, 0.19, seed=11,
                                                 perm=I.permutation(1 << 20, seed=11))),
        ("uniform, smaller", 5000, I.uniform_pairs(5000, 2400, seed=12, tag=I.TAG_EDGES)),
    ]
    for name, n, e in cases:
        edges = torch.from_numpy(np.ascontiguousarray(e)).cuda()
        labels = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        st = lib.cc_components_static(edges.data_ptr(), edges.shape[0], n, labels.data_ptr(),
                                      status.data_ptr(), stream.cuda_stream)
        assert st == cc.CC_OK, lib.cc_last_error_string()
        with cc.Forest(n) as f:
            f.bulk_update(edges)
            want = f.labels()
            f.sync()
        torch.cuda.synchronize()
        assert torch.equal(labels, want), name
        assert int(status.item()) == 0, name


def test_static_rejects_sizes_beyond_the_maximum(lib):
    from paper_1602_05232_gb300 import cc
    edges = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    labels = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = lib.cc_components_static(edges.data_ptr(), 1, MAX_VERTICES + 1, labels.data_ptr(),
                                  None, None)
    assert st == cc.CC_ERR_ARG
    assert b"CC_STATIC_MAX_VERTICES" in lib.cc_last_error_string()
