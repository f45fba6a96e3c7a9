"""cc_components_static: labelling without any device allocation.

Some callers cannot allocate device memory: real-time loops that cannot take
cudaMalloc's implicit synchronisation and unbounded latency, and plugins whose
host framework owns all device memory and offers them no allocator.
cc_components_static serves them from a static array inside libcc. This test
calls it through the C-ABI twice in a row, on two different graphs (the second
smaller, so anything left over from the first call would show), and checks
each result bit for bit against the oracle's minimum-id labels and against the
regular path (cc_create + cc_bulk_update + cc_labels) on the same edges. It
also checks the status word's range bit on a list with ids -1 and n (those
edges are skipped, as the oracle skips them), and the size limit.

The file is named so that pytest collects it last.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle

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


def static_labels(lib, e: np.ndarray, n: int):
    """One call of the entry point; returns (status code, labels, status word)."""
    stream = torch.cuda.current_stream()
    edges = torch.from_numpy(np.ascontiguousarray(e, dtype=np.int32).reshape(-1, 2)).cuda()
    labels = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    st = lib.cc_components_static(edges.data_ptr(), edges.shape[0], n, labels.data_ptr(),
                                  status.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return st, labels, int(status.item())


def oracle_labels(e: np.ndarray, n: int) -> np.ndarray:
    uf = oracle.OracleUF(n)
    uf.bulk_update(np.ascontiguousarray(e, dtype=np.int32).reshape(-1, 2))
    return uf.labels()


def test_static_labels_match_oracle_and_regular_path(lib):
    from paper_1602_05232_gb300 import cc, inputs as I
    cases = [
        ("R-MAT scale 20", 1 << 20, I.rmat_edges(20, 3 << 19, 0.57, 0.19, 0.19, seed=11,
                                                 perm=I.permutation(1 << 20, seed=11))),
        ("uniform, smaller", 5000, I.uniform_pairs(5000, 2400, seed=12, tag=I.TAG_EDGES)),
    ]
    for name, n, e in cases:
        st, labels, status = static_labels(lib, e, n)
        assert st == cc.CC_OK, lib.cc_last_error_string()
        assert status == 0, name
        assert np.array_equal(labels.cpu().numpy(), oracle_labels(e, n)), name
        with cc.Forest(n) as f:
            f.bulk_update(torch.from_numpy(np.ascontiguousarray(e)).cuda())
            want = f.labels()
            f.sync()
        torch.cuda.synchronize()
        assert torch.equal(labels, want), name


def test_static_skips_and_reports_ids_out_of_range(lib):
    from paper_1602_05232_gb300 import cc
    n = 10
    e = np.array([[0, 1], [-1, 2], [3, n], [2, 3], [n, -1], [8, 9], [9, 0]], dtype=np.int32)
    st, labels, status = static_labels(lib, e, n)
    assert st == cc.CC_OK, lib.cc_last_error_string()
    assert status == 1                         # bit 1: an id outside [0, n) was skipped
    want = oracle_labels(e, n)                 # the oracle skips those edges too
    assert want.tolist() == [0, 0, 2, 2, 4, 5, 6, 7, 0, 0]
    assert np.array_equal(labels.cpu().numpy(), want)
    # the next call starts from a clear status word
    st, labels, status = static_labels(lib, e[[0, 3]], n)
    assert st == cc.CC_OK and status == 0
    assert np.array_equal(labels.cpu().numpy(), oracle_labels(e[[0, 3]], n))


def test_static_rejects_sizes_beyond_the_maximum(lib):
    from paper_1602_05232_gb300 import cc
    edges = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    labels = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = lib.cc_components_static(edges.data_ptr(), 1, MAX_VERTICES + 1, labels.data_ptr(),
                                  None, None)
    assert st == cc.CC_ERR_ARG
    assert b"CC_STATIC_MAX_VERTICES" in lib.cc_last_error_string()
