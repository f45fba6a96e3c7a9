"""Python binding of libcc (the C-ABI in include/cc.h).

Argument marshalling only: tensors are checked (CUDA, int32/uint8,
contiguous) and their device pointers, sizes and the current CUDA stream are
passed through ctypes. Every step of the bulk operations runs in libcc's
kernels. There is no fallback: if ``libcc.so`` is missing or cannot be
loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np
import torch

from ._build import LIBCC

CC_OK, CC_ERR_ARG, CC_ERR_OOM, CC_ERR_CUDA, CC_ERR_RANGE, CC_ERR_CORRUPT, CC_ERR_LABELS, \
    CC_ERR_UNSUPPORTED = range(8)
COMPRESS_ALL, COMPRESS_TOUCHED = 0, 1
OPT_BLOCK, OPT_EDGES_PER_THREAD, OPT_COMPRESS_EVERY, OPT_COMPRESS_SCOPE, OPT_QUERY_HALVING, \
    OPT_PROFILE, OPT_UPDATE_VARIANT, OPT_L2_PERSIST = range(8)
OPTIONS = {"block": OPT_BLOCK, "edges_per_thread": OPT_EDGES_PER_THREAD,
           "compress_every": OPT_COMPRESS_EVERY, "compress_scope": OPT_COMPRESS_SCOPE,
           "query_halving": OPT_QUERY_HALVING, "profile": OPT_PROFILE,
           "update_variant": OPT_UPDATE_VARIANT, "l2_persist": OPT_L2_PERSIST,
           "seg_block": 8, "seg_edges_per_thread": 9, "seg_smem_cap": 10, "seg_graph": 11,
           "seg_max_ctas": 12, "update_schedule": 13, "link": 14,
           "bulk_find": 15, "query_variant": 16, "pdl": 17,
           "query_pairs_per_thread": 18, "hook": 19, "sv_graph": 20, "edge_order": 21,
           "hook_warp": 22, "big_filter": 23}
OP_UPDATE, OP_QUERY = 0, 1
# Layout of cc_op (include/cc.h): graph, kind, data pointer, k, out pointer.
OP_DTYPE = np.dtype([("graph", "<i4"), ("kind", "<i4"), ("data", "<u8"), ("k", "<i8"),
                     ("out", "<u8")])
KERNELS = ["update", "compress_all", "compress_touched", "query", "labels", "reset", "load",
           "segmented", "order", "big_pick"]

_lib: ctypes.CDLL | None = None


class CCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


def _status_name(s: int) -> str:
    names = ["CC_OK", "CC_ERR_ARG", "CC_ERR_OOM", "CC_ERR_CUDA", "CC_ERR_RANGE",
             "CC_ERR_CORRUPT", "CC_ERR_LABELS", "CC_ERR_UNSUPPORTED"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def load(path: str | Path | None = None) -> ctypes.CDLL:
    """Load libcc.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIBCC
    if not p.exists():
        raise RuntimeError(f"libcc.so not found at {p}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(str(p))
    vp, i64, i32, u64p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    sig = {
        "cc_create": [i64, ctypes.POINTER(ctypes.c_void_p)],
        "cc_destroy": [vp],
        "cc_set_stream": [vp, vp],
        "cc_sync": [vp],
        "cc_reset": [vp],
        "cc_bulk_update": [vp, vp, i64],
        "cc_bulk_query": [vp, vp, i64, vp],
        "cc_compress": [vp, i32, vp, i64],
        "cc_labels": [vp, vp],
        "cc_load_labels": [vp, vp],
        "cc_copy_parent": [vp, vp],
        "cc_components": [vp, ctypes.POINTER(ctypes.c_int64)],
        "cc_set_option": [vp, i32, i64],
        "cc_get_option": [vp, i32, ctypes.POINTER(ctypes.c_int64)],
        "cc_kernel_stats": [vp, u64p, vp],
        "cc_create_segmented": [i32, vp, ctypes.POINTER(ctypes.c_void_p)],
        "cc_submit": [vp, vp, i64],
        "cc_server_create": [vp, vp, ctypes.POINTER(ctypes.c_void_p)],
        "cc_server_enqueue": [vp, i32, vp, i64, vp, ctypes.POINTER(ctypes.c_uint64)],
        "cc_server_enqueue_many": [vp, i64, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)],
        "cc_server_wait": [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)],
        "cc_server_drain": [vp],
        "cc_server_get_stats": [vp, vp],
        "cc_server_latencies": [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)],
        "cc_server_destroy": [vp],
        "cc_device_can_read": [vp, ctypes.POINTER(ctypes.c_int32)],
        "cc_schedule_stats": [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)],
        "cc_copy_nonloop": [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)],
        "cc_forest_depth": [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)],
        "cc_bulk_find": [vp, vp, i64, vp],
        "cc_bulk_find_stats": [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_int32)],
        "cc_load_forest": [vp, vp],
        "cc_big_filter_stats": [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.cc_num_vertices.argtypes = [vp]
    L.cc_num_vertices.restype = i64
    L.cc_status_string.argtypes = [ctypes.c_int]
    L.cc_status_string.restype = ctypes.c_char_p
    L.cc_last_error_string.argtypes = []
    L.cc_last_error_string.restype = ctypes.c_char_p
    if path is None:
        _lib = L
    return L


def check(status: int, L: ctypes.CDLL | None = None) -> None:
    if status != CC_OK:
        L = L or load()
        raise CCError(status, (L.cc_last_error_string() or b"").decode())


def device_can_read(t: torch.Tensor) -> bool:
    """True if libcc's kernels can read this tensor's memory directly (device
    memory, or pinned host memory mapped for the device)."""
    ok = ctypes.c_int32()
    check(load().cc_device_can_read(t.data_ptr(), ctypes.byref(ok)))
    return bool(ok.value)


def _pairs_ptr(t: torch.Tensor, name: str) -> tuple[int, int]:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a tensor")
    if not t.is_cuda and not (t.is_pinned() and device_can_read(t)):
        raise TypeError(f"{name}: expected a CUDA tensor or device-readable pinned host memory")
    if t.dtype != torch.int32 or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous int32 tensor")
    if t.numel() % 2:
        raise ValueError(f"{name}: expected (k, 2) pairs")
    return t.data_ptr(), t.numel() // 2


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)


class Forest:
    """A device-resident union-find forest over vertices 0..n-1 (libcc handle).

    All calls are enqueued on the bound stream (default: the current torch
    stream at construction)."""

    def __init__(self, n: int, stream=None, _sizes=None, **options):
        self._L = load()
        h = ctypes.c_void_p()
        if _sizes is None:
            check(self._L.cc_create(int(n), ctypes.byref(h)), self._L)
            self.offsets = np.array([0, int(n)], dtype=np.int64)
        else:
            sizes = np.ascontiguousarray(_sizes, dtype=np.int64)
            check(self._L.cc_create_segmented(len(sizes), sizes.ctypes.data, ctypes.byref(h)),
                  self._L)
            self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self._h = h
        self.n = int(self.offsets[-1])
        self.set_stream(stream)
        for k, v in options.items():
            self.set_option(k, v)

    @classmethod
    def segmented(cls, n_per_graph, stream=None, **options) -> "Forest":
        """Many independent graphs (local ids 0..n_g-1) in one handle."""
        return cls(0, stream=stream, _sizes=n_per_graph, **options)

    # lifetime ---------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None):
            check(self._L.cc_destroy(self._h), self._L)
            self._h = None

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                self._L.cc_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream=None) -> None:
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        check(self._L.cc_set_stream(self._h, _stream_handle(self.stream)), self._L)

    def sync(self) -> None:
        check(self._L.cc_sync(self._h), self._L)

    def reset(self) -> None:
        check(self._L.cc_reset(self._h), self._L)

    # bulk operations ---------------------------------------------------
    def bulk_update(self, edges: torch.Tensor) -> None:
        p, k = _pairs_ptr(edges, "edges")
        check(self._L.cc_bulk_update(self._h, p, k), self._L)

    def bulk_query(self, pairs: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        p, k = _pairs_ptr(pairs, "pairs")
        if out is None:
            out = (torch.empty(k, dtype=torch.uint8, device=pairs.device) if pairs.is_cuda
                   else torch.empty(k, dtype=torch.uint8, pin_memory=True))
        if out.dtype != torch.uint8 or not out.is_contiguous() or out.numel() < k:
            raise TypeError("out: expected a contiguous uint8 tensor of k elements")
        if k and not out.is_cuda and not (out.is_pinned() and device_can_read(out)):
            raise TypeError("out: expected CUDA or device-readable pinned host memory")
        check(self._L.cc_bulk_query(self._h, p, k, out.data_ptr()), self._L)
        return out

    def compress(self, scope: str = "all", edges: torch.Tensor | None = None) -> None:
        if scope == "all":
            check(self._L.cc_compress(self._h, COMPRESS_ALL, None, 0), self._L)
        else:
            p, k = _pairs_ptr(edges, "edges")
            check(self._L.cc_compress(self._h, COMPRESS_TOUCHED, p, k), self._L)

    def labels(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.n, dtype=torch.int32, device="cuda")
        if out.dtype != torch.int32 or not out.is_contiguous() or out.numel() < self.n:
            raise TypeError("out: expected a contiguous int32 tensor of n elements")
        check(self._L.cc_labels(self._h, out.data_ptr()), self._L)
        return out

    def load_labels(self, labels: torch.Tensor) -> None:
        if labels.dtype != torch.int32 or not labels.is_contiguous() or labels.numel() != self.n:
            raise TypeError("labels: expected a contiguous int32 tensor of n elements")
        check(self._L.cc_load_labels(self._h, labels.data_ptr()), self._L)

    def parent(self) -> torch.Tensor:
        out = torch.empty(self.n, dtype=torch.int32, device="cuda")
        check(self._L.cc_copy_parent(self._h, out.data_ptr()), self._L)
        return out

    def components(self) -> int:
        v = ctypes.c_int64()
        check(self._L.cc_components(self._h, ctypes.byref(v)), self._L)
        return v.value

    def bulk_find(self, S: torch.Tensor, res: torch.Tensor | None = None) -> torch.Tensor:
        """Bulk-Find (Algorithm 4): roots of the int32 vertices S, compressing
        every path walked."""
        if not S.is_cuda or S.dtype != torch.int32 or not S.is_contiguous():
            raise TypeError("S: expected a contiguous CUDA int32 tensor")
        if res is None:
            res = torch.empty(S.numel(), dtype=torch.int32, device=S.device)
        check(self._L.cc_bulk_find(self._h, S.data_ptr(), S.numel(), res.data_ptr()), self._L)
        return res

    def bulk_find_stats(self) -> tuple[int, int, int]:
        """(traversed non-root vertices, Phase I levels, Phase II levels)."""
        t, u, d = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        check(self._L.cc_bulk_find_stats(self._h, ctypes.byref(t), ctypes.byref(u), ctypes.byref(d)),
              self._L)
        return t.value, u.value, d.value

    def load_forest(self, parent: torch.Tensor) -> None:
        if parent.dtype != torch.int32 or not parent.is_contiguous() or parent.numel() != self.n:
            raise TypeError("parent: expected a contiguous int32 tensor of n elements")
        check(self._L.cc_load_forest(self._h, parent.data_ptr()), self._L)

    def big_filter_stats(self) -> tuple[int, int]:
        """(root R whose tree the largest-component bitmap marks or -1 when the
        filter is off, vertices marked by the last compression pass)."""
        r, m = ctypes.c_int32(), ctypes.c_int64()
        check(self._L.cc_big_filter_stats(self._h, ctypes.byref(r), ctypes.byref(m)), self._L)
        return r.value, m.value

    def depth(self) -> tuple[int, float]:
        """(max, mean) distance from a vertex to its root."""
        mx, mean = ctypes.c_int32(), ctypes.c_double()
        check(self._L.cc_forest_depth(self._h, ctypes.byref(mx), ctypes.byref(mean)), self._L)
        return mx.value, mean.value

    def schedule_stats(self) -> tuple[int, int]:
        """(|A''|, connected-components rounds) of the last Bulk-Update under
        the paper's schedule (update_schedule=1)."""
        m, r = ctypes.c_int64(), ctypes.c_int32()
        check(self._L.cc_schedule_stats(self._h, ctypes.byref(m), ctypes.byref(r)), self._L)
        return m.value, r.value

    def nonloop_edges(self) -> torch.Tensor:
        """A'' of the last Bulk-Update under the paper's schedule: (m, 2) int32."""
        m, _ = self.schedule_stats()
        out = torch.empty((max(m, 1), 2), dtype=torch.int32, device="cuda")
        cnt = ctypes.c_int64()
        check(self._L.cc_copy_nonloop(self._h, out.data_ptr(), m, ctypes.byref(cnt)), self._L)
        return out[:m]

    def submit(self, ops) -> None:
        """Run bulk operations in one persistent launch (cc_submit). ``ops`` is
        an ``OP_DTYPE`` array, or a list of (graph, kind, data, out) with
        ``data`` an int32 (k, 2) CUDA tensor of local ids and ``out`` a uint8
        CUDA tensor (queries) or None."""
        if not isinstance(ops, np.ndarray):
            arr = np.zeros(len(ops), dtype=OP_DTYPE)
            for i, (g, kind, data, out) in enumerate(ops):
                p, k = _pairs_ptr(data, "data")
                arr[i] = (g, kind, p, k, out.data_ptr() if out is not None else 0)
            ops = arr
        if ops.dtype != OP_DTYPE or not ops.flags.c_contiguous:
            raise TypeError("ops: expected a contiguous OP_DTYPE array")
        check(self._L.cc_submit(self._h, ops.ctypes.data, len(ops)), self._L)

    # tunables and counters ---------------------------------------------
    def set_option(self, name: str, value: int) -> None:
        check(self._L.cc_set_option(self._h, OPTIONS[name], int(value)), self._L)

    def get_option(self, name: str) -> int:
        v = ctypes.c_int64()
        check(self._L.cc_get_option(self._h, OPTIONS[name], ctypes.byref(v)), self._L)
        return v.value

    def kernel_stats(self, timing: bool = False) -> dict:
        """{kind: launches} and, with timing=True, {kind: (launches, ms)}
        (the ms sums cover launches since the previous timing read)."""
        n = len(KERNELS)
        counts = (ctypes.c_uint64 * n)()
        ms = (ctypes.c_double * n)() if timing else None
        check(self._L.cc_kernel_stats(self._h, counts, ms), self._L)
        if timing:
            return {k: (int(counts[i]), float(ms[i])) for i, k in enumerate(KERNELS)}
        return {k: int(counts[i]) for i, k in enumerate(KERNELS)}


class _ServerConfig(ctypes.Structure):
    _fields_ = [("ring_pairs", ctypes.c_int64), ("max_group_pairs", ctypes.c_int64),
                ("merge", ctypes.c_int32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in
                ("requests", "updates", "queries", "completed", "groups", "edges", "pairs")]


class Server:
    """Continuous-batching request loop over a Forest (cc_server_*).

    ``enqueue`` takes HOST tensors (pinned for overlapped copies): int32 (k, 2)
    data and, for queries, a uint8 (k,) output that is filled before the
    request completes. The Forest must not be used directly while the server
    runs."""

    def __init__(self, forest: Forest, ring_pairs: int = 0, max_group_pairs: int = 0,
                 merge: bool = True):
        self._L = forest._L
        self.forest = forest
        cfg = _ServerConfig(ring_pairs, max_group_pairs, 1 if merge else 0)
        h = ctypes.c_void_p()
        check(self._L.cc_server_create(forest._h, ctypes.byref(cfg), ctypes.byref(h)), self._L)
        self._h = h
        self._keep: dict[int, tuple] = {}

    def enqueue(self, kind: int, data: torch.Tensor, out: torch.Tensor | None = None) -> int:
        if data.is_cuda or data.dtype != torch.int32 or not data.is_contiguous():
            raise TypeError("data: expected a contiguous host int32 tensor")
        k = data.numel() // 2
        optr = 0
        if kind == OP_QUERY:
            if out is None or out.is_cuda or out.dtype != torch.uint8 or out.numel() < k:
                raise TypeError("out: expected a host uint8 tensor of k elements")
            optr = out.data_ptr()
        t = ctypes.c_uint64()
        check(self._L.cc_server_enqueue(self._h, kind, data.data_ptr(), k, optr, ctypes.byref(t)),
              self._L)
        self._keep[t.value] = (data, out)   # keep the buffers alive until drained
        return t.value

    def enqueue_many(self, kinds: np.ndarray, data_ptrs: np.ndarray, ks: np.ndarray,
                     out_ptrs: np.ndarray | None = None, keep=None) -> int:
        """n requests in one call (cc_server_enqueue_many): int32 kinds, uint64
        host addresses of the int32 (k, 2) data, int64 k (pairs), and uint64
        host addresses of the uint8 outputs (0 for updates). The caller keeps
        the buffers alive until the requests complete (or passes them in
        `keep`). Returns the first ticket; request i has ticket first + i."""
        kinds = np.ascontiguousarray(kinds, dtype=np.int32)
        data_ptrs = np.ascontiguousarray(data_ptrs, dtype=np.uint64)
        ks = np.ascontiguousarray(ks, dtype=np.int64)
        n = len(kinds)
        if len(data_ptrs) != n or len(ks) != n or (out_ptrs is not None and len(out_ptrs) != n):
            raise ValueError("enqueue_many: arrays of different lengths")
        optr = None
        if out_ptrs is not None:
            out_ptrs = np.ascontiguousarray(out_ptrs, dtype=np.uint64)
            optr = out_ptrs.ctypes.data
        t = ctypes.c_uint64()
        check(self._L.cc_server_enqueue_many(self._h, n, kinds.ctypes.data, data_ptrs.ctypes.data,
                                             ks.ctypes.data, optr, ctypes.byref(t)), self._L)
        if keep is not None:
            self._keep[t.value] = keep
        return t.value

    def enqueue_list(self, requests) -> int:
        """[(kind, data, out)] as for enqueue, in one call; returns the first ticket."""
        kinds, dp, ks, op = [], [], [], []
        for kind, data, out in requests:
            if data.is_cuda or data.dtype != torch.int32 or not data.is_contiguous():
                raise TypeError("data: expected a contiguous host int32 tensor")
            k = data.numel() // 2
            if kind == OP_QUERY and (out is None or out.is_cuda or out.dtype != torch.uint8
                                     or out.numel() < k):
                raise TypeError("out: expected a host uint8 tensor of k elements")
            kinds.append(kind)
            dp.append(data.data_ptr())
            ks.append(k)
            op.append(out.data_ptr() if kind == OP_QUERY else 0)
        return self.enqueue_many(np.array(kinds), np.array(dp, dtype=np.uint64), np.array(ks),
                                 np.array(op, dtype=np.uint64), keep=list(requests))

    def wait(self, ticket: int) -> float:
        lat = ctypes.c_double()
        check(self._L.cc_server_wait(self._h, ticket, ctypes.byref(lat)), self._L)
        return lat.value

    def drain(self) -> None:
        check(self._L.cc_server_drain(self._h), self._L)
        self._keep.clear()

    def stats(self) -> dict:
        st = _ServerStats()
        check(self._L.cc_server_get_stats(self._h, ctypes.byref(st)), self._L)
        return {f: getattr(st, f) for f, _ in st._fields_}

    def latencies(self) -> np.ndarray:
        n = self.stats()["requests"]
        out = np.empty(n, dtype=np.float64)
        w = ctypes.c_int64()
        check(self._L.cc_server_latencies(self._h, out.ctypes.data, n, ctypes.byref(w)), self._L)
        return out[:w.value]

    def close(self) -> None:
        if getattr(self, "_h", None):
            check(self._L.cc_server_destroy(self._h), self._L)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
