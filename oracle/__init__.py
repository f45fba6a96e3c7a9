"""CPU oracle for bulk incremental connectivity -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA path and
imports nothing from it. ``cc_oracle.c`` holds the arithmetic: a sequential
union-find with union by rank and full path compression, the paper's
"UF (p.c.)" baseline (Section 5.3), answering Bulk-Query (Algorithm 1's
contract) and producing minimum-id component labels. This module only builds
and loads it and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "cc_oracle.c"
LIB = HERE / "liboracle.so"

_lib = None


def build(force: bool = False, src: Path = SRC, out: Path = LIB) -> Path:
    """Compile ``src`` to ``out`` with gcc (in place, under a file lock)."""
    lock = HERE / ".build.lock"
    with open(lock, "w") as fh:
        fcntl.flock(fh, fcntl.LOCK_EX)
        try:
            if force or not out.exists() or out.stat().st_mtime < src.stat().st_mtime:
                tmp = out.with_suffix(".so.tmp")
                r = subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", str(src),
                                    "-o", str(tmp)], capture_output=True, text=True)
                if r.returncode != 0:
                    raise RuntimeError(f"oracle build failed:\n{r.stderr}")
                os.replace(tmp, out)
        finally:
            fcntl.flock(fh, fcntl.LOCK_UN)
    return out


def load(path: Path | None = None) -> ctypes.CDLL:
    """Load the oracle library (``path`` selects another build of it)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(str(path)))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(str(build())))
    return _lib


def _bind(L: ctypes.CDLL) -> ctypes.CDLL:
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    L.oracle_create.argtypes = [i64]
    L.oracle_create.restype = p
    L.oracle_destroy.argtypes = [p]
    L.oracle_destroy.restype = None
    L.oracle_bulk_update.argtypes = [p, p, i64]
    L.oracle_bulk_update.restype = i64
    L.oracle_bulk_query.argtypes = [p, p, i64, p]
    L.oracle_bulk_query.restype = None
    L.oracle_labels.argtypes = [p, p]
    L.oracle_labels.restype = None
    L.oracle_relabel.argtypes = [p, p, i64, p]
    L.oracle_relabel.restype = i64
    L.oracle_bulk_find.argtypes = [i64, p, p, i64, p, p]
    L.oracle_bulk_find.restype = i64
    for f in ("oracle_n", "oracle_unions", "oracle_errors", "oracle_components"):
        getattr(L, f).argtypes = [p]
        getattr(L, f).restype = i64
    return L


def _pairs(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int32)
    if a.size == 0:
        return a.reshape(0, 2)
    assert a.ndim == 2 and a.shape[1] == 2 or a.ndim == 1 and a.size % 2 == 0
    return a.reshape(-1, 2)


class OracleUF:
    """Sequential union-find over vertices 0..n-1 (starts as n singletons)."""

    def __init__(self, n: int, lib: ctypes.CDLL | None = None):
        self._L = lib if lib is not None else load()
        self._h = self._L.oracle_create(int(n))
        if not self._h:
            raise ValueError(f"oracle_create({n}) failed")
        self.n = int(n)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.oracle_destroy(h)
            self._h = None

    def bulk_update(self, edges) -> int:
        """Add the edges (k x 2 int32) in array order; returns the unions made."""
        e = _pairs(edges)
        return int(self._L.oracle_bulk_update(self._h, e.ctypes.data_as(ctypes.c_void_p),
                                              e.shape[0]))

    def bulk_query(self, pairs) -> np.ndarray:
        """uint8 answers, 1 iff the two ids are connected."""
        q = _pairs(pairs)
        out = np.empty(q.shape[0], dtype=np.uint8)
        self._L.oracle_bulk_query(self._h, q.ctypes.data_as(ctypes.c_void_p), q.shape[0],
                                  out.ctypes.data_as(ctypes.c_void_p))
        return out

    def relabel(self, edges) -> np.ndarray:
        """A'' of Algorithm 2 for these edges against the current graph:
        (id(u), id(v)) with minimum-id component identifiers, self-loops
        dropped, edge order kept. Does not add the edges."""
        e = _pairs(edges)
        out = np.empty((e.shape[0], 2), dtype=np.int32)
        m = int(self._L.oracle_relabel(self._h, e.ctypes.data_as(ctypes.c_void_p), e.shape[0],
                                       out.ctypes.data_as(ctypes.c_void_p)))
        return out[:m]

    def labels(self) -> np.ndarray:
        """int32 labels: the minimum vertex id of each vertex's component."""
        out = np.empty(self.n, dtype=np.int32)
        self._L.oracle_labels(self._h, out.ctypes.data_as(ctypes.c_void_p))
        return out

    @property
    def unions(self) -> int:
        return int(self._L.oracle_unions(self._h))

    @property
    def errors(self) -> int:
        return int(self._L.oracle_errors(self._h))

    @property
    def components(self) -> int:
        return int(self._L.oracle_components(self._h))


def bulk_find(parent, S, lib: ctypes.CDLL | None = None):
    """Bulk-Find (Algorithm 4) on the forest `parent`: returns (new parent
    array, res = root of each S[i], number of traversed non-root nodes)."""
    L = lib if lib is not None else load()
    par = np.ascontiguousarray(parent, dtype=np.int32)
    q = np.ascontiguousarray(S, dtype=np.int32)
    out = np.empty_like(par)
    res = np.empty(q.size, dtype=np.int32)
    t = int(L.oracle_bulk_find(par.size, par.ctypes.data_as(ctypes.c_void_p),
                               q.ctypes.data_as(ctypes.c_void_p), q.size,
                               out.ctypes.data_as(ctypes.c_void_p),
                               res.ctypes.data_as(ctypes.c_void_p)))
    if t < 0:
        raise ValueError("bulk_find: the forest has a cycle")
    return out, res, t
