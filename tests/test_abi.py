"""The C-ABI library loads and exports every symbol include/cc.h declares,
and its host-side argument checks work (no GPU needed: none of these calls
reaches a kernel or the CUDA runtime)."""
from __future__ import annotations

import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def L():
    from paper_1602_05232_gb300 import _build, cc
    _build.build_cc()
    return cc.load()


def declared_functions() -> list[str]:
    names = []
    for h in sorted((ROOT / "include").glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(cc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("cc_create", "cc_bulk_update", "cc_bulk_query", "cc_labels", "cc_destroy",
                     "cc_sync", "cc_compress", "cc_load_labels"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert missing == []


def test_argument_errors_without_gpu(L):
    from paper_1602_05232_gb300 import cc
    h = ctypes.c_void_p()
    assert L.cc_create(0, ctypes.byref(h)) == cc.CC_ERR_ARG
    assert L.cc_create(1 << 31, ctypes.byref(h)) == cc.CC_ERR_ARG
    assert b"out of" in L.cc_last_error_string()
    assert L.cc_create(5, None) == cc.CC_ERR_ARG
    assert L.cc_bulk_update(None, None, 0) == cc.CC_ERR_ARG
    assert L.cc_bulk_query(None, None, 0, None) == cc.CC_ERR_ARG
    assert L.cc_labels(None, None) == cc.CC_ERR_ARG
    assert L.cc_set_option(None, 0, 256) == cc.CC_ERR_ARG
    counts = (ctypes.c_uint64 * 8)()
    assert L.cc_kernel_stats(None, counts, None) == cc.CC_ERR_ARG
    assert L.cc_destroy(None) == cc.CC_OK
    assert L.cc_num_vertices(None) == 0
    assert L.cc_status_string(cc.CC_ERR_RANGE) == b"CC_ERR_RANGE"


def test_product_path_fails_loudly_without_the_library(tmp_path):
    from paper_1602_05232_gb300 import cc
    with pytest.raises(RuntimeError, match="libcc.so not found"):
        cc.load(tmp_path / "libcc.so")


def test_binding_option_numbers_match_the_header():
    """cc.OPTIONS names every CC_OPT_* of include/cc.h with the header's number."""
    from paper_1602_05232_gb300 import cc
    text = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / "cc.h").read_text(), flags=re.S)
    body = re.search(r"typedef enum \{([^}]*)\}\s*cc_option;", text).group(1)
    enum = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"\bCC_OPT_(\w+)\s*=\s*(\d+)", body) if m.group(1) != "_COUNT"}
    count = int(re.search(r"\bCC_OPT__COUNT\s*=\s*(\d+)", body).group(1))
    assert sorted(enum.values()) == list(range(count))
    assert enum == cc.OPTIONS
