"""The C-ABI library loads and exports every declared entry point (no GPU needed).

Only argument checks that return before any CUDA call are exercised here.
"""
import ctypes
import glob
import os
import re

import pytest

from paper_1503_04359_b300 import build as build_mod
from paper_1503_04359_b300 import dobfs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|const char\*|void|int32_t|int64_t)\s+(dobfs_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return dobfs.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_python_binding_has_same_names():
    for n in _declared():
        if n in ("dobfs_set_allocator", "dobfs_last_error"):
            continue
        assert hasattr(dobfs, n), n


def test_argument_errors_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.dobfs_graph_create_rmat(0, 10, 0, 0, 0, 1, 0, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_INVALID
    assert "R-MAT" in dobfs.last_error()
    assert lib.dobfs_graph_create_rmat(10, 10, 5, 3, 9, 1, 0, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_INVALID
    assert lib.dobfs_graph_create_from_pairs(None, None, -1, 10, 0, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_INVALID
    assert lib.dobfs_run(None, 0, None, None, None, None) == dobfs.DOBFS_ERR_INVALID
    assert lib.dobfs_graph_get_info(None, None) == dobfs.DOBFS_ERR_INVALID
    assert lib.dobfs_graph_destroy(None) == dobfs.DOBFS_OK
    assert lib.dobfs_graph_wait(None, 0) == dobfs.DOBFS_ERR_INVALID
    assert lib.dobfs_graph_save(None, b"x", None) == dobfs.DOBFS_ERR_INVALID
    assert lib.dobfs_graph_load(None, 0, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_INVALID
    assert lib.dobfs_graph_load(b"x", 0x80, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_INVALID
    o = dobfs.dobfs_run_opts()
    assert lib.dobfs_run_opts_init(ctypes.byref(o)) == 0
    assert (o.direction, o.alpha, o.beta) == (dobfs.DOBFS_DIR_AUTO, 14, 24)
    assert (o.td_bitmap_div, o.td_small_max, o.td_chunk, o.bu_scan, o.td_split_pct) == (2, 0, 0, 0, 150)
    # the library writes exactly the bytes of the binding's struct: no field is missing at the end
    buf = (ctypes.c_ubyte * (ctypes.sizeof(dobfs.dobfs_run_opts) + 64))(*([0xA5] * (ctypes.sizeof(dobfs.dobfs_run_opts) + 64)))
    assert lib.dobfs_run_opts_init(ctypes.cast(buf, ctypes.POINTER(dobfs.dobfs_run_opts))) == 0
    assert list(buf[ctypes.sizeof(dobfs.dobfs_run_opts):]) == [0xA5] * 64
    last = dobfs.dobfs_run_opts.td_split_pct.offset
    assert list(buf[last:last + 4]) == [150, 0, 0, 0]
    assert (o.bu_threads, o.td_threads, o.out_threads) == (0, 0, 0)
    tail = dobfs.dobfs_run_opts.out_threads.offset
    assert tail + 4 == ctypes.sizeof(dobfs.dobfs_run_opts) and list(buf[tail:tail + 4]) == [0, 0, 0, 0]
    # allocator hook: both or neither
    assert lib.dobfs_set_allocator(dobfs.ALLOC_FN(lambda n, s, c: None), dobfs.FREE_FN(), None) == dobfs.DOBFS_ERR_INVALID
    assert lib.dobfs_set_allocator(dobfs.ALLOC_FN(), dobfs.FREE_FN(), None) == dobfs.DOBFS_OK


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(dobfs, "_lib", None)
    monkeypatch.setattr(dobfs, "LIB_PATH", "/nonexistent/libdobfs.so")
    with pytest.raises(ImportError):
        dobfs.load()


def test_graph_file_header_checks_without_gpu(lib, tmp_path):
    """dobfs_graph_load refuses missing files and bad headers before any CUDA call."""
    h = ctypes.c_void_p()
    assert lib.dobfs_graph_load(os.fsencode(tmp_path / "missing.dobfs"), 0, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_IO
    assert "cannot open" in dobfs.last_error()
    short = tmp_path / "short.dobfs"
    short.write_bytes(b"DOBFSCSR")
    assert lib.dobfs_graph_load(os.fsencode(short), 0, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_IO
    assert "truncated" in dobfs.last_error()
    other = tmp_path / "other.dobfs"
    other.write_bytes(b"NOTAGRPH" + bytes(56))
    assert lib.dobfs_graph_load(os.fsencode(other), 0, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_IO
    assert "not a dobfs graph file" in dobfs.last_error()
    newer = tmp_path / "newer.dobfs"
    newer.write_bytes(b"DOBFSCSR" + (99).to_bytes(4, "little") + bytes(52))
    assert lib.dobfs_graph_load(os.fsencode(newer), 0, None, ctypes.byref(h)) == dobfs.DOBFS_ERR_IO
    assert "version 99" in dobfs.last_error()
    assert not h.value
