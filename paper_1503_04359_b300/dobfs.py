"""Python binding of libdobfs (argument marshalling only).

Every function named ``dobfs_*`` here forwards to the C entry point of the
same name in ``_lib/libdobfs.so`` (declared in ``include/dobfs.h``): it turns
torch tensors / numpy arrays into pointers and sizes, raises ``DobfsError`` on
a non-zero status, and does nothing else. Every step of the BFS runs in the
library's CUDA kernels; there is no CPU path. If the library is missing,
importing this module raises.

PyTorch provides device memory and streams: ``use_torch_allocator()`` routes
the library's device allocations through PyTorch's caching allocator, and
``stream=None`` means PyTorch's current stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdobfs.so")
# DOBFS_BOUNDS_CHECK=1 selects the bounds-check build (device index checks)
if os.environ.get("DOBFS_BOUNDS_CHECK", "0") not in ("", "0"):
    LIB_PATH = os.path.join(_HERE, "_lib", "libdobfs_bc.so")

DOBFS_OK, DOBFS_PENDING = 0, 1
DOBFS_ERR_INVALID, DOBFS_ERR_OOM, DOBFS_ERR_CUDA = -1, -2, -3
DOBFS_BATCH_ALPHA = 4
DOBFS_ERR_BAD_GRAPH, DOBFS_ERR_TIMEOUT, DOBFS_ERR_BUSY, DOBFS_ERR_IO, DOBFS_ERR_BOUNDS = -4, -5, -6, -7, -8

DOBFS_GRAPH_SYMMETRIZE = 0x1
DOBFS_GRAPH_REINDEX = 0x2
DOBFS_GRAPH_DEVICE_PTRS = 0x4
DOBFS_GRAPH_VALIDATE = 0x8
DOBFS_GRAPH_OFFSETS64 = 0x10
DOBFS_GRAPH_REINDEX_EXACT = 0x20
DOBFS_GRAPH_CHUNKED = 0x40

DOBFS_DIR_AUTO, DOBFS_DIR_TOPDOWN, DOBFS_DIR_BOTTOMUP, DOBFS_DIR_RANDOM, DOBFS_DIR_STATIC = 0, 1, 2, 3, 4
DOBFS_RUN_CANONICAL_PARENT = 0x1
DOBFS_RUN_HOST_LOOP = 0x2
DOBFS_RUN_SYNC_STATS = 0x4
DOBFS_RUN_LEVEL_GRAPH = 0x8
DOBFS_STATIC_MAX_VERTICES = 1 << 20


class DobfsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("dobfs status %d: %s" % (status, msg))
        self.status = status


class dobfs_graph_info(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_entries", ctypes.c_int64), ("n_nonisolated", ctypes.c_int64),
                ("max_degree", ctypes.c_int64), ("offsets_int64", ctypes.c_int32), ("reindexed", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("build_ms", ctypes.c_float)]


class dobfs_run_opts(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int32), ("alpha", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("static_pct", ctypes.c_int32), ("bu_steps", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("schedule_seed", ctypes.c_uint64), ("stream", ctypes.c_void_p), ("td_bitmap_div", ctypes.c_int32),
                ("td_small_max", ctypes.c_int32), ("td_chunk", ctypes.c_int32), ("bu_scan", ctypes.c_int32),
                ("td_split_pct", ctypes.c_int32), ("bu_threads", ctypes.c_int32), ("td_threads", ctypes.c_int32),
                ("out_threads", ctypes.c_int32)]


class dobfs_run_stats(ctypes.Structure):
    _fields_ = [("device_ms", ctypes.c_float), ("levels", ctypes.c_int32), ("td_levels", ctypes.c_int32),
                ("bu_levels", ctypes.c_int32), ("reached", ctypes.c_int64), ("teps_edges", ctypes.c_int64),
                ("edges_examined", ctypes.c_int64), ("alg_bytes", ctypes.c_int64)]


class dobfs_level_trace(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("direction", ctypes.c_int32), ("n_frontier", ctypes.c_int64),
                ("m_frontier", ctypes.c_int64), ("m_unvisited", ctypes.c_int64), ("n_next", ctypes.c_int64),
                ("edges_examined", ctypes.c_int64), ("vertices_scanned", ctypes.c_int64),
                ("alg_bytes", ctypes.c_int64), ("ms", ctypes.c_float), ("ms_main", ctypes.c_float)]


class dobfs_serve_opts(ctypes.Structure):
    _fields_ = [("max_device_bytes", ctypes.c_int64), ("groups_per_graph", ctypes.c_int32),
                ("max_groups_per_graph", ctypes.c_int32), ("alpha", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("admit_div", ctypes.c_int32), ("join_window", ctypes.c_int32),
                ("flush_delay", ctypes.c_int32), ("gather_us", ctypes.c_int32), ("ss_max", ctypes.c_int32),
                ("ss_backlog", ctypes.c_int32), ("lane_words", ctypes.c_int32)]


class dobfs_query_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("levels", ctypes.c_int32), ("submit_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64), ("latency_ns", ctypes.c_int64)]


class dobfs_serve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("completed", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("groups_created", ctypes.c_int64), ("reserved_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("cohorts", ctypes.c_int64), ("lanes_admitted", ctypes.c_int64),
                ("group_steps", ctypes.c_int64), ("single_source", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def load() -> ctypes.CDLL:
    """Loads libdobfs.so; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdobfs.so not built (%s); run python -m paper_1503_04359_b300.build" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    c_int, i64, i32, u32, u64, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    G = ctypes.c_void_p
    sig = {
        "dobfs_set_allocator": (c_int, [ALLOC_FN, FREE_FN, vp]),
        "dobfs_last_error": (ctypes.c_char_p, []),
        "dobfs_graph_create": (c_int, [vp, c_int, vp, i64, i64, u32, vp, ctypes.POINTER(G)]),
        "dobfs_graph_create_from_pairs": (c_int, [vp, vp, i64, i64, u32, vp, ctypes.POINTER(G)]),
        "dobfs_graph_create_rmat": (c_int, [c_int, i64, u32, u32, u32, u64, u32, vp, ctypes.POINTER(G)]),
        "dobfs_graph_create_chunglu": (c_int, [vp, i64, i64, u64, u32, vp, ctypes.POINTER(G)]),
        "dobfs_graph_destroy": (c_int, [G]),
        "dobfs_graph_get_info": (c_int, [G, ctypes.POINTER(dobfs_graph_info)]),
        "dobfs_graph_export": (c_int, [G, vp, vp, vp, vp]),
        "dobfs_graph_degrees": (c_int, [G, vp, vp]),
        "dobfs_graph_save": (c_int, [G, ctypes.c_char_p, vp]),
        "dobfs_debug_set_column": (c_int, [G, i64, i32]),
        "dobfs_debug_grid_barrier": (c_int, [i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                             ctypes.POINTER(i32)]),
        "dobfs_debug_random_access": (c_int, [i64, i64, i32, i32, ctypes.POINTER(ctypes.c_float),
                                              ctypes.POINTER(i64)]),
        "dobfs_graph_wait": (c_int, [G, i32]),
        "dobfs_graph_load": (c_int, [ctypes.c_char_p, u32, vp, ctypes.POINTER(G)]),
        "dobfs_run_opts_init": (c_int, [ctypes.POINTER(dobfs_run_opts)]),
        "dobfs_run": (c_int, [G, i32, vp, vp, ctypes.POINTER(dobfs_run_opts), ctypes.POINTER(dobfs_run_stats)]),
        "dobfs_last_trace": (c_int, [G, ctypes.POINTER(dobfs_level_trace), i32, ctypes.POINTER(i32)]),
        "dobfs_run_static": (c_int, [vp, vp, i32, i32, vp, vp, vp]),
        "dobfs_run_batch": (c_int, [G, vp, i32, vp, vp, ctypes.POINTER(dobfs_run_opts), ctypes.POINTER(dobfs_run_stats)]),
        "dobfs_serve_opts_init": (c_int, [ctypes.POINTER(dobfs_serve_opts)]),
        "dobfs_serve_create": (c_int, [ctypes.POINTER(dobfs_serve_opts), ctypes.POINTER(vp)]),
        "dobfs_serve_add_graph": (c_int, [vp, G, ctypes.POINTER(i32)]),
        "dobfs_serve_submit": (c_int, [vp, i32, i32, vp, vp, ctypes.POINTER(u64)]),
        "dobfs_serve_poll": (c_int, [vp, u64, ctypes.POINTER(dobfs_query_result)]),
        "dobfs_serve_get_stats": (c_int, [vp, ctypes.POINTER(dobfs_serve_stats)]),
        "dobfs_serve_collect": (c_int, [vp, ctypes.POINTER(u64), ctypes.POINTER(dobfs_query_result), i32,
                                        ctypes.POINTER(i32)]),
        "dobfs_serve_destroy": (c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().dobfs_last_error().decode(errors="replace")


def _check(status: int) -> int:
    if status < 0:
        raise DobfsError(status, last_error())
    return status


def _ptr(x) -> int | None:
    """Data pointer of a torch tensor or numpy array (None for None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "array must be C-contiguous"
        return x.ctypes.data
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(x))


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------- allocator
_alloc_keepalive = None


def use_torch_allocator(device: int | None = None) -> None:
    """Routes every device allocation of the library through PyTorch's caching allocator."""
    global _alloc_keepalive
    import torch
    dev = torch.cuda.current_device() if device is None else device

    @ALLOC_FN
    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:  # OOM -> NULL -> DOBFS_ERR_OOM
            return None

    @FREE_FN
    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _check(load().dobfs_set_allocator(_alloc, _free, None))
    _alloc_keepalive = (_alloc, _free)


def use_default_allocator() -> None:
    global _alloc_keepalive
    _check(load().dobfs_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _alloc_keepalive = None


# ---------------------------------------------------------------- C entry points (same names)
def dobfs_graph_create(row_offsets, col_indices, n_vertices: int, flags: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    off64 = 1 if str(getattr(row_offsets, "dtype", "")).endswith("int64") else 0
    n_entries = int(col_indices.shape[0]) if col_indices is not None else 0
    _check(load().dobfs_graph_create(_ptr(row_offsets), off64, _ptr(col_indices), n_vertices, n_entries, flags,
                                     _stream(stream), ctypes.byref(h)))
    return h.value


def dobfs_graph_create_from_pairs(src, dst, n_vertices: int, flags: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().dobfs_graph_create_from_pairs(_ptr(src), _ptr(dst), int(src.shape[0]), n_vertices, flags,
                                                _stream(stream), ctypes.byref(h)))
    return h.value


def dobfs_graph_create_rmat(scale: int, n_pairs: int, t_a: int, t_ab: int, t_abc: int, seed: int, flags: int = 0,
                            stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().dobfs_graph_create_rmat(scale, n_pairs, t_a, t_ab, t_abc, seed, flags, _stream(stream),
                                          ctypes.byref(h)))
    return h.value


def dobfs_graph_create_chunglu(cdf: np.ndarray, n_pairs: int, seed: int, flags: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    cdf = np.ascontiguousarray(cdf, dtype=np.uint64)
    _check(load().dobfs_graph_create_chunglu(cdf.ctypes.data, len(cdf), n_pairs, seed, flags, _stream(stream),
                                             ctypes.byref(h)))
    return h.value


def dobfs_graph_destroy(g: int) -> None:
    _check(load().dobfs_graph_destroy(g))


def dobfs_graph_get_info(g: int) -> dobfs_graph_info:
    info = dobfs_graph_info()
    _check(load().dobfs_graph_get_info(g, ctypes.byref(info)))
    return info


def dobfs_graph_export(g: int, offsets_out=None, cols_out=None, new2orig_out=None, stream=None) -> None:
    _check(load().dobfs_graph_export(g, _ptr(offsets_out), _ptr(cols_out), _ptr(new2orig_out), _stream(stream)))


def dobfs_graph_degrees(g: int, deg_out, stream=None) -> None:
    _check(load().dobfs_graph_degrees(g, _ptr(deg_out), _stream(stream)))


def dobfs_debug_set_column(g: int, pos: int, value: int) -> None:
    _check(load().dobfs_debug_set_column(g, pos, value))


def dobfs_debug_grid_barrier(blocks: int, rounds: int, missing: int = 0) -> tuple[int, int, bool]:
    """(rounds passed, rounds with a short count, timed out) of the grid-barrier self-test."""
    p, sc, to = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().dobfs_debug_grid_barrier(int(blocks), int(rounds), int(missing), ctypes.byref(p),
                                           ctypes.byref(sc), ctypes.byref(to)))
    return p.value, sc.value, bool(to.value)


def dobfs_debug_random_access(array_bytes: int, accesses: int, width: int, write: bool = False) -> tuple[float, int]:
    """(milliseconds, accesses made) of one launch of scattered accesses (see the header)."""
    ms, made = ctypes.c_float(), ctypes.c_int64()
    _check(load().dobfs_debug_random_access(int(array_bytes), int(accesses), int(width), int(bool(write)),
                                            ctypes.byref(ms), ctypes.byref(made)))
    return ms.value, made.value


def dobfs_graph_wait(g: int, timeout_ms: int = -1) -> bool:
    """True once the graph's queued work is done, False if it is still running
    after timeout_ms (< 0: no limit); raises if it failed."""
    st = load().dobfs_graph_wait(g, int(timeout_ms))
    if st == DOBFS_ERR_TIMEOUT:
        return False
    _check(st)
    return True


def dobfs_graph_save(g: int, path: str, stream=None) -> None:
    _check(load().dobfs_graph_save(g, os.fsencode(path), _stream(stream)))


def dobfs_graph_load(path: str, flags: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().dobfs_graph_load(os.fsencode(path), flags, _stream(stream), ctypes.byref(h)))
    return h.value


def make_opts(direction: int = DOBFS_DIR_AUTO, alpha: int | None = None, beta: int | None = None,
              static_pct: int | None = None, bu_steps: int | None = None, flags: int = 0, schedule_seed: int = 0,
              stream=None, td_bitmap_div: int | None = None, td_small_max: int | None = None,
              td_chunk: int | None = None, bu_scan: int | None = None,
              td_split_pct: int | None = None, bu_threads: int | None = None, td_threads: int | None = None,
              out_threads: int | None = None) -> dobfs_run_opts:
    o = dobfs_run_opts()
    _check(load().dobfs_run_opts_init(ctypes.byref(o)))
    o.direction = direction
    if alpha is not None:
        o.alpha = alpha
    if beta is not None:
        o.beta = beta
    if static_pct is not None:
        o.static_pct = static_pct
    if bu_steps is not None:
        o.bu_steps = bu_steps
    if td_bitmap_div is not None:
        o.td_bitmap_div = td_bitmap_div
    if td_small_max is not None:
        o.td_small_max = td_small_max
    if td_chunk is not None:
        o.td_chunk = td_chunk
    if bu_scan is not None:
        o.bu_scan = bu_scan
    if td_split_pct is not None:
        o.td_split_pct = td_split_pct
    if bu_threads is not None:
        o.bu_threads = bu_threads
    if td_threads is not None:
        o.td_threads = td_threads
    if out_threads is not None:
        o.out_threads = out_threads
    o.flags = flags
    o.schedule_seed = schedule_seed
    o.stream = _stream(stream)
    return o


def dobfs_run(g: int, root: int, level_out, parent_out=None, opts: dobfs_run_opts | None = None,
              want_stats: bool = False) -> dobfs_run_stats | None:
    if opts is None:
        opts = make_opts()
    st = dobfs_run_stats() if want_stats else None
    _check(load().dobfs_run(g, int(root), _ptr(level_out), _ptr(parent_out), ctypes.byref(opts),
                            ctypes.byref(st) if st is not None else None))
    return st


def dobfs_run_batch(g: int, roots, level_out, parent_out=None, opts: dobfs_run_opts | None = None,
                    want_stats: bool = False) -> dobfs_run_stats | None:
    """Batched BFS: level_out[len(roots)][n] receives one level row per root."""
    if opts is None:
        opts = make_opts()
    st = dobfs_run_stats() if want_stats else None
    _check(load().dobfs_run_batch(g, _ptr(roots), int(roots.shape[0]), _ptr(level_out), _ptr(parent_out),
                                  ctypes.byref(opts), ctypes.byref(st) if st is not None else None))
    return st


def dobfs_run_opts_init() -> dobfs_run_opts:
    o = dobfs_run_opts()
    _check(load().dobfs_run_opts_init(ctypes.byref(o)))
    return o


def dobfs_serve_opts_init() -> dobfs_serve_opts:
    o = dobfs_serve_opts()
    _check(load().dobfs_serve_opts_init(ctypes.byref(o)))
    return o


def make_serve_opts(max_device_bytes: int = 0, groups_per_graph: int | None = None,
                    max_groups_per_graph: int | None = None,
                    alpha: int | None = None, beta: int | None = None, direction: int = DOBFS_DIR_AUTO,
                    admit_div: int | None = None, join_window: int | None = None,
                    flush_delay: int | None = None, gather_us: int | None = None, ss_max: int | None = None,
                    ss_backlog: int | None = None, lane_words: int | None = None) -> dobfs_serve_opts:
    o = dobfs_serve_opts()
    _check(load().dobfs_serve_opts_init(ctypes.byref(o)))
    if admit_div is not None:
        o.admit_div = admit_div
    if join_window is not None:
        o.join_window = join_window
    if flush_delay is not None:
        o.flush_delay = flush_delay
    if gather_us is not None:
        o.gather_us = gather_us
    if lane_words is not None:
        o.lane_words = lane_words
    if ss_max is not None:
        o.ss_max = ss_max
    if ss_backlog is not None:
        o.ss_backlog = ss_backlog
    o.max_device_bytes = max_device_bytes
    if groups_per_graph is not None:
        o.groups_per_graph = groups_per_graph
    if max_groups_per_graph is not None:
        o.max_groups_per_graph = max_groups_per_graph
    if alpha is not None:
        o.alpha = alpha
    if beta is not None:
        o.beta = beta
    o.direction = direction
    return o


def dobfs_serve_create(opts: dobfs_serve_opts | None = None) -> int:
    h = ctypes.c_void_p()
    _check(load().dobfs_serve_create(ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
    return h.value


def dobfs_serve_add_graph(server: int, g: int) -> int:
    gid = ctypes.c_int32()
    _check(load().dobfs_serve_add_graph(server, g, ctypes.byref(gid)))
    return gid.value


def dobfs_serve_submit(server: int, gid: int, root: int, level_out, parent_out=None) -> int:
    t = ctypes.c_uint64()
    _check(load().dobfs_serve_submit(server, int(gid), int(root), _ptr(level_out), _ptr(parent_out),
                                     ctypes.byref(t)))
    return t.value


def dobfs_serve_poll(server: int, ticket: int) -> dobfs_query_result | None:
    """The result once the query is done, None while it is pending; raises if it failed."""
    r = dobfs_query_result()
    st = _check(load().dobfs_serve_poll(server, int(ticket), ctypes.byref(r)))
    return None if st == DOBFS_PENDING else r


class Collector:
    """Reusable buffers for dobfs_serve_collect."""

    def __init__(self, cap: int = 4096):
        self.cap = cap
        self.tickets = (ctypes.c_uint64 * cap)()
        self.results = (dobfs_query_result * cap)()
        self.n = ctypes.c_int32()


def dobfs_serve_collect(server: int, col: Collector) -> list[tuple[int, dobfs_query_result]]:
    _check(load().dobfs_serve_collect(server, col.tickets, col.results, col.cap, ctypes.byref(col.n)))
    return [(col.tickets[i], col.results[i]) for i in range(col.n.value)]


def dobfs_serve_get_stats(server: int) -> dobfs_serve_stats:
    st = dobfs_serve_stats()
    _check(load().dobfs_serve_get_stats(server, ctypes.byref(st)))
    return st


def dobfs_serve_destroy(server: int) -> None:
    _check(load().dobfs_serve_destroy(server))


def dobfs_last_trace(g: int, max_levels: int = 4096) -> list[dobfs_level_trace]:
    buf = (dobfs_level_trace * max_levels)()
    n = ctypes.c_int32(0)
    _check(load().dobfs_last_trace(g, buf, max_levels, ctypes.byref(n)))
    return [buf[i] for i in range(n.value)]


def dobfs_run_static(row_offsets, col_indices, n_vertices: int, root: int, level_out, parent_out=None,
                     stream=None) -> None:
    """BFS on a caller's device CSR (int32 offsets) with no device allocation: the
    library's working memory is a fixed static device array (see include/dobfs.h)."""
    _check(load().dobfs_run_static(_ptr(row_offsets), _ptr(col_indices), int(n_vertices), int(root),
                                   _ptr(level_out), _ptr(parent_out), _stream(stream)))


# ---------------------------------------------------------------- convenience wrapper
@dataclass
class Graph:
    """Owning handle of a device graph."""

    handle: int

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            try:
                dobfs_graph_destroy(self.handle)
            finally:
                self.handle = 0

    @property
    def info(self) -> dobfs_graph_info:
        return dobfs_graph_get_info(self.handle)

    @property
    def n(self) -> int:
        return int(self.info.n_vertices)

    def export(self):
        """(offsets int64[n+1], cols int32[nnz], new2orig int32[n]) as numpy arrays."""
        info = self.info
        off = np.empty(info.n_vertices + 1, dtype=np.int64)
        cols = np.empty(max(info.n_entries, 1), dtype=np.int32)
        n2o = np.empty(info.n_vertices, dtype=np.int32)
        dobfs_graph_export(self.handle, off, cols, n2o)
        return off, cols[:info.n_entries], n2o

    def degrees(self, out=None):
        if out is None:
            out = np.empty(self.n, dtype=np.int32)
        dobfs_graph_degrees(self.handle, out)
        return out

    def save(self, path: str) -> None:
        """Writes the graph file `path` (dobfs_graph_save)."""
        dobfs_graph_save(self.handle, path)

    def run(self, root: int, level_out, parent_out=None, opts=None, want_stats: bool = False):
        return dobfs_run(self.handle, root, level_out, parent_out, opts, want_stats)

    def wait(self, timeout_ms: int = -1) -> bool:
        return dobfs_graph_wait(self.handle, timeout_ms)

    def trace(self):
        return dobfs_last_trace(self.handle)


def rmat_graph(spec, flags: int = DOBFS_GRAPH_REINDEX, stream=None) -> Graph:
    """Device graph of a dobfs_inputs.RmatSpec workload."""
    ta, tab, tabc = spec.thresholds
    return Graph(dobfs_graph_create_rmat(spec.scale, spec.n_pairs, ta, tab, tabc, spec.seed, flags, stream))


def chunglu_graph(spec, cdf: np.ndarray, flags: int = DOBFS_GRAPH_REINDEX, stream=None) -> Graph:
    return Graph(dobfs_graph_create_chunglu(cdf, spec.n_pairs, spec.seed, flags, stream))


def load_graph(path: str, validate: bool = False, stream=None) -> Graph:
    """Device graph read from a graph file written by Graph.save (dobfs_graph_load)."""
    return Graph(dobfs_graph_load(path, DOBFS_GRAPH_VALIDATE if validate else 0, stream))


def pairs_graph(n_vertices: int, src, dst, flags: int = 0, stream=None) -> Graph:
    return Graph(dobfs_graph_create_from_pairs(src, dst, n_vertices, flags, stream))


def csr_graph(row_offsets, col_indices, n_vertices: int, flags: int = 0, stream=None) -> Graph:
    return Graph(dobfs_graph_create(row_offsets, col_indices, n_vertices, flags, stream))
