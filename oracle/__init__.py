"""CPU oracle for direction-optimized BFS — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package. It shares no code
with the CUDA library in ``paper_1503_04359_b300``; both read their inputs from
``dobfs_inputs`` only.

What it computes (see ``dobfs_oracle.c`` for the passages followed):

* ``csr_from_pairs`` / ``csr_from_rmat`` — the undirected graph as CSR, each
  undirected edge stored as two directed edges, self-loops and duplicates
  dropped, rows sorted (Sec. 4, "Methodology").
* ``csr_from_rmat_par`` / ``csr_from_pairs_par`` — the same CSRs built by
  several threads (host graphs of billions of entries).
* ``bfs`` — serial FIFO-queue BFS: level = hop distance (the result every
  top-down / bottom-up schedule of Algorithm 1 reaches), canonical parent =
  smallest-ID neighbour one level up.
* ``bfs_partial`` — the same BFS stopped after a given number of adjacency
  entries (a bounded timing sample on graphs too large to traverse on one
  core in the time allowed); every level it writes is the full BFS level.
* ``check_bfs`` / ``check_bfs_rmat_stream`` — the BFS invariants (level[root]=0,
  |level(u)-level(v)| <= 1 on every edge, every reached vertex has a neighbour
  one level up, every parent a neighbour one level up, reached set = the
  root's union-find component).
* ``teps_edges`` — undirected edges in the traversed component, the TEPS
  numerator (Sec. 4, "Methodology").
* ``brute_levels`` (``brute.py``) — levels from boolean matrix powers, for
  graphs with at most a few dozen vertices.

Pins (tests/test_oracle.py): brute force on all roots of random tiny graphs;
closed forms (path, cycle, star, complete graph, binary tree, grid, Petersen
graph, disjoint unions, isolated root); planted mistakes caught by the
invariant checker; the threaded CSR equal to the set-based and serial ones;
the stopped BFS a prefix of the closed-form path levels and, with no limit,
equal to the full BFS. Parity status: levels and canonical parents pinned; no
numeric example is printed in the paper, so no value is taken from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .brute import brute_levels, brute_canonical_parent  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dobfs_oracle.c")
_GEN_H = os.path.join(os.path.dirname(_HERE), "dobfs_inputs", "gen.h")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lib = None

RULES = {
    0: "ok",
    1: "level[root] != 0",
    2: "parent[root] != root",
    3: "edge spans more than one level",
    4: "edge joins reached and unreached vertex",
    5: "parent is not a neighbour",
    6: "parent is not one level up",
    7: "unreached vertex with level/parent not -1",
    8: "reached set differs from root component",
    9: "parent is not a neighbour (stream check)",
    10: "reached vertex without a neighbour one level up",
}


def build(force: bool = False) -> str:
    """Compile dobfs_oracle.c with gcc into _oracle.so (OpenMP for the
    multi-root driver and the streaming check)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_GEN_H))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, i32, u32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
        P64, P32, P8 = ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_csr_from_pairs.restype = i64
        lib.oracle_csr_from_pairs.argtypes = [i64, i64, P32, P32, P64, P32]
        lib.oracle_csr_from_rmat.restype = i64
        lib.oracle_csr_from_rmat.argtypes = [ctypes.c_int, i64, u32, u32, u32, u64, P64, P32]
        lib.oracle_csr_from_rmat_par.restype = i64
        lib.oracle_csr_from_rmat_par.argtypes = [ctypes.c_int, i64, u32, u32, u32, u64, P64, P32, i32]
        lib.oracle_csr_from_pairs_par.restype = i64
        lib.oracle_csr_from_pairs_par.argtypes = [i64, i64, P32, P32, P64, P32, i32]
        lib.oracle_bfs.restype = i32
        lib.oracle_bfs.argtypes = [i64, P64, P32, i32, P32, P32]
        lib.oracle_bfs_partial.restype = i64
        lib.oracle_bfs_partial.argtypes = [i64, P64, P32, i32, P32, i64]
        lib.oracle_bfs_many.restype = None
        lib.oracle_bfs_many.argtypes = [i64, P64, P32, i32, P32, P32, P32, i32]
        lib.oracle_components.restype = None
        lib.oracle_components.argtypes = [i64, P64, P32, P32]
        lib.oracle_check_bfs.restype = i32
        lib.oracle_check_bfs.argtypes = [i64, P64, P32, i32, P32, P32, P64]
        lib.oracle_teps_edges.restype = i64
        lib.oracle_teps_edges.argtypes = [i64, P64, P32]
        lib.oracle_check_bfs_rmat_stream.restype = i32
        lib.oracle_check_bfs_rmat_stream.argtypes = [ctypes.c_int, i64, u32, u32, u32, u64, i32, P32, P32,
                                                     P32, P8, i32, P64]
        lib.oracle_check_bfs_rmat_stream_multi.restype = i32
        lib.oracle_check_bfs_rmat_stream_multi.argtypes = [ctypes.c_int, i64, u32, u32, u32, u64, i32, P32, P32,
                                                           P32, P32, i32, P32, P64, i32]
        lib.oracle_check_bfs_pairs_multi.restype = i32
        lib.oracle_check_bfs_pairs_multi.argtypes = [i64, i64, P32, P32, i32, P32, P32, P32, P32, P8, i32, P32, P64,
                                                     i32]
        _lib = lib
    return _lib


class Csr:
    """Host CSR built by the oracle: off int64[n+1], cols int32[nnz]."""

    def __init__(self, off: np.ndarray, cols: np.ndarray):
        self.off = off
        self.cols = cols

    @property
    def n(self) -> int:
        return len(self.off) - 1

    @property
    def nnz(self) -> int:
        return int(self.off[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.off)

    def row(self, u: int) -> np.ndarray:
        return self.cols[self.off[u]:self.off[u + 1]]


def csr_from_pairs(n: int, src, dst) -> Csr:
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = len(src)
    off = np.zeros(n + 1, dtype=np.int64)
    cols = np.empty(max(2 * m, 1), dtype=np.int32)
    nnz = lib.oracle_csr_from_pairs(n, m, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                                    _p(off, ctypes.c_int64), _p(cols, ctypes.c_int32))
    if nnz < 0:
        raise ValueError("endpoint out of range")
    return Csr(off, cols[:nnz].copy())


def csr_from_rmat(spec) -> Csr:
    """CSR of an R-MAT workload (dobfs_inputs.RmatSpec), pairs regenerated in two passes."""
    lib = _load()
    n, m = spec.n_vertices, spec.n_pairs
    off = np.zeros(n + 1, dtype=np.int64)
    cols = np.empty(2 * m, dtype=np.int32)
    ta, tab, tabc = spec.thresholds
    nnz = lib.oracle_csr_from_rmat(spec.scale, m, ta, tab, tabc, spec.seed, _p(off, ctypes.c_int64),
                                   _p(cols, ctypes.c_int32))
    return Csr(off, cols[:nnz].copy())


def csr_from_rmat_par(spec, n_threads: int | None = None) -> Csr:
    """The CSR of csr_from_rmat built by several threads (host graphs of
    billions of entries). The column array is returned as a view of the
    placement buffer (2 * n_pairs entries) to avoid a second copy."""
    lib = _load()
    n, m = spec.n_vertices, spec.n_pairs
    off = np.zeros(n + 1, dtype=np.int64)
    cols = np.empty(2 * m, dtype=np.int32)
    ta, tab, tabc = spec.thresholds
    nnz = lib.oracle_csr_from_rmat_par(spec.scale, m, ta, tab, tabc, spec.seed, _p(off, ctypes.c_int64),
                                       _p(cols, ctypes.c_int32), n_threads or os.cpu_count() or 1)
    return Csr(off, cols[:nnz])


def csr_from_pairs_par(n: int, src, dst, n_threads: int | None = None) -> Csr:
    """The CSR of csr_from_pairs built by several threads; the column array is
    a view of the placement buffer."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = len(src)
    off = np.zeros(n + 1, dtype=np.int64)
    cols = np.empty(max(2 * m, 1), dtype=np.int32)
    nnz = lib.oracle_csr_from_pairs_par(n, m, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                                        _p(off, ctypes.c_int64), _p(cols, ctypes.c_int32),
                                        n_threads or os.cpu_count() or 1)
    if nnz < 0:
        raise ValueError("endpoint out of range")
    return Csr(off, cols[:nnz])


def bfs(g: Csr, root: int, want_parent: bool = True):
    """Serial BFS: (level, canonical parent or None, number of levels)."""
    lib = _load()
    level = np.empty(g.n, dtype=np.int32)
    parent = np.empty(g.n, dtype=np.int32) if want_parent else None
    nlev = lib.oracle_bfs(g.n, _p(g.off, ctypes.c_int64), _p(g.cols, ctypes.c_int32), int(root),
                          _p(level, ctypes.c_int32), _p(parent, ctypes.c_int32) if want_parent else None)
    return level, parent, nlev


def bfs_partial(g: Csr, root: int, max_entries: int):
    """The serial BFS stopped after reading max_entries adjacency entries:
    (level, entries read). Every level written is the full BFS level."""
    lib = _load()
    level = np.empty(g.n, dtype=np.int32)
    read = lib.oracle_bfs_partial(g.n, _p(g.off, ctypes.c_int64), _p(g.cols, ctypes.c_int32), int(root),
                                  _p(level, ctypes.c_int32), int(max_entries))
    return level, int(read)


def bfs_many(g: Csr, roots, want_parent: bool = True, n_threads: int | None = None):
    """oracle BFS for every root (OpenMP over roots): level [R, n], parent [R, n] or None."""
    lib = _load()
    roots = np.ascontiguousarray(roots, dtype=np.int32)
    r = len(roots)
    level = np.empty((r, g.n), dtype=np.int32)
    parent = np.empty((r, g.n), dtype=np.int32) if want_parent else None
    lib.oracle_bfs_many(g.n, _p(g.off, ctypes.c_int64), _p(g.cols, ctypes.c_int32), r,
                        _p(roots, ctypes.c_int32), _p(level, ctypes.c_int32),
                        _p(parent, ctypes.c_int32) if want_parent else None,
                        n_threads or os.cpu_count() or 1)
    return level, parent


def components(g: Csr) -> np.ndarray:
    lib = _load()
    comp = np.empty(g.n, dtype=np.int32)
    lib.oracle_components(g.n, _p(g.off, ctypes.c_int64), _p(g.cols, ctypes.c_int32), _p(comp, ctypes.c_int32))
    return comp


def check_bfs(g: Csr, root: int, level, parent=None) -> tuple[int, int]:
    """(rule, vertex): rule 0 when every BFS invariant holds."""
    lib = _load()
    level = np.ascontiguousarray(level, dtype=np.int32)
    if parent is not None:
        parent = np.ascontiguousarray(parent, dtype=np.int32)
    bad = ctypes.c_int64(0)
    rc = lib.oracle_check_bfs(g.n, _p(g.off, ctypes.c_int64), _p(g.cols, ctypes.c_int32), int(root),
                              _p(level, ctypes.c_int32),
                              _p(parent, ctypes.c_int32) if parent is not None else None, ctypes.byref(bad))
    return int(rc), int(bad.value)


def teps_edges(g: Csr, level) -> int:
    lib = _load()
    level = np.ascontiguousarray(level, dtype=np.int32)
    return int(lib.oracle_teps_edges(g.n, _p(g.off, ctypes.c_int64), _p(level, ctypes.c_int32)))


def check_bfs_rmat_stream(spec, root: int, level, parent=None, want_canon: bool = False,
                          want_has_nbr: bool = False, n_threads: int | None = None):
    """Invariant check of a BFS on an R-MAT workload with the pairs regenerated
    (no CSR held). Returns (rule, vertex, canon or None, has_nbr or None)."""
    lib = _load()
    n = spec.n_vertices
    level = np.ascontiguousarray(level, dtype=np.int32)
    if parent is not None:
        parent = np.ascontiguousarray(parent, dtype=np.int32)
    canon = np.empty(n, dtype=np.int32) if want_canon else None
    has_nbr = np.empty(n, dtype=np.uint8) if want_has_nbr else None
    bad = ctypes.c_int64(0)
    ta, tab, tabc = spec.thresholds
    rc = lib.oracle_check_bfs_rmat_stream(
        spec.scale, spec.n_pairs, ta, tab, tabc, spec.seed, int(root), _p(level, ctypes.c_int32),
        _p(parent, ctypes.c_int32) if parent is not None else None,
        _p(canon, ctypes.c_int32) if want_canon else None,
        _p(has_nbr, ctypes.c_uint8) if want_has_nbr else None,
        n_threads or os.cpu_count() or 1, ctypes.byref(bad))
    return int(rc), int(bad.value), canon, has_nbr


def _multi_outputs(roots, levels, parents, n, want_canon, vertex_major):
    roots = np.ascontiguousarray(roots, dtype=np.int32)
    R = len(roots)
    shape = (n, R) if vertex_major else (R, n)
    levels = np.ascontiguousarray(levels, dtype=np.int32).reshape(shape)
    if parents is not None:
        parents = np.ascontiguousarray(parents, dtype=np.int32).reshape(shape)
    canon = np.empty(shape, dtype=np.int32) if want_canon else None
    return roots, R, levels, parents, canon


def check_bfs_rmat_stream_multi(spec, roots, levels, parents=None, want_canon=False, n_threads=None,
                                vertex_major=False):
    """Streaming invariant check of R BFS results on an R-MAT workload in one
    pass over the regenerated pairs. levels / parents are [R, n], or [n, R]
    with vertex_major (a pair's entries for all roots side by side: far less
    memory traffic for many roots). Returns (rules[R], bad[R], canon or None),
    canon in the layout of levels."""
    lib = _load()
    n = spec.n_vertices
    roots, R, levels, parents, canon = _multi_outputs(roots, levels, parents, n, want_canon, vertex_major)
    rc = np.zeros(R, dtype=np.int32)
    bad = np.zeros(R, dtype=np.int64)
    ta, tab, tabc = spec.thresholds
    lib.oracle_check_bfs_rmat_stream_multi(
        spec.scale, spec.n_pairs, ta, tab, tabc, spec.seed, R, _p(roots, ctypes.c_int32), _p(levels, ctypes.c_int32),
        _p(parents, ctypes.c_int32) if parents is not None else None,
        _p(canon, ctypes.c_int32) if want_canon else None, n_threads or os.cpu_count() or 1,
        _p(rc, ctypes.c_int32), _p(bad, ctypes.c_int64), 1 if vertex_major else 0)
    return rc, bad, canon


def check_bfs_pairs_multi(n, src, dst, roots, levels, parents=None, want_canon=False, want_has_nbr=False,
                          n_threads=None, vertex_major=False):
    """Streaming invariant check of R BFS results on the graph of the pairs (src, dst)
    (layouts as for check_bfs_rmat_stream_multi).
    Returns (rules[R], bad[R], canon or None, has_nbr or None)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    roots, R, levels, parents, canon = _multi_outputs(roots, levels, parents, n, want_canon, vertex_major)
    has_nbr = np.empty(n, dtype=np.uint8) if want_has_nbr else None
    rc = np.zeros(R, dtype=np.int32)
    bad = np.zeros(R, dtype=np.int64)
    lib.oracle_check_bfs_pairs_multi(
        n, len(src), _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32), R, _p(roots, ctypes.c_int32),
        _p(levels, ctypes.c_int32), _p(parents, ctypes.c_int32) if parents is not None else None,
        _p(canon, ctypes.c_int32) if want_canon else None,
        _p(has_nbr, ctypes.c_uint8) if want_has_nbr else None, n_threads or os.cpu_count() or 1,
        _p(rc, ctypes.c_int32), _p(bad, ctypes.c_int64), 1 if vertex_major else 0)
    return rc, bad, canon, has_nbr
