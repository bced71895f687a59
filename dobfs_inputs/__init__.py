"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no BFS arithmetic. It defines the graph workloads (R-MAT with
Graph500 quadrant probabilities, Chung-Lu power-law graphs), their seeds, the
integer thresholds and weight tables the generators in ``gen.h`` consume, and
the seeded root sampler. The paper measures on Graph500 synthetic graphs built
with the Graph500 reference generator and parameters (Sec. 4, "Workloads"); that
code is not available here, so the R-MAT stream of ``gen.h`` with the same
quadrant probabilities and edge factor stands in for it.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_gen.so")
_lib = None

MASK64 = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile the host batch generator (gen_lib.c) into _gen.so."""
    src = os.path.join(_HERE, "gen_lib.c")
    hdr = os.path.join(_HERE, "gen.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u32, u64, i64, i32p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
        lib.gen_c_mix64.restype = u64
        lib.gen_c_mix64.argtypes = [u64]
        lib.gen_c_perm.restype = u32
        lib.gen_c_perm.argtypes = [u32, u32, u64]
        for name in ("gen_c_rmat_pairs", "gen_c_rmat_pairs_raw"):
            f = getattr(lib, name)
            f.restype = None
            f.argtypes = [ctypes.c_int, u32, u32, u32, u64, u64, i64, i32p, i32p]
        lib.gen_c_chunglu_pairs.restype = None
        lib.gen_c_chunglu_pairs.argtypes = [ctypes.POINTER(ctypes.c_uint64), u32, u64, u64, i64, i32p, i32p, ctypes.c_int]
        _lib = lib
    return _lib


def mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood 2014), as in gen.h."""
    z = (z + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


# --------------------------------------------------------------------------- R-MAT
@dataclasses.dataclass(frozen=True)
class RmatSpec:
    """R-MAT workload: 2^scale vertices, edgefactor * 2^scale undirected pairs."""

    scale: int
    edgefactor: int = 16
    a: float = 0.57
    b: float = 0.19
    c: float = 0.19
    seed: int = 0

    @property
    def n_vertices(self) -> int:
        return 1 << self.scale

    @property
    def n_pairs(self) -> int:
        return self.edgefactor << self.scale

    @property
    def thresholds(self) -> tuple[int, int, int]:
        return rmat_thresholds(self.a, self.b, self.c)


def rmat_thresholds(a: float, b: float, c: float) -> tuple[int, int, int]:
    """Integer cut points on a 32-bit uniform draw for quadrants A | B | C | D."""
    def cut(p: float) -> int:
        return max(0, min((1 << 32) - 1, int(math.floor(p * 4294967296.0))))
    return cut(a), cut(a + b), cut(a + b + c)


def rmat_seed(scale: int) -> int:
    """Graph seed of the R-MAT workloads at `scale` (one fixed seed per scale)."""
    return 0x5EED0000 + scale


def root_seed(graph_seed: int) -> int:
    return graph_seed ^ 0xB00F


def rmat(scale: int, edgefactor: int = 16, seed: int | None = None) -> RmatSpec:
    return RmatSpec(scale=scale, edgefactor=edgefactor, seed=rmat_seed(scale) if seed is None else seed)


def rmat_pairs(spec: RmatSpec, k0: int = 0, count: int | None = None, relabel: bool = True):
    """Pairs k0 .. k0+count-1 of the R-MAT stream as two int32 arrays."""
    lib = _load()
    if count is None:
        count = spec.n_pairs - k0
    src = np.empty(count, dtype=np.int32)
    dst = np.empty(count, dtype=np.int32)
    f = lib.gen_c_rmat_pairs if relabel else lib.gen_c_rmat_pairs_raw
    ta, tab, tabc = spec.thresholds
    f(spec.scale, ta, tab, tabc, spec.seed, k0, count, _i32p(src), _i32p(dst))
    return src, dst


def perm(x: int, n: int, seed: int) -> int:
    """The seeded relabelling bijection of [0, n) used by the generators."""
    return int(_load().gen_c_perm(x, n, seed))


# --------------------------------------------------------------------------- Chung-Lu
@dataclasses.dataclass(frozen=True)
class ChungLuSpec:
    """Chung-Lu power-law workload: weights w_i = c (i + i0)^(-1/(gamma-1)),
    c and i0 chosen so that max w = max_weight and mean w = mean_degree;
    n * mean_degree / 2 undirected pairs."""

    log2_n: int
    gamma: float = 2.1
    mean_degree: float = 35.0
    max_weight: float = float(1 << 20)
    seed: int = 0

    @property
    def n_vertices(self) -> int:
        return 1 << self.log2_n

    @property
    def n_pairs(self) -> int:
        return int(round(self.n_vertices * self.mean_degree / 2.0))


def chunglu(log2_n: int, seed: int | None = None, **kw) -> ChungLuSpec:
    return ChungLuSpec(log2_n=log2_n, seed=(0xC4C10000 + log2_n) if seed is None else seed, **kw)


def chunglu_cdf(spec: ChungLuSpec) -> np.ndarray:
    """Inclusive cumulative integer weight table (uint64) for gen_cdf_pick.

    i0 is solved by bisection on the integral approximation of the mean
    weight; the weights are then rescaled so their mean is exactly
    mean_degree, and quantised to integers with 20 fractional bits."""
    n = spec.n_vertices
    e = 1.0 / (spec.gamma - 1.0)
    wmax = min(spec.max_weight, float(n))

    def mean_of(i0: float) -> float:
        c = wmax * i0 ** e
        return c * ((n + i0) ** (1.0 - e) - i0 ** (1.0 - e)) / ((1.0 - e) * n)

    lo, hi = 1e-12, 1e15
    for _ in range(400):
        mid = math.sqrt(lo * hi)
        if mean_of(mid) < spec.mean_degree:
            lo = mid
        else:
            hi = mid
    i0 = math.sqrt(lo * hi)
    idx = np.arange(n, dtype=np.float64)
    w = wmax * (i0 / (idx + i0)) ** e
    w *= spec.mean_degree * n / float(w.sum())
    wi = np.floor(w * float(1 << 20)).astype(np.uint64)
    wi[wi == 0] = 1
    return np.cumsum(wi, dtype=np.uint64)


def chunglu_pairs(spec: ChungLuSpec, cdf: np.ndarray | None = None, k0: int = 0, count: int | None = None,
                  plain_search: bool = False):
    lib = _load()
    if cdf is None:
        cdf = chunglu_cdf(spec)
    cdf = np.ascontiguousarray(cdf, dtype=np.uint64)
    if count is None:
        count = spec.n_pairs - k0
    src = np.empty(count, dtype=np.int32)
    dst = np.empty(count, dtype=np.int32)
    lib.gen_c_chunglu_pairs(cdf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), spec.n_vertices,
                            spec.seed, k0, count, _i32p(src), _i32p(dst), 1 if plain_search else 0)
    return src, dst


# --------------------------------------------------------------------------- roots
def sample_roots(seed: int, n_vertices: int, count: int, has_edge) -> np.ndarray:
    """`count` distinct roots drawn uniformly from vertices with degree >= 1.

    Candidate j is mix64(mix64(seed) ^ j) mod n; a candidate is kept if
    has_edge[candidate] is true and it was not drawn before. `has_edge` is any
    indexable of booleans (a numpy array of degrees > 0, for instance)."""
    key = mix64(seed & MASK64)
    out: list[int] = []
    seen: set[int] = set()
    j = 0
    limit = 64 * n_vertices + 1024
    while len(out) < count and j < limit:
        cand = mix64(key ^ j) % n_vertices
        j += 1
        if cand in seen or not bool(has_edge[cand]):
            continue
        seen.add(cand)
        out.append(cand)
    if len(out) < count:
        raise ValueError("graph has fewer than %d vertices with an edge" % count)
    return np.asarray(out, dtype=np.int32)


__all__ = [
    "RmatSpec", "ChungLuSpec", "rmat", "chunglu", "rmat_pairs", "chunglu_pairs", "chunglu_cdf",
    "rmat_thresholds", "rmat_seed", "root_seed", "sample_roots", "mix64", "perm", "build",
]

if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
