"""Autotuner for the direction-switch policy and the top-down variants.

The run options that decide how a BFS proceeds change only its speed, never
its result (levels are unique; parents stay valid), so they can be tuned per
graph by timing the library on a sample of roots. Two policies are tuned
and the faster one is kept:

  alpha/beta  the rule of the direction-optimizing BFS the paper builds on:
              top-down -> bottom-up when m_f * alpha > m_u, back when
              n_f * beta < n (knobs: alpha, beta, td_bitmap_div, td_split_pct);
  static      the paper's own policy (Sec. 3.3): bottom-up once the next
              frontier, estimated as static_pct percent of the frontier's
              out-edges, exceeds n / beta, then bu_steps bottom-up levels
              (knobs: static_pct, bu_steps, td_bitmap_div, td_split_pct).

Both also tune the degree-bin cutoffs of the step kernels (td_small_max,
td_chunk, bu_scan) and the threads per block of the bottom-up, top-down and
output kernels (bu_threads, td_threads, out_threads); batched runs tune
alpha, beta, td_chunk, bu_scan, bu_threads and td_threads.
The search is coordinate descent over small grids (each knob in turn, the
best value kept, until a sweep changes nothing). A result can be cached in a
JSON file under a key describing the graph.

    from paper_1503_04359_b300 import autotune
    opts, record = autotune.tune(g, sample_roots)          # dobfs_run_opts
    bopts, brecord = autotune.tune_batch(g, sample_roots)  # for dobfs_run_batch
"""
from __future__ import annotations

import json
import os
from typing import Callable

import numpy as np

from . import dobfs

# degree-bin cutoffs (thread-per-row limit, chunk-record length, bottom-up
# scan depth before a row goes warp-wide), tuned after the policy knobs
CUTOFF_GRID = {
    "td_small_max": [8, 16, 32, 64],
    "td_chunk": [256, 512, 1024, 2048],
    "bu_scan": [8, 16, 32, 64],
    # threads per block of the bottom-up, top-down and output kernels
    "bu_threads": [128, 256, 512],
    "td_threads": [128, 256, 512],
    "out_threads": [128, 256, 512],
}
CUTOFF_DEFAULTS = {"td_small_max": 16, "td_chunk": 512, "bu_scan": 32, "bu_threads": 256, "td_threads": 256,
                   "out_threads": 256}
ALPHA_BETA_GRID = {
    "alpha": [4, 8, 14, 24, 48],
    "beta": [8, 16, 24, 48, 96],
    "td_bitmap_div": [0, 1, 2, 4, 16],
    "td_split_pct": [0, 75, 150, 300, 600],
    **CUTOFF_GRID,
}
STATIC_GRID = {
    "static_pct": [2, 5, 10, 20, 40],
    "bu_steps": [1, 2, 3, 4, 6],
    "td_bitmap_div": [0, 1, 2, 4, 16],
    "td_split_pct": [0, 75, 150, 300, 600],
    **CUTOFF_GRID,
}
BATCH_GRID = {"alpha": [2, 4, 8, 14, 32], "beta": [8, 24, 64], "td_chunk": [256, 512, 1024, 2048, 4096],
              "bu_scan": [8, 16, 32, 64, 128], "bu_threads": [128, 256, 512], "td_threads": [128, 256, 512]}
BATCH_DEFAULTS = {"td_chunk": 1024, "bu_scan": 32, "bu_threads": 256, "td_threads": 256}


def graph_key(g: dobfs.Graph, kind: str) -> str:
    i = g.info
    return "%s:n=%d:nnz=%d:nonisolated=%d:maxdeg=%d:reindexed=%d:off64=%d" % (
        kind, i.n_vertices, i.n_entries, i.n_nonisolated, i.max_degree, i.reindexed, i.offsets_int64)


def load_cache(path: str | None) -> dict:
    if not path:
        return {}
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, key: str, record: dict) -> None:
    cache = load_cache(path)
    cache[key] = record
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def descend(grid: dict, measure: Callable[[dict], float], start: dict, max_sweeps: int = 3,
            min_gain: float = 0.01) -> tuple[dict, float, list]:
    """Coordinate descent: for each knob in turn try every grid value with the
    others fixed, keep a value only if it is faster by more than `min_gain`
    (relative); stop after a sweep with no change. Returns (best, best_ms, log)."""
    best = dict(start)
    best_ms = measure(best)
    log = [(dict(best), best_ms)]
    seen = {tuple(sorted(best.items())): best_ms}
    for _ in range(max_sweeps):
        changed = False
        for k, values in grid.items():
            for v in values:
                if v == best[k]:
                    continue
                cand = dict(best)
                cand[k] = v
                key = tuple(sorted(cand.items()))
                if key in seen:
                    ms = seen[key]
                else:
                    ms = measure(cand)
                    seen[key] = ms
                    log.append((cand, ms))
                if ms < best_ms * (1.0 - min_gain):
                    best, best_ms, changed = cand, ms, True
        if not changed:
            break
    return best, best_ms, log


def _time_single(g, roots, params: dict, level, parent, reps: int) -> float:
    """Mean device ms per root (after one warm run)."""
    opts = dobfs.make_opts(**params)
    g.run(int(roots[0]), level, parent, opts)
    total = 0.0
    for _ in range(reps):
        for r in roots:
            total += g.run(int(r), level, parent, opts, want_stats=True).device_ms
    return total / (reps * len(roots))


def tune(g: dobfs.Graph, roots, cache_path: str | None = None, key: str | None = None,
         policies=("alpha_beta", "static"), reps: int = 1) -> tuple[dobfs.dobfs_run_opts, dict]:
    """Tunes single-source runs on `roots`; returns (options, record). The
    record holds the chosen policy and values, its mean ms per root on the
    sample, the library defaults' mean ms, and each policy's best."""
    import torch
    key = key or graph_key(g, "single")
    cached = load_cache(cache_path).get(key)
    if cached:
        return dobfs.make_opts(**cached["params"]), cached
    n = g.n
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    d = dobfs.dobfs_run_opts_init()

    def measure(p):
        return _time_single(g, roots, p, level, parent, reps)

    default = {"direction": dobfs.DOBFS_DIR_AUTO, "alpha": d.alpha, "beta": d.beta, "td_bitmap_div": d.td_bitmap_div,
               "td_split_pct": d.td_split_pct}
    default_ms = measure(default)
    per_policy = {}
    if "alpha_beta" in policies:
        grid = ALPHA_BETA_GRID
        start = dict({k: default[k] for k in ("alpha", "beta", "td_bitmap_div", "td_split_pct")}, **CUTOFF_DEFAULTS)
        b, ms, log = descend(grid, lambda p: measure(dict(p, direction=dobfs.DOBFS_DIR_AUTO)), start)
        per_policy["alpha_beta"] = (dict(b, direction=dobfs.DOBFS_DIR_AUTO), ms, len(log))
    if "static" in policies:
        grid = STATIC_GRID
        start = dict({"static_pct": d.static_pct, "bu_steps": d.bu_steps, "td_bitmap_div": d.td_bitmap_div,
                      "td_split_pct": d.td_split_pct}, **CUTOFF_DEFAULTS)
        b, ms, log = descend(grid, lambda p: measure(dict(p, direction=dobfs.DOBFS_DIR_STATIC, beta=d.beta)), start)
        per_policy["static"] = (dict(b, direction=dobfs.DOBFS_DIR_STATIC, beta=d.beta), ms, len(log))
    name = min(per_policy, key=lambda k: per_policy[k][1])
    params, ms, _ = per_policy[name]
    record = {"policy": name, "params": params, "ms": ms, "default_ms": default_ms, "roots": len(roots),
              "policies": {k: {"params": v[0], "ms": v[1], "evaluations": v[2]} for k, v in per_policy.items()}}
    del level, parent
    if cache_path:
        save_cache(cache_path, key, record)
    return dobfs.make_opts(**params), record


def tune_batch(g: dobfs.Graph, roots, cache_path: str | None = None, key: str | None = None,
               reps: int = 2) -> tuple[dobfs.dobfs_run_opts, dict]:
    """Tunes alpha, beta and the cutoffs of batched runs on one lane group (up to 64 roots)."""
    import torch
    key = key or graph_key(g, "batch")
    cached = load_cache(cache_path).get(key)
    if cached:
        return dobfs.make_opts(**cached["params"]), cached
    roots = np.ascontiguousarray(np.asarray(roots[:64], dtype=np.int32))
    rt = torch.from_numpy(roots).cuda()
    out = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")

    def measure(p):
        o = dobfs.make_opts(**p)
        dobfs.dobfs_run_batch(g.handle, rt, out, opts=o)
        return min(dobfs.dobfs_run_batch(g.handle, rt, out, opts=o, want_stats=True).device_ms for _ in range(reps))

    d = dobfs.dobfs_run_opts_init()
    start = dict({"alpha": dobfs.DOBFS_BATCH_ALPHA, "beta": d.beta}, **BATCH_DEFAULTS)
    default_ms = measure(start)
    best, ms, log = descend(BATCH_GRID, measure, start)
    record = {"policy": "alpha_beta", "params": best, "ms": ms, "default_ms": default_ms, "roots": len(roots),
              "evaluations": len(log)}
    del out
    if cache_path:
        save_cache(cache_path, key, record)
    return dobfs.make_opts(**best), record
