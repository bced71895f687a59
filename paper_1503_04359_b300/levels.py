"""Per-level profile of direction-optimized BFS on an R-MAT graph.

    python -m paper_1503_04359_b300.levels [--scale S] [--roots R] [--max-root-degree D]
                                           [--modes auto,topdown] [--no-reindex] [--json]
                                           [--alpha A] [--beta B] [--td-bitmap-div D] [--td-split-pct P]
                                           [--batch K]

For every root and direction policy it runs one BFS driven from the host
(``DOBFS_RUN_HOST_LOOP``), so each level's kernels are timed with CUDA
events, and prints one line per level: direction, frontier size n_f and edge
count m_f, vertices discovered, adjacency entries examined, vertices scanned
bottom-up, algorithmic bytes, time and GB/s. This is the per-level view of the
paper's Fig. 1 (time per level) and Fig. 4 (top-down-only against
direction-optimized, per level), on one GPU. Device-driven (graph) time of
the same root is printed beside it.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


DIRS = {0: "TD", 1: "BU", 2: "MX"}  # MX: mixed level (bottom-up for high degrees, top-down for the rest)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=28)
    ap.add_argument("--roots", type=int, default=2)
    ap.add_argument("--max-root-degree", type=int, default=0, help="keep only roots of at most this degree")
    ap.add_argument("--modes", default="auto")
    ap.add_argument("--no-reindex", action="store_true")
    ap.add_argument("--json", action="store_true")
    ap.add_argument("--batch", type=int, default=0, help="also profile one batched run of this many roots")
    ap.add_argument("--alpha", type=int, default=None, help="direction switch alpha (default: the library's)")
    ap.add_argument("--beta", type=int, default=None)
    ap.add_argument("--td-bitmap-div", type=int, default=None,
                    help="top-down steps with m_f * div >= n mark a bitmap (0: never)")
    ap.add_argument("--td-split-pct", type=int, default=None, help="mixed-level threshold (0: no mixed levels)")
    args = ap.parse_args(argv)

    import torch

    import dobfs_inputs as inputs
    from paper_1503_04359_b300 import build, dobfs

    build.build()
    dobfs.load()
    dobfs.use_torch_allocator()
    modes = {"auto": dobfs.DOBFS_DIR_AUTO, "topdown": dobfs.DOBFS_DIR_TOPDOWN, "bottomup": dobfs.DOBFS_DIR_BOTTOMUP,
             "static": dobfs.DOBFS_DIR_STATIC}
    spec = inputs.rmat(args.scale)
    g = dobfs.rmat_graph(spec, flags=0 if args.no_reindex else dobfs.DOBFS_GRAPH_REINDEX)
    n = g.n
    deg = g.degrees()
    ok = deg > 0 if args.max_root_degree <= 0 else (deg > 0) & (deg <= args.max_root_degree)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), n, args.roots, ok)
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    pa = torch.empty(n, dtype=torch.int32, device="cuda")
    out = []
    knobs = {"alpha": args.alpha, "beta": args.beta, "td_bitmap_div": args.td_bitmap_div,
             "td_split_pct": args.td_split_pct}
    for name in args.modes.split(","):
        mode = modes[name]
        for r in roots:
            g.run(int(r), lv, pa, dobfs.make_opts(direction=mode, **knobs))  # warm
            st = g.run(int(r), lv, pa, dobfs.make_opts(direction=mode, **knobs), want_stats=True)
            sh = g.run(int(r), lv, pa, dobfs.make_opts(direction=mode, flags=dobfs.DOBFS_RUN_HOST_LOOP, **knobs),
                       want_stats=True)
            rec = {"mode": name, "root": int(r), "root_degree": int(deg[r]), "graph_ms": st.device_ms,
                   "host_loop_ms": sh.device_ms, "levels": st.levels, "reached": st.reached,
                   "teps_edges": st.teps_edges, "gteps": st.teps_edges / (st.device_ms * 1e-3) / 1e9,
                   "per_level": []}
            for t in g.trace():
                rec["per_level"].append({
                    "level": t.level, "dir": DIRS.get(t.direction, "?"), "n_f": t.n_frontier,
                    "m_f": t.m_frontier, "n_next": t.n_next, "examined": t.edges_examined,
                    "scanned": t.vertices_scanned, "alg_bytes": t.alg_bytes, "ms": t.ms, "ms_main": t.ms_main,
                    "gbs": t.alg_bytes / (t.ms_main * 1e-3) / 1e9 if t.ms_main > 0 else 0.0})
            out.append(rec)
            if not args.json:
                print("%s root %d (degree %d): graph %.3f ms (%.0f GTEPS), host-driven %.3f ms, %d levels, "
                      "reached %d" % (name, r, deg[r], st.device_ms, rec["gteps"], sh.device_ms, st.levels,
                                      st.reached))
                for p in rec["per_level"]:
                    print("  L%-3d %s n_f=%-11d m_f=%-12d n_next=%-11d examined=%-11d scanned=%-11d "
                          "bytes=%-12d %.3f ms (main %.3f ms, %.0f GB/s)" % (
                              p["level"], p["dir"], p["n_f"], p["m_f"], p["n_next"], p["examined"], p["scanned"],
                              p["alg_bytes"], p["ms"], p["ms_main"], p["gbs"]))
    if args.batch > 0:
        broots = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0xBA7C, n, args.batch, deg > 0)
        bout = torch.empty((args.batch, n), dtype=torch.int32, device="cuda")
        rt = torch.from_numpy(np.ascontiguousarray(broots)).cuda()
        for name in args.modes.split(","):
            o = dobfs.make_opts(direction=modes[name], **knobs)
            st = dobfs.dobfs_run_batch(g.handle, rt, bout, opts=o, want_stats=True)
            o.flags = dobfs.DOBFS_RUN_HOST_LOOP
            sh = dobfs.dobfs_run_batch(g.handle, rt, bout, opts=o, want_stats=True)
            tr = g.trace()
            rec = {"mode": name, "batch": args.batch, "graph_ms": st.device_ms, "host_loop_ms": sh.device_ms,
                   "levels": st.levels, "per_level": [
                       {"level": t.level, "dir": DIRS.get(t.direction, "?"), "n_f": t.n_frontier,
                        "m_f": t.m_frontier, "examined": t.edges_examined, "ms": t.ms} for t in tr]}
            out.append(rec)
            if not args.json:
                print("batch %s, %d roots: graph %.3f ms (%.0f roots/s), host-driven %.3f ms, %d levels (first group)"
                      % (name, args.batch, st.device_ms, args.batch / (st.device_ms * 1e-3), sh.device_ms, st.levels))
                for p in rec["per_level"]:
                    print("  L%-3d %s n_f=%-11d m_f=%-12d examined=%-12d %.3f ms" % (
                        p["level"], p["dir"], p["n_f"], p["m_f"], p["examined"], p["ms"]))
    if args.json:
        print(json.dumps(out))
    torch.cuda.synchronize()
    g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
