"""Runs in a child process with DOBFS_BOUNDS_CHECK=1 (the bounds-check build
libdobfs_bc.so); started by test_gpu_bounds_check.py.

1. On valid graphs no check fires: single-source runs in every direction
   policy, canonical parents, batches and served queries all return the
   oracle's results.
2. A graph corrupted on purpose (a stored column set to n + 3, inside the
   allocation slack of this build) makes each path fail with
   DOBFS_ERR_BOUNDS instead of reading out of bounds, and the library stays
   usable afterwards; the same for a caller's CSR given to dobfs_run_static.
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import dobfs_inputs as inputs  # noqa: E402
import oracle  # noqa: E402
from paper_1503_04359_b300 import dobfs as d  # noqa: E402


def levels(g, r, **kw):
    lv = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    pa = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    g.run(int(r), lv, pa, d.make_opts(**kw))
    torch.cuda.synchronize()
    return lv.cpu().numpy(), pa.cpu().numpy()


def serve_one(g, r):
    srv = d.dobfs_serve_create()
    try:
        gid = d.dobfs_serve_add_graph(srv, g.handle)
        out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        t = d.dobfs_serve_submit(srv, gid, int(r), out)
        t0 = time.time()
        while True:
            res = d.dobfs_serve_poll(srv, t)
            if res is not None:
                return res.status, out.cpu().numpy()
            assert time.time() - t0 < 60, "query did not finish"
            time.sleep(0.001)
    finally:
        d.dobfs_serve_destroy(srv)


def expect_bounds(fn, what):
    try:
        fn()
    except d.DobfsError as e:
        assert e.status == d.DOBFS_ERR_BOUNDS, (what, e)
        print("%s: %s" % (what, e), flush=True)
        return
    raise AssertionError("%s: no bounds failure reported" % what)


def clean_runs():
    for flags, spec in ((d.DOBFS_GRAPH_REINDEX, inputs.rmat(12)), (0, inputs.rmat(11)),
                        (d.DOBFS_GRAPH_REINDEX | d.DOBFS_GRAPH_OFFSETS64, inputs.rmat(10))):
        og = oracle.csr_from_rmat(spec)
        roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 70, og.degrees() > 0)
        ref_l, ref_p = oracle.bfs_many(og, roots)
        g = d.rmat_graph(spec, flags=flags)
        for i, r in enumerate(roots[:4]):
            for mode in (0, 1, 2):
                lv, _ = levels(g, r, direction=mode)
                np.testing.assert_array_equal(lv, ref_l[i])
            lv, pa = levels(g, r, flags=d.DOBFS_RUN_CANONICAL_PARENT)
            np.testing.assert_array_equal(pa, ref_p[i])
            lv, _ = levels(g, r, td_split_pct=100000)  # mixed levels, all vertices bottom-up
            np.testing.assert_array_equal(lv, ref_l[i])
        out = torch.full((len(roots), og.n), 7, dtype=torch.int32, device="cuda")
        d.dobfs_run_batch(g.handle, torch.from_numpy(np.ascontiguousarray(roots)).cuda(), out)
        np.testing.assert_array_equal(out.cpu().numpy(), ref_l)
        st, lv = serve_one(g, roots[5])
        assert st == 0
        np.testing.assert_array_equal(lv, ref_l[5])
        g.close()
    print("clean runs: no check fired", flush=True)


def corrupted_runs():
    spec = inputs.rmat(10)
    og = oracle.csr_from_rmat(spec)
    deg = og.degrees()
    root = int(inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 1, deg > 0)[0])
    bad = og.n + 3

    def fresh():
        # no renumbering: internal IDs are original IDs, so rows are the oracle's
        return d.rmat_graph(spec, flags=0)

    # top-down: the root's own row is read in full at level 0
    g = fresh()
    d.dobfs_debug_set_column(g.handle, int(og.off[root]) + int(deg[root]) - 1, bad)
    expect_bounds(lambda: levels(g, root, direction=d.DOBFS_DIR_TOPDOWN), "top-down")
    g.close()
    # a neighbour w of the root: its first entry is tested by the bottom-up
    # step at level 0 and its row read by any top-down step at level 1
    w = int(og.cols[og.off[root]])
    g = fresh()
    d.dobfs_debug_set_column(g.handle, int(og.off[w]), bad)
    expect_bounds(lambda: levels(g, root, direction=d.DOBFS_DIR_BOTTOMUP), "bottom-up")
    expect_bounds(lambda: d.dobfs_run_batch(g.handle, torch.tensor([root], dtype=torch.int32, device="cuda"),
                                            torch.empty((1, og.n), dtype=torch.int32, device="cuda")), "batch")
    expect_bounds(lambda: serve_one(g, root), "serve")
    # values the debug call refuses
    for v in (-1, og.n + 1024):
        try:
            d.dobfs_debug_set_column(g.handle, 0, v)
            raise AssertionError("value %d accepted" % v)
        except d.DobfsError as e:
            assert e.status == d.DOBFS_ERR_INVALID
    g.close()
    # the library is usable afterwards
    g = fresh()
    lv, _ = levels(g, root)
    np.testing.assert_array_equal(lv, oracle.bfs(og, root)[0])
    g.close()
    static_corrupted(spec, og, root)
    print("corrupted runs: every path reported DOBFS_ERR_BOUNDS", flush=True)


def static_corrupted(spec, og, root):
    """dobfs_run_static on a caller CSR with one column set to n + 3: the
    root's last entry (read by the top-down step of level 0), then the first
    entry of a neighbour (read at level 1 in either direction). The output
    buffers have 1024 entries of slack past n, so even a missed check would
    stay inside them."""
    n = og.n
    off = torch.from_numpy(og.off.astype(np.int32)).cuda()
    lv = torch.full((n + 1024,), 7, dtype=torch.int32, device="cuda")
    pa = torch.full((n + 1024,), 7, dtype=torch.int32, device="cuda")
    w = int(og.cols[og.off[root]])
    for pos, what in ((int(og.off[root + 1]) - 1, "static top-down"), (int(og.off[w]), "static level 1")):
        cols = og.cols.copy()
        cols[pos] = n + 3
        cd = torch.from_numpy(cols).cuda()
        expect_bounds(lambda: (d.dobfs_run_static(off, cd, n, root, lv, pa), torch.cuda.synchronize()), what)
    cd = torch.from_numpy(og.cols).cuda()
    d.dobfs_run_static(off, cd, n, root, lv, pa)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lv[:n].cpu().numpy(), oracle.bfs(og, root)[0])


def main():
    assert d.LIB_PATH.endswith("libdobfs_bc.so"), d.LIB_PATH
    d.load()
    d.use_torch_allocator()
    clean_runs()
    corrupted_runs()
    print("OK", flush=True)


if __name__ == "__main__":
    main()
