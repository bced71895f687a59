"""GPU parity at the full sizes of the benchmark workloads.

- R-MAT scale 22 (int64 offsets, renumbered), 64 seeded roots: levels
  bit-exact with the oracle's serial BFS on its own CSR, parents valid,
  canonical parents bit-exact.
- R-MAT scale 24, the bench's 1024-root batch (eight 128-lane groups):
  every 16th row bit-exact with the oracle, another 64 rows through the
  streaming checker, every row equal to the single-source run of its root.
- Serving: the bench's five resident graphs (R-MAT scales 18-26), queries
  arriving at Poisson-spaced times: every result through the streaming
  checker, a sample bit-exact with the oracle.
- R-MAT scale 28, R-MAT scale 29 (chunked build) and Chung-Lu 2^26: the
  oracle cannot hold a CSR within the test's time, so the GPU results are
  checked by the streaming invariant
  checker over the regenerated (R-MAT) or host-generated (Chung-Lu) pairs.
  The invariants characterise BFS levels exactly (level = distance), and the
  checker computes the canonical parent by its definition, compared
  bit-exact. Roots here are endpoints of seeded pairs of the input stream
  (degree >= 1 by construction, degree-biased), so no root comes from the
  CUDA path.
"""
import os
import time

import numpy as np
import pytest

import dobfs_inputs as inputs
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def d():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_04359_b300 import build, dobfs
    build.build()
    dobfs.load()
    dobfs.use_torch_allocator()
    return dobfs


def _gpu_runs(d, g, roots, flags=0):
    n = g.n
    lv = np.empty((len(roots), n), dtype=np.int32)
    pa = np.empty((len(roots), n), dtype=np.int32)
    l_dev = torch.empty(n, dtype=torch.int32, device="cuda")
    p_dev = torch.empty(n, dtype=torch.int32, device="cuda")
    for i, r in enumerate(roots):
        g.run(int(r), l_dev, p_dev, d.make_opts(flags=flags))
        torch.cuda.synchronize()
        lv[i] = l_dev.cpu().numpy()
        pa[i] = p_dev.cpu().numpy()
    return lv, pa


def _pair_roots(src, dst, seed, count):
    """Endpoints of seeded pairs that are not self-loops."""
    out, j = [], 0
    while len(out) < count:
        k = inputs.mix64(inputs.mix64(seed) ^ j) % len(src)
        j += 1
        if src[k] != dst[k] and int(src[k]) not in out:
            out.append(int(src[k]))
    return np.asarray(out, dtype=np.int32)


def test_config2_rmat22_64_roots(d):
    spec = inputs.rmat(22)
    og = oracle.csr_from_rmat_par(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 64, og.degrees() > 0)
    ref_l, ref_p = oracle.bfs_many(og, roots)
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX | d.DOBFS_GRAPH_OFFSETS64)
    assert g.info.offsets_int64 == 1 and g.info.n_entries == og.nnz
    lv, pa = _gpu_runs(d, g, roots)
    np.testing.assert_array_equal(lv, ref_l)
    for i in range(0, 64, 8):
        rule, bad = oracle.check_bfs(og, int(roots[i]), lv[i], pa[i])
        assert rule == 0, (i, oracle.RULES[rule], bad)
    lv_c, pa_c = _gpu_runs(d, g, roots[:8], flags=d.DOBFS_RUN_CANONICAL_PARENT)
    np.testing.assert_array_equal(lv_c, ref_l[:8])
    np.testing.assert_array_equal(pa_c, ref_p[:8])


def _gpu_runs_vm(d, g, roots, flags=0):
    """Levels and parents of every root, vertex-major on the host ([n, R]:
    a vertex's entries for all roots side by side, the layout in which the
    streaming checker reads many roots fastest); transposed on the device."""
    n, R = g.n, len(roots)
    lv = torch.empty((R, n), dtype=torch.int32, device="cuda")
    pa = torch.empty((R, n), dtype=torch.int32, device="cuda")
    for i, r in enumerate(roots):
        g.run(int(r), lv[i], pa[i], d.make_opts(flags=flags))
    torch.cuda.synchronize()
    out = lv.t().contiguous().cpu().numpy(), pa.t().contiguous().cpu().numpy()
    del lv, pa
    torch.cuda.empty_cache()
    return out


def test_config3a_rmat28_streaming_check(d):
    """Scale 28: 20 roots in one pass of the streaming checker, 16 with the
    default parents and 4 with canonical parents, compared bit-exact with
    the checker's canonical parents."""
    spec = inputs.rmat(28)
    src, dst = inputs.rmat_pairs(spec, count=1 << 20)
    roots = _pair_roots(src, dst, inputs.root_seed(spec.seed), 20)
    del src, dst
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    n = g.n
    lv = torch.empty((20, n), dtype=torch.int32, device="cuda")
    pa = torch.empty((20, n), dtype=torch.int32, device="cuda")
    for i, r in enumerate(roots):
        g.run(int(r), lv[i], pa[i], d.make_opts(flags=d.DOBFS_RUN_CANONICAL_PARENT if i >= 16 else 0))
    torch.cuda.synchronize()
    g.close()
    levels, parents = lv.t().contiguous().cpu().numpy(), pa.t().contiguous().cpu().numpy()
    del lv, pa
    torch.cuda.empty_cache()
    t0 = time.time()
    rc, bad, canon = oracle.check_bfs_rmat_stream_multi(spec, roots, levels, parents, want_canon=True,
                                                        vertex_major=True)
    print("scale 28: 20 roots checked in %.0f s" % (time.time() - t0), flush=True)
    assert rc.tolist() == [0] * 20, [(oracle.RULES[int(r)], int(b)) for r, b in zip(rc, bad)]
    np.testing.assert_array_equal(parents[:, 16:], canon[:, 16:])
    assert all(int((levels[:, i] >= 0).sum()) > 1000 for i in range(20))


@pytest.mark.skipif(os.environ.get("DOBFS_FULL_VALIDATION", "0") in ("", "0"),
                    reason="set DOBFS_FULL_VALIDATION=1 (64 roots at scale 28: about 45 GB of host memory, minutes)")
def test_rmat28_all_64_roots_validated(d):
    """Graph500-style validation of every one of 64 roots at scale 28: levels
    and parents of each run pass the streaming invariant checker (level =
    distance, every parent a neighbour one level up), in four batches of 16
    roots per pass over the regenerated pairs."""
    spec = inputs.rmat(28)
    src, dst = inputs.rmat_pairs(spec, count=1 << 20)
    roots = _pair_roots(src, dst, inputs.root_seed(spec.seed), 64)
    del src, dst
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    for b in range(4):
        batch = roots[16 * b:16 * (b + 1)]
        lv, pa = _gpu_runs_vm(d, g, batch)
        t0 = time.time()
        rc, bad, _ = oracle.check_bfs_rmat_stream_multi(spec, batch, lv, pa, vertex_major=True)
        reached = [int((lv[:, i] >= 0).sum()) for i in range(len(batch))]
        print("batch %d: roots %s, reached min %d max %d, depth max %d, checked in %.0f s" %
              (b, batch.tolist(), min(reached), max(reached), int(lv.max()), time.time() - t0), flush=True)
        assert rc.tolist() == [0] * len(batch), [(oracle.RULES[int(r)], int(x)) for r, x in zip(rc, bad)]
        assert min(reached) > 1000
        del lv, pa
    g.close()


def test_rmat29_chunked_build_streaming_check(d):
    """Scale 29 (17 G stored entries): too large for the one-shot build's key
    buffers, so the graph is built in chunks of source rows; one root with
    any parents, one with canonical parents, checked over the regenerated
    pair stream."""
    spec = inputs.rmat(29)
    src, dst = inputs.rmat_pairs(spec, count=1 << 20)
    roots = _pair_roots(src, dst, inputs.root_seed(spec.seed), 2)
    del src, dst
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    assert g.info.offsets_int64 == 1 and g.info.n_entries > (1 << 33)
    lv, pa = _gpu_runs_vm(d, g, roots[:1])
    lv_c, pa_c = _gpu_runs_vm(d, g, roots[1:], flags=d.DOBFS_RUN_CANONICAL_PARENT)
    g.close()
    torch.cuda.empty_cache()
    levels = np.ascontiguousarray(np.concatenate([lv, lv_c], axis=1))
    parents = np.ascontiguousarray(np.concatenate([pa, pa_c], axis=1))
    del lv, pa, lv_c, pa_c
    rc, bad, canon = oracle.check_bfs_rmat_stream_multi(spec, roots, levels, parents, want_canon=True,
                                                        vertex_major=True)
    assert rc.tolist() == [0, 0], [(oracle.RULES[int(r)], int(b)) for r, b in zip(rc, bad)]
    np.testing.assert_array_equal(parents[:, 1:], canon[:, 1:])
    assert all(int((levels[:, i] >= 0).sum()) > 1000 for i in range(2))


def test_config3b_chunglu26_streaming_check(d):
    spec = inputs.chunglu(26)
    cdf = inputs.chunglu_cdf(spec)
    g = d.chunglu_graph(spec, cdf)
    src, dst = inputs.chunglu_pairs(spec, cdf)
    roots = _pair_roots(src, dst, spec.seed ^ 0xB00F, 4)
    lv, pa = _gpu_runs(d, g, roots[:2])
    lv_c, pa_c = _gpu_runs(d, g, roots[2:], flags=d.DOBFS_RUN_CANONICAL_PARENT)
    g.close()
    levels = np.concatenate([lv, lv_c])
    parents = np.concatenate([pa, pa_c])
    rc, bad, canon, _ = oracle.check_bfs_pairs_multi(spec.n_vertices, src, dst, roots, levels, parents,
                                                     want_canon=True)
    assert rc.tolist() == [0, 0, 0, 0], [(oracle.RULES[int(r)], int(b)) for r, b in zip(rc, bad)]
    np.testing.assert_array_equal(parents[2:], canon[2:])
    assert all(int((levels[i] >= 0).sum()) > 1000 for i in range(4))


def test_config2_rmat22_batched_256_roots(d):
    """Batched BFS at scale 22 in 128-lane groups (256 roots = two full
    groups): every 16th row bit-exact with the oracle's serial BFS, the rest
    through the streaming invariant checker."""
    spec = inputs.rmat(22)
    og = oracle.csr_from_rmat_par(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0x256, og.n, 256, og.degrees() > 0)
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    out = torch.empty((256, og.n), dtype=torch.int32, device="cuda")
    d.dobfs_run_batch(g.handle, torch.from_numpy(np.ascontiguousarray(roots)).cuda(), out)
    lv = out[::16].cpu().numpy()
    lv_vm = out.t().contiguous().cpu().numpy()  # vertex-major for the streaming check
    del out
    g.close()
    ref, _ = oracle.bfs_many(og, roots[::16], want_parent=False)
    np.testing.assert_array_equal(lv, ref)
    rc, bad, _ = oracle.check_bfs_rmat_stream_multi(spec, roots, lv_vm, vertex_major=True)
    assert rc.tolist() == [0] * 256, [(i, oracle.RULES[int(r)], int(x)) for i, (r, x) in enumerate(zip(rc, bad)) if r]


def test_config5_served_mix_rmat18_20(d):
    """The server with its default options (128-lane groups, one group per
    graph) on R-MAT scale 18 and 20 graphs, 150 queries per graph submitted at
    once: every 10th result bit-exact with the oracle, every result through
    the streaming invariant checker."""
    specs = [inputs.rmat(18), inputs.rmat(20)]
    graphs = [d.rmat_graph(s, flags=d.DOBFS_GRAPH_REINDEX) for s in specs]
    srv = d.dobfs_serve_create()
    try:
        gids = [d.dobfs_serve_add_graph(srv, g.handle) for g in graphs]
        outs, tickets, roots = {}, {}, {}
        ogs = [oracle.csr_from_rmat_par(s) for s in specs]
        for gi, og in enumerate(ogs):
            roots[gi] = inputs.sample_roots(inputs.root_seed(specs[gi].seed) ^ 0x5E7E, og.n, 150, og.degrees() > 0)
        for k in range(150):
            for gi, g in enumerate(graphs):
                out = torch.full((g.n,), 9, dtype=torch.int32, device="cuda")
                outs[(gi, k)] = out
                tickets[(gi, k)] = d.dobfs_serve_submit(srv, gids[gi], int(roots[gi][k]), out)
        t0 = time.time()
        for key, t in tickets.items():
            while d.dobfs_serve_poll(srv, t) is None:
                assert time.time() - t0 < 300, "queries did not finish"
                time.sleep(0.001)
        for gi, spec in enumerate(specs):
            lv = np.stack([outs[(gi, k)].cpu().numpy() for k in range(150)])
            ref, _ = oracle.bfs_many(ogs[gi], roots[gi][::10], want_parent=False)
            np.testing.assert_array_equal(lv[::10], ref)
            rc, bad, _ = oracle.check_bfs_rmat_stream_multi(spec, roots[gi], lv)
            assert rc.tolist() == [0] * 150, [(oracle.RULES[int(r)], int(x)) for r, x in zip(rc, bad)]
    finally:
        d.dobfs_serve_destroy(srv)
        for g in graphs:
            g.close()


@pytest.fixture(scope="module")
def s24():
    """The oracle's CSR of R-MAT scale 24 (threaded build), shared by the
    batched and served tests."""
    spec = inputs.rmat(24)
    return spec, oracle.csr_from_rmat_par(spec)


def test_config4_rmat24_batch_1024_roots(d, s24):
    """The bench's largest batch: R-MAT scale 24, the bench's 1024 seeded
    roots in eight 128-lane groups. Every 16th row is bit-exact with the
    oracle's serial BFS, the rows in between at offset 8 pass the streaming
    checker, and every row equals the single-source run of its root (itself
    bit-exact with the oracle wherever it is tested)."""
    spec, og = s24
    n = og.n
    roots = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0xBA7C, n, 1024, og.degrees() > 0)
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    out = torch.full((1024, n), 7, dtype=torch.int32, device="cuda")
    d.dobfs_run_batch(g.handle, torch.from_numpy(np.ascontiguousarray(roots)).cuda(), out)
    torch.cuda.synchronize()
    one = torch.empty(n, dtype=torch.int32, device="cuda")
    differ = []
    for i in range(1024):
        g.run(int(roots[i]), one)
        if not torch.equal(out[i], one):
            differ.append(i)
    assert not differ, "batch rows differ from single-source runs: %s" % differ[:10]
    lv = out[::16].cpu().numpy()
    lv_vm = out[8::16].t().contiguous().cpu().numpy()
    del out, one
    g.close()
    torch.cuda.empty_cache()
    ref, _ = oracle.bfs_many(og, roots[::16], want_parent=False)
    np.testing.assert_array_equal(lv, ref)
    rc, bad, _ = oracle.check_bfs_rmat_stream_multi(spec, roots[8::16], lv_vm, vertex_major=True)
    assert rc.tolist() == [0] * 64, [(i, oracle.RULES[int(r)], int(x)) for i, (r, x) in enumerate(zip(rc, bad)) if r]


def test_config5_served_five_graphs_poisson(d, s24):
    """The bench's serving workload: R-MAT scales 18, 20, 22, 24 and 26
    resident (default server options), 200 queries with graph ids uniform and
    roots from each graph's seeded pool, submitted at Poisson-spaced times
    (20,000 queries/s offered). Every result passes the streaming checker of
    its graph; the first 4 of every graph but the largest are bit-exact with
    the oracle's serial BFS."""
    scales = (18, 20, 22, 24, 26)
    specs = [inputs.rmat(sc) for sc in scales]
    graphs = [d.rmat_graph(sp, flags=d.DOBFS_GRAPH_REINDEX) for sp in specs]
    rng = np.random.default_rng(0xC0F5)
    n_q = 200
    gaps = rng.exponential(1.0 / 20000, n_q)
    which = rng.integers(0, len(scales), n_q)
    ridx = rng.integers(0, 1024, n_q)
    pools = []
    for sp, g in zip(specs, graphs):
        # the same pool the bench draws from: degree >= 1 vertices, seeded (degrees from the oracle's
        # CSR where it is built anyway, else the generator's pairs)
        if sp.scale == 24:
            has_edge = s24[1].degrees() > 0
        else:
            src, dst = inputs.rmat_pairs(sp)
            has_edge = np.zeros(sp.n_vertices, dtype=bool)
            keep = src != dst
            has_edge[src[keep]] = True
            has_edge[dst[keep]] = True
            del src, dst, keep
        pools.append(inputs.sample_roots(inputs.root_seed(sp.seed) ^ 0x5E7E, sp.n_vertices, 1024, has_edge))
    srv = d.dobfs_serve_create()
    outs, tickets = [], []
    try:
        gids = [d.dobfs_serve_add_graph(srv, g.handle) for g in graphs]
        t_start = time.perf_counter()
        due = np.cumsum(gaps)
        for i in range(n_q):
            while time.perf_counter() - t_start < due[i]:
                pass
            gi = int(which[i])
            out = torch.full((graphs[gi].n,), 9, dtype=torch.int32, device="cuda")
            outs.append(out)
            tickets.append(d.dobfs_serve_submit(srv, gids[gi], int(pools[gi][ridx[i]]), out))
        t0 = time.time()
        for t in tickets:
            while d.dobfs_serve_poll(srv, t) is None:
                assert time.time() - t0 < 300, "queries did not finish"
                time.sleep(0.0005)
    finally:
        d.dobfs_serve_destroy(srv)
        for g in graphs:
            g.close()
    for gi, sp in enumerate(specs):
        idx = [i for i in range(n_q) if which[i] == gi]
        roots = np.asarray([pools[gi][ridx[i]] for i in idx], dtype=np.int32)
        lv_vm = torch.stack([outs[i] for i in idx], dim=1).cpu().numpy()
        rc, bad, _ = oracle.check_bfs_rmat_stream_multi(sp, roots, lv_vm, vertex_major=True)
        assert rc.tolist() == [0] * len(idx), (sp.scale, [(int(r), int(x)) for r, x in zip(rc, bad) if r])
        if sp.scale <= 24:
            og = s24[1] if sp.scale == 24 else oracle.csr_from_rmat_par(sp)
            ref, _ = oracle.bfs_many(og, roots[:4], want_parent=False)
            np.testing.assert_array_equal(lv_vm[:, :4].T, ref)
        for i in idx:
            outs[i] = None
        torch.cuda.empty_cache()
