"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Levels must match the oracle bit-exact in every direction policy (levels are
unique, so any top-down / bottom-up schedule of Algorithm 1 reaches the same
array); default parents must satisfy the BFS invariants; canonical parents
must match bit-exact.
"""
import numpy as np
import pytest

import dobfs_inputs as inputs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def d():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_04359_b300 import build, dobfs
    build.build()
    dobfs.load()
    dobfs.use_torch_allocator()
    return dobfs


MODES = [("auto", 0, 0), ("topdown", 1, 0), ("bottomup", 2, 0), ("random1", 3, 1), ("random2", 3, 2),
         ("random3", 3, 77), ("static", 4, 0)]


def _run(d, g, root, mode=0, seed=0, flags=0, host=False, **kw):
    n = g.n
    if host:
        lv = np.empty(n, dtype=np.int32)
        pa = np.empty(n, dtype=np.int32)
    else:
        lv = torch.empty(n, dtype=torch.int32, device="cuda")
        pa = torch.empty(n, dtype=torch.int32, device="cuda")
    st = g.run(root, lv, pa, d.make_opts(direction=mode, schedule_seed=seed, flags=flags, **kw), want_stats=True)
    torch.cuda.synchronize()
    if not host:
        lv, pa = lv.cpu().numpy(), pa.cpu().numpy()
    return lv, pa, st


def _check_run(og, root, lv, pa, ref_level, ref_parent=None):
    np.testing.assert_array_equal(lv, ref_level)
    rule, bad = oracle.check_bfs(og, root, lv, pa)
    assert rule == 0, (oracle.RULES[rule], bad)
    if ref_parent is not None:
        np.testing.assert_array_equal(pa, ref_parent)


# ------------------------------------------------------------------ CSR build
@pytest.mark.parametrize("scale", [6, 11, 16])
def test_csr_build_matches_oracle_no_reindex(d, scale):
    spec = inputs.rmat(scale)
    og = oracle.csr_from_rmat(spec)
    g = d.rmat_graph(spec, flags=0)
    off, cols, n2o = g.export()
    np.testing.assert_array_equal(off, og.off)
    np.testing.assert_array_equal(cols, og.cols)
    np.testing.assert_array_equal(n2o, np.arange(spec.n_vertices, dtype=np.int32))
    info = g.info
    deg = og.degrees()
    assert info.n_entries == og.nnz and info.reindexed == 0
    assert info.n_nonisolated == int((deg > 0).sum()) and info.max_degree == int(deg.max())
    np.testing.assert_array_equal(g.degrees(), deg)


def _degree_class(deg, exact):
    """Renumbering class, written out from the definition in include/dobfs.h."""
    if exact:
        return deg.astype(np.int64)
    out = np.empty(len(deg), dtype=np.int64)
    for i, d in enumerate(deg.tolist()):
        if d >= 4096:
            out[i] = 64 + d
        elif d < 8:
            out[i] = d
        else:
            e = d.bit_length() - 1
            out[i] = 8 + 4 * (e - 3) + ((d >> (e - 2)) & 3)
    return out


@pytest.mark.parametrize("scale,flags,exact", [(11, 0x20, True), (14, 0x10 | 0x20, True), (11, 0x2, False),
                                               (14, 0x10 | 0x2, False)])
def test_csr_build_reindex(d, scale, flags, exact):
    spec = inputs.rmat(scale)
    og = oracle.csr_from_rmat(spec)
    g = d.rmat_graph(spec, flags=flags)
    off, cols, n2o = g.export()
    deg = og.degrees()
    cls = _degree_class(deg, exact)
    ids = np.arange(og.n)
    # new ID = rank by (degree class descending, original ID ascending)
    np.testing.assert_array_equal(n2o, np.lexsort((ids, -cls)).astype(np.int32))
    for i in range(og.n):
        row = cols[off[i]:off[i + 1]]
        assert np.all(np.diff(row) > 0)                         # sorted by new ID
        np.testing.assert_array_equal(np.sort(n2o[row]), og.row(int(n2o[i])))
        if len(row) > 1:                                        # highest-class neighbour first
            assert np.all(np.diff(cls[n2o[row]]) <= 0)
    assert g.info.offsets_int64 == (1 if flags & 0x10 else 0)
    np.testing.assert_array_equal(g.degrees(), deg)
    assert g.info.reindexed == 1


@pytest.mark.parametrize("scale", [10, 14, 16])
@pytest.mark.parametrize("flags", [0, 0x2, 0x2 | 0x10, 0x20])
def test_chunked_rmat_build_matches_one_shot(d, scale, flags):
    """The chunked build (edge stream regenerated per chunk of source rows,
    forced here with several chunks) gives the same CSR, renumbering and
    statistics as the one-shot build."""
    spec = inputs.rmat(scale)
    g1 = d.rmat_graph(spec, flags=flags)
    g2 = d.rmat_graph(spec, flags=flags | d.DOBFS_GRAPH_CHUNKED)
    i1, i2 = g1.info, g2.info
    for f in ("n_vertices", "n_entries", "n_nonisolated", "max_degree", "offsets_int64", "reindexed"):
        assert getattr(i1, f) == getattr(i2, f), f
    for a, b in zip(g1.export(), g2.export()):
        np.testing.assert_array_equal(a, b)
    og = oracle.csr_from_rmat(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 3, og.degrees() > 0)
    ref, _ = oracle.bfs_many(og, roots, want_parent=False)
    for k, r in enumerate(roots):
        lv, pa, _ = _run(d, g2, int(r))
        _check_run(og, int(r), lv, pa, ref[k])


def test_pairs_and_csr_inputs(d):
    rng = np.random.default_rng(11)
    n = 3000
    src = rng.integers(0, n, 20000).astype(np.int32)
    dst = rng.integers(0, n, 20000).astype(np.int32)
    og = oracle.csr_from_pairs(n, src, dst)
    for flags in (0, d.DOBFS_GRAPH_REINDEX):
        g = d.pairs_graph(n, src, dst, flags=flags)
        off, cols, n2o = g.export()
        if not flags:
            np.testing.assert_array_equal(off, og.off)
            np.testing.assert_array_equal(cols, og.cols)
        else:
            assert g.info.n_entries == og.nnz
    # device pointers for the pairs give the same graph
    g2 = d.pairs_graph(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    np.testing.assert_array_equal(g2.export()[1], og.cols)
    # a directed CSR made symmetric by the library
    order = np.lexsort((dst, src))
    s_sorted, d_sorted = src[order], dst[order]
    doff = np.zeros(n + 1, dtype=np.int64)
    np.add.at(doff, s_sorted + 1, 1)
    doff = np.cumsum(doff)
    g3 = d.csr_graph(doff, d_sorted.copy(), n, flags=d.DOBFS_GRAPH_SYMMETRIZE)
    off3, cols3, _ = g3.export()
    np.testing.assert_array_equal(off3, og.off)
    np.testing.assert_array_equal(cols3, og.cols)
    # the symmetric CSR passes VALIDATE; the directed one does not
    d.csr_graph(og.off, og.cols, n, flags=d.DOBFS_GRAPH_VALIDATE).close()
    with pytest.raises(d.DobfsError) as e:
        d.csr_graph(doff, d_sorted.copy(), n, flags=d.DOBFS_GRAPH_VALIDATE)
    assert e.value.status == d.DOBFS_ERR_BAD_GRAPH
    bad = og.cols.copy()
    bad[5] = n
    with pytest.raises(d.DobfsError) as e:
        d.csr_graph(og.off, bad, n)
    assert e.value.status == d.DOBFS_ERR_BAD_GRAPH
    with pytest.raises(d.DobfsError) as e:
        d.pairs_graph(n, src, np.full_like(dst, -1))
    assert e.value.status == d.DOBFS_ERR_BAD_GRAPH


# ------------------------------------------------------------------ BFS parity
@pytest.fixture(scope="module")
def s16(d):
    """R-MAT scale 16, edgefactor 16, int32 offsets, relabel on, reindex off; 16 roots."""
    spec = inputs.rmat(16)
    og = oracle.csr_from_rmat(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 16, og.degrees() > 0)
    lv, pa = oracle.bfs_many(og, roots)
    return spec, og, roots, lv, pa


@pytest.mark.parametrize("name,mode,seed", MODES)
def test_levels_bit_exact_s16_no_reindex(d, s16, name, mode, seed):
    spec, og, roots, ref_l, ref_p = s16
    g = d.rmat_graph(spec, flags=0)
    assert g.info.offsets_int64 == 0
    for i, r in enumerate(roots):
        lv, pa, st = _run(d, g, int(r), mode, seed)
        _check_run(og, int(r), lv, pa, ref_l[i])
        assert st.teps_edges == oracle.teps_edges(og, ref_l[i])
        assert st.reached == int((ref_l[i] >= 0).sum())
        assert st.levels == int(ref_l[i].max()) + 1
        if mode == 1:
            assert st.bu_levels == 0
        if mode == 2:
            assert st.td_levels == 0


@pytest.mark.parametrize("name,mode,seed", MODES)
def test_levels_bit_exact_s16_reindex_off64(d, s16, name, mode, seed):
    spec, og, roots, ref_l, ref_p = s16
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX | d.DOBFS_GRAPH_OFFSETS64)
    for i, r in enumerate(roots[:6]):
        lv, pa, st = _run(d, g, int(r), mode, seed)
        _check_run(og, int(r), lv, pa, ref_l[i])


def test_levels_bit_exact_s16_exact_reindex(d, s16):
    spec, og, roots, ref_l, ref_p = s16
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX_EXACT)
    for i, r in enumerate(roots[:6]):
        for mode in (0, 2):
            lv, pa, _ = _run(d, g, int(r), mode)
            _check_run(og, int(r), lv, pa, ref_l[i])


@pytest.mark.parametrize("div", [0, 1 << 30])
@pytest.mark.parametrize("split", [0, 1, 150, 5000])
@pytest.mark.parametrize("mode,seed", [(0, 0), (1, 0), (3, 5), (3, 9)])
def test_topdown_bitmap_output(d, s16, div, split, mode, seed):
    """Top-down levels with bitmap output and parent recovery (div = 2^30 makes
    every top-down level take it) against the queue form (div = 0); on the
    degree-sorted graph, bitmap-output levels are mixed levels unless split = 0
    (split = 1 puts every vertex in the bottom-up part, 5000 only the hubs)."""
    spec, og, roots, ref_l, ref_p = s16
    for flags in (0, d.DOBFS_GRAPH_REINDEX):
        g = d.rmat_graph(spec, flags=flags)
        mixed = 0
        for i, r in enumerate(roots[:4]):
            lv, pa, st = _run(d, g, int(r), mode, seed, td_bitmap_div=div, td_split_pct=split)
            _check_run(og, int(r), lv, pa, ref_l[i])
            assert st.teps_edges == oracle.teps_edges(og, ref_l[i])
            mixed += sum(t.direction == 2 for t in g.trace())
            lv, pa, _ = _run(d, g, int(r), mode, seed, flags=d.DOBFS_RUN_CANONICAL_PARENT, td_bitmap_div=div,
                             td_split_pct=split)
            _check_run(og, int(r), lv, pa, ref_l[i], ref_p[i])
        if flags == 0 or split == 0 or div == 0:
            assert mixed == 0
        elif mode == 1 and split in (1, 150):  # every level top-down: the heavy ones are mixed
            assert mixed > 0


@pytest.mark.parametrize("cut", [dict(td_small_max=8, td_chunk=256, bu_scan=1),
                                 dict(td_small_max=256, td_chunk=8192, bu_scan=256),
                                 dict(td_small_max=33, td_chunk=1152, bu_scan=7)])
@pytest.mark.parametrize("mode,seed", [(0, 0), (3, 5)])
def test_degree_bin_cutoffs(d, s16, cut, mode, seed):
    """Non-default degree-bin cutoffs change which kernel expands a row, never
    the levels; the bitmap-output top-down form is covered too."""
    spec, og, roots, ref_l, ref_p = s16
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    for i, r in enumerate(roots[:4]):
        for div in (0, 2, 1 << 30):
            lv, pa, _ = _run(d, g, int(r), mode, seed, td_bitmap_div=div, **cut)
            _check_run(og, int(r), lv, pa, ref_l[i])


@pytest.mark.parametrize("blocks", [dict(bu_threads=128, td_threads=512, out_threads=128),
                                    dict(bu_threads=512, td_threads=128, out_threads=512),
                                    dict(bu_threads=128, td_threads=128, out_threads=256)])
@pytest.mark.parametrize("mode,seed", [(0, 0), (3, 7)])
def test_block_sizes(d, s16, blocks, mode, seed):
    """Threads per block of the step and output kernels change only the
    speed: levels bit-exact and parents valid for every block size, with the
    level graph rebuilt when the block sizes change between runs, and in
    host-driven levels."""
    spec, og, roots, ref_l, ref_p = s16
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    for i, r in enumerate(roots[:3]):
        for div in (0, 2):
            lv, pa, _ = _run(d, g, int(r), mode, seed, td_bitmap_div=div, **blocks)
            _check_run(og, int(r), lv, pa, ref_l[i])
            lv, pa, _ = _run(d, g, int(r), mode, seed, td_bitmap_div=div)  # back to the defaults
            _check_run(og, int(r), lv, pa, ref_l[i])
        lv, pa, _ = _run(d, g, int(r), mode, seed, flags=d.DOBFS_RUN_HOST_LOOP, **blocks)
        _check_run(og, int(r), lv, pa, ref_l[i])


@pytest.mark.parametrize("bad", [dict(td_small_max=7), dict(td_small_max=257), dict(td_chunk=200),
                                 dict(td_chunk=8320), dict(td_chunk=300), dict(bu_scan=-1), dict(bu_scan=257),
                                 dict(td_split_pct=-1), dict(td_split_pct=100001), dict(bu_threads=64),
                                 dict(td_threads=1024), dict(out_threads=300)])
def test_bad_cutoffs_rejected(d, s16, bad):
    spec, og, roots, ref_l, ref_p = s16
    g = d.rmat_graph(spec)
    with pytest.raises(d.DobfsError) as e:
        _run(d, g, int(roots[0]), **bad)
    assert e.value.status == d.DOBFS_ERR_INVALID


def test_canonical_parent_bit_exact(d, s16):
    spec, og, roots, ref_l, ref_p = s16
    for flags in (0, d.DOBFS_GRAPH_REINDEX):
        g = d.rmat_graph(spec, flags=flags)
        for i, r in enumerate(roots[:8]):
            lv, pa, _ = _run(d, g, int(r), 0, flags=d.DOBFS_RUN_CANONICAL_PARENT)
            _check_run(og, int(r), lv, pa, ref_l[i], ref_p[i])


def test_host_outputs_and_host_loop(d, s16):
    spec, og, roots, ref_l, ref_p = s16
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    r = int(roots[0])
    lv, pa, st = _run(d, g, r, host=True)
    _check_run(og, r, lv, pa, ref_l[0])
    # host levels alone (no parent array)
    lv1 = np.full(og.n, 7, dtype=np.int32)
    g.run(r, lv1)
    np.testing.assert_array_equal(lv1, ref_l[0])
    lv2, pa2, st2 = _run(d, g, r, flags=d.DOBFS_RUN_HOST_LOOP)
    _check_run(og, r, lv2, pa2, ref_l[0])
    tr = g.trace()
    assert len(tr) == st2.levels
    assert sum(t.n_next for t in tr) + 1 == st2.reached
    assert all(t.ms > 0 for t in tr)
    assert [t.level for t in tr] == list(range(len(tr)))
    # the same schedule and counters as the graph-driven run
    _run(d, g, r)
    tr1 = g.trace()
    assert [(t.direction, t.n_frontier, t.m_frontier, t.n_next) for t in tr1] == \
           [(t.direction, t.n_frontier, t.m_frontier, t.n_next) for t in tr]
    # direction-optimized: some level bottom-up, the first top-down
    assert tr1[0].direction == 0 and any(t.direction == 1 for t in tr1)


@pytest.mark.parametrize("name,mode,seed", MODES)
def test_fused_loop_matches_level_graph(d, s16, name, mode, seed):
    """A small graph runs all its levels in one cooperative kernel; the same
    runs through the CUDA level graph (DOBFS_RUN_LEVEL_GRAPH) take the same
    schedule with the same per-level counters, and both reach the oracle's
    levels, also with bitmap-output top-down and mixed levels."""
    spec, og, roots, ref_l, ref_p = s16
    for flags in (0, d.DOBFS_GRAPH_REINDEX | d.DOBFS_GRAPH_OFFSETS64):
        g = d.rmat_graph(spec, flags=flags)
        for i, r in enumerate(roots[:3]):
            for div in (0, 2, 1 << 30):
                traces, stats = [], []
                for rf in (0, d.DOBFS_RUN_LEVEL_GRAPH):
                    lv, pa, st = _run(d, g, int(r), mode, seed, flags=rf, td_bitmap_div=div)
                    _check_run(og, int(r), lv, pa, ref_l[i])
                    traces.append([(t.direction, t.n_frontier, t.m_frontier, t.n_next, t.edges_examined, t.vertices_scanned,
                                    t.alg_bytes) for t in g.trace()])
                    stats.append((st.levels, st.td_levels, st.bu_levels, st.reached, st.teps_edges, st.alg_bytes))
                assert traces[0] == traces[1], (flags, div)
                assert stats[0] == stats[1], (flags, div)
        g.close()


def test_fused_loop_at_its_size_bound(d):
    """R-MAT scale 21 (1.24 M vertices with edges, below the fused loop's
    bound of 2^21, 64 M stored entries): the fused loop's largest graphs.
    Levels bit-exact against the oracle, parents valid, and the same
    schedule and counters as the level graph."""
    spec = inputs.rmat(21)
    og = oracle.csr_from_rmat_par(spec)
    assert (og.degrees() > 0).sum() <= 1 << 21 and og.nnz <= 1 << 27
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 2, og.degrees() > 0)
    for r in roots:
        ref = oracle.bfs(og, int(r), want_parent=False)[0]
        traces = []
        for rf in (0, d.DOBFS_RUN_LEVEL_GRAPH):
            lv, pa, st = _run(d, g, int(r), flags=rf)
            _check_run(og, int(r), lv, pa, ref)
            traces.append([(t.direction, t.n_frontier, t.m_frontier, t.n_next) for t in g.trace()])
        assert traces[0] == traces[1]
    g.close()


def _pairs_graph(d, n, pairs, flags=0):
    src = np.array([p[0] for p in pairs], dtype=np.int32)
    dst = np.array([p[1] for p in pairs], dtype=np.int32)
    return d.pairs_graph(n, src, dst, flags=flags), oracle.csr_from_pairs(n, src, dst)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("flags", [0, 0x2])
@pytest.mark.parametrize("div", [16, 1 << 30])
def test_closed_forms(d, mode, flags, div):
    n = 2000  # path: 2000 levels
    g, og = _pairs_graph(d, n, [(i, i + 1) for i in range(n - 1)], flags)
    lv, pa, st = _run(d, g, 0, mode, seed=5, td_bitmap_div=div)
    assert lv.tolist() == list(range(n)) and st.levels == n
    lv, pa, _ = _run(d, g, 700, mode, seed=5, td_bitmap_div=div)
    assert lv.tolist() == [abs(i - 700) for i in range(n)]
    # star with 5000 leaves: one long row (chunked top-down, deferred bottom-up)
    n = 5001
    g, og = _pairs_graph(d, n, [(0, i) for i in range(1, n)], flags)
    lv, pa, _ = _run(d, g, 0, mode, seed=5, td_bitmap_div=div)
    assert lv.tolist() == [0] + [1] * (n - 1) and np.all(pa[1:] == 0)
    lv, pa, _ = _run(d, g, 4321, mode, seed=5, td_bitmap_div=div)
    assert lv[0] == 1 and lv[4321] == 0 and int((lv == 2).sum()) == n - 2
    _check_run(og, 4321, lv, pa, oracle.bfs(og, 4321)[0])
    # binary tree in heap order, plus a separate cycle and an isolated vertex
    t = 1023
    pairs = [((i - 1) // 2, i) for i in range(1, t)] + [(t + i, t + (i + 1) % 50) for i in range(50)]
    n = t + 51
    g, og = _pairs_graph(d, n, pairs, flags)
    lv, pa, _ = _run(d, g, 0, mode, seed=5, flags=d.DOBFS_RUN_CANONICAL_PARENT, td_bitmap_div=div)
    assert lv[:t].tolist() == [int(np.floor(np.log2(i + 1))) for i in range(t)]
    assert np.all(lv[t:] == -1) and np.all(pa[t:] == -1)
    assert pa[:t].tolist() == [0] + [(i - 1) // 2 for i in range(1, t)]
    lv, pa, st = _run(d, g, n - 1, mode, seed=5, td_bitmap_div=div)  # isolated root
    assert lv.tolist() == [-1] * (n - 1) + [0] and pa[n - 1] == n - 1 and st.teps_edges == 0


def test_root_out_of_range(d, s16):
    spec = s16[0]
    g = d.rmat_graph(spec, flags=0)
    lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for r in (-1, g.n):
        with pytest.raises(d.DobfsError) as e:
            g.run(r, lv)
        assert e.value.status == d.DOBFS_ERR_INVALID


def test_chunglu_small(d):
    spec = inputs.chunglu(13, max_weight=float(1 << 9))
    cdf = inputs.chunglu_cdf(spec)
    src, dst = inputs.chunglu_pairs(spec, cdf)
    og = oracle.csr_from_pairs(spec.n_vertices, src, dst)
    g = d.chunglu_graph(spec, cdf, flags=0)
    off, cols, _ = g.export()
    np.testing.assert_array_equal(off, og.off)
    np.testing.assert_array_equal(cols, og.cols)
    gr = d.chunglu_graph(spec, cdf)
    roots = inputs.sample_roots(5, og.n, 4, og.degrees() > 0)
    for r in roots:
        ref, _, _ = oracle.bfs(og, int(r), want_parent=False)
        for gg in (g, gr):
            lv, pa, _ = _run(d, gg, int(r))
            _check_run(og, int(r), lv, pa, ref)


def test_repeated_runs_and_streams(d, s16):
    spec, og, roots, ref_l, _ = s16
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for i, r in enumerate(roots[:6]):
        s = s1 if i % 2 else s2
        lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(s):
            g.run(int(r), lv, None, d.make_opts(stream=s))
        outs.append((i, lv, s))
    torch.cuda.synchronize()
    for i, lv, s in outs:
        np.testing.assert_array_equal(lv.cpu().numpy(), ref_l[i])


@pytest.mark.parametrize("mode", [0, 1])
def test_trace_counts_match_the_oracle(d, s16, mode):
    """Per-level frontier sizes and degree sums (the switch's inputs) against
    the oracle's levels and degrees, renumbered and not: the new frontier's
    degree sum is read from the degree-class ranges for small degrees."""
    spec, og, roots, ref_l, _ = s16
    deg = og.degrees().astype(np.int64)
    for flags in (0, d.DOBFS_GRAPH_REINDEX, d.DOBFS_GRAPH_REINDEX_EXACT):
        g = d.rmat_graph(spec, flags=flags)
        for i, r in enumerate(roots[:3]):
            _run(d, g, int(r), mode=mode)
            tr = g.trace()
            lv = ref_l[i]
            assert len(tr) == int(lv.max()) + 1
            for t in tr:
                at = lv == t.level
                assert t.n_frontier == int(at.sum()), (flags, t.level)
                assert t.m_frontier == int(deg[at].sum()), (flags, t.level)
                assert t.n_next == int((lv == t.level + 1).sum())
        g.close()
