"""GPU parity of batched (bit-parallel lane groups) BFS against the CPU oracle.

Every row of the batch output must equal the oracle's level array for that
root bit-exact, whatever the direction schedule, the batch size (full and
partial lane groups, several groups, 64- and 128-lane groups) or repeated roots.
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


@pytest.fixture(scope="module")
def s14():
    spec = inputs.rmat(14)
    og = oracle.csr_from_rmat(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 300, og.degrees() > 0)
    lv, _ = oracle.bfs_many(og, roots, want_parent=False)
    return spec, og, roots, lv


def _batch(d, g, roots, mode=0, seed=0, host=False, **kw):
    n = g.n
    roots = np.asarray(roots, dtype=np.int32)
    if host:
        out = np.full((len(roots), n), 7, dtype=np.int32)
        d.dobfs_run_batch(g.handle, roots, out, opts=d.make_opts(direction=mode, schedule_seed=seed, **kw))
        return out
    out = torch.full((len(roots), n), 7, dtype=torch.int32, device="cuda")
    d.dobfs_run_batch(g.handle, torch.from_numpy(roots).cuda(), out,
                      opts=d.make_opts(direction=mode, schedule_seed=seed, **kw))
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("mode,seed", [(0, 0), (1, 0), (2, 0), (3, 1), (3, 2)])
@pytest.mark.parametrize("flags", [0, 0x2])
def test_batch_levels_bit_exact(d, s14, mode, seed, flags):
    spec, og, roots, ref = s14
    g = d.rmat_graph(spec, flags=flags)
    out = _batch(d, g, roots, mode, seed)          # two full 128-lane groups and a partial one of 44
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("cut", [dict(td_chunk=256, bu_scan=1), dict(td_chunk=8192, bu_scan=256),
                                 dict(td_chunk=640, bu_scan=9)])
def test_batch_degree_bin_cutoffs(d, s14, cut):
    spec, og, roots, ref = s14
    g = d.rmat_graph(spec, flags=0x2)
    for mode, seed in ((0, 0), (3, 4)):
        np.testing.assert_array_equal(_batch(d, g, roots[:64], mode, seed, **cut), ref[:64])
    with pytest.raises(d.DobfsError):
        _batch(d, g, roots[:4], td_chunk=100)


@pytest.mark.parametrize("blocks", [dict(bu_threads=128, td_threads=512), dict(bu_threads=512, td_threads=128)])
def test_batch_block_sizes(d, s14, blocks):
    """Threads per block of the batched step kernels change only the speed;
    the loop graph is rebuilt when they change between batches."""
    spec, og, roots, ref = s14
    g = d.rmat_graph(spec, flags=0x2)
    for mode, seed in ((0, 0), (3, 4)):
        np.testing.assert_array_equal(_batch(d, g, roots[:64], mode, seed, **blocks), ref[:64])
        np.testing.assert_array_equal(_batch(d, g, roots[:64], mode, seed), ref[:64])
        np.testing.assert_array_equal(_batch(d, g, roots[:200], mode, seed, **blocks), ref[:200])


def test_batch_sizes_duplicates_host(d, s14):
    spec, og, roots, ref = s14
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX | d.DOBFS_GRAPH_OFFSETS64)
    # 64 roots or fewer: one 64-lane group; more: 128-lane groups, full and partial
    for k in (1, 3, 63, 64, 65, 127, 128, 129, 300):
        np.testing.assert_array_equal(_batch(d, g, roots[:k]), ref[:k])
    np.testing.assert_array_equal(_batch(d, g, roots[:40]), ref[:40])  # back to 64 lanes
    dup = np.array([roots[0], roots[1], roots[0], roots[0]], dtype=np.int32)
    np.testing.assert_array_equal(_batch(d, g, dup), ref[[0, 1, 0, 0]])
    np.testing.assert_array_equal(_batch(d, g, roots[:70], host=True), ref[:70])
    np.testing.assert_array_equal(_batch(d, g, roots[:200], host=True), ref[:200])
    # same as single-source runs of the same graph
    lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
    g.run(int(roots[5]), lv)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lv.cpu().numpy(), ref[5])


def test_batch_closed_forms(d):
    # a path of 3000 vertices (levels up to 2999: iteration planes cleared as they come into use),
    # a star, and a separate triangle plus an isolated vertex
    n_path = 3000
    pairs = [(i, i + 1) for i in range(n_path - 1)]
    star0 = n_path
    pairs += [(star0, star0 + i) for i in range(1, 200)]
    tri = star0 + 200
    pairs += [(tri, tri + 1), (tri + 1, tri + 2), (tri + 2, tri)]
    n = tri + 4
    src = np.array([p[0] for p in pairs], dtype=np.int32)
    dst = np.array([p[1] for p in pairs], dtype=np.int32)
    og = oracle.csr_from_pairs(n, src, dst)
    roots = np.array([0, 1500, n_path - 1, star0, star0 + 7, tri, n - 1], dtype=np.int32)
    ref = np.stack([oracle.bfs(og, int(r), want_parent=False)[0] for r in roots])
    for flags in (0, 0x2):
        g = d.pairs_graph(n, src, dst, flags=flags)
        for mode in (0, 1, 2):
            np.testing.assert_array_equal(_batch(d, g, roots, mode), ref)


def test_batch_rejects_parents_and_bad_roots(d, s14):
    spec, og, roots, ref = s14
    g = d.rmat_graph(spec, flags=0)
    out = torch.empty((2, g.n), dtype=torch.int32, device="cuda")
    with pytest.raises(d.DobfsError) as e:
        d.dobfs_run_batch(g.handle, roots[:2], out, parent_out=out)
    assert e.value.status == d.DOBFS_ERR_INVALID
    with pytest.raises(d.DobfsError) as e:
        d.dobfs_run_batch(g.handle, np.array([0, g.n], dtype=np.int32), out)
    assert e.value.status == d.DOBFS_ERR_INVALID


def test_batch_alg_bytes_closed_form(d, s14):
    """The batch's algorithmic byte count in closed form. One root, top-down
    only, one 64-lane mask word: every reached vertex is active once (its
    seen and next masks, 16 bytes), every entry of its row is examined once
    (the neighbour's mask and the column, 12 bytes), and the flush writes one
    4-byte level per vertex: 16 reached + 12 * (sum of their degrees) + 4 n."""
    spec, og, roots, ref = s14
    g = d.rmat_graph(spec, flags=0x2)
    for i in range(3):
        r = np.asarray(roots[i:i + 1], dtype=np.int32)
        out = torch.empty((1, og.n), dtype=torch.int32, device="cuda")
        st = d.dobfs_run_batch(g.handle, torch.from_numpy(r).cuda(), out,
                               opts=d.make_opts(direction=d.DOBFS_DIR_TOPDOWN), want_stats=True)
        reached = ref[i] >= 0
        deg_sum = int(og.degrees()[reached].sum())
        assert st.edges_examined == deg_sum
        assert st.alg_bytes == 16 * int(reached.sum()) + 12 * deg_sum + 4 * og.n
    g.close()
