"""dobfs_run_static: BFS with no device allocation, checked against dobfs_run.

dobfs_run_static exists for callers that cannot allocate device memory when
they need a BFS (a memory budget reserved up front, allocation-free serving
paths, plugins inside a framework that owns all allocations): its working
memory is one static device array. This test calls it through the C ABI on a
caller-owned device CSR and compares two calls in a row with the main entry
point on the same graph: levels bit-exact (the tolerance of every BFS test
here) and parents valid BFS parents. The file is named so that pytest
collects it last.
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
    return dobfs


def test_static_entry_matches_dobfs_run_twice(d):
    spec = inputs.rmat(16)
    g = d.rmat_graph(spec, flags=0)  # original IDs, sorted rows
    off64, cols, _ = g.export()
    n = g.n
    off_dev = torch.from_numpy(off64.astype(np.int32)).cuda()
    cols_dev = torch.from_numpy(cols).cuda()
    og = oracle.Csr(off64, cols)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), n, 2, og.degrees() > 0)
    for r in roots:  # two calls in a row share the static array
        ref = torch.empty(n, dtype=torch.int32, device="cuda")
        g.run(int(r), ref)
        lv = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        pa = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        d.dobfs_run_static(off_dev, cols_dev, n, int(r), lv, pa)
        torch.cuda.synchronize()
        lvh, pah = lv.cpu().numpy(), pa.cpu().numpy()
        np.testing.assert_array_equal(lvh, ref.cpu().numpy())
        rule, bad = oracle.check_bfs(og, int(r), lvh, pah)
        assert rule == 0, (oracle.RULES[rule], bad)
    g.close()


def _static_vs_run(d, g, og, roots, parent_none=()):
    """dobfs_run_static on g's exported CSR against dobfs_run on g for every
    root: levels bit-exact, parents valid (or NULL for the listed roots).
    Returns the direction sequence of every dobfs_run (its trace)."""
    n = g.n
    off_dev = torch.from_numpy(og.off.astype(np.int32)).cuda()
    cols_dev = torch.from_numpy(og.cols).cuda()
    dirs = []
    for i, r in enumerate(roots):
        ref = torch.empty(n, dtype=torch.int32, device="cuda")
        g.run(int(r), ref, None, d.make_opts(), want_stats=True)
        dirs.append([t.direction for t in g.trace()])
        lv = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        pa = None if i in parent_none else torch.full((n,), 7, dtype=torch.int32, device="cuda")
        d.dobfs_run_static(off_dev, cols_dev, n, int(r), lv, pa)
        torch.cuda.synchronize()
        lvh = lv.cpu().numpy()
        np.testing.assert_array_equal(lvh, ref.cpu().numpy())
        if pa is not None:
            rule, bad = oracle.check_bfs(og, int(r), lvh, pa.cpu().numpy())
            assert rule == 0, (oracle.RULES[rule], bad)
    return dirs


def test_static_entry_at_max_vertices(d):
    """R-MAT scale 20: n is DOBFS_STATIC_MAX_VERTICES, so the bitmaps and
    queues of the static array are used to their last word."""
    spec = inputs.rmat(20)
    assert spec.n_vertices == d.DOBFS_STATIC_MAX_VERTICES
    g = d.rmat_graph(spec, flags=0)
    off64, cols, _ = g.export()
    og = oracle.Csr(off64, cols)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0x57A7, g.n, 4, og.degrees() > 0)
    dirs = _static_vs_run(d, g, og, roots, parent_none=(1,))
    # dobfs_run_static takes its directions by the same alpha/beta rule on the
    # same counts: the traces show that the calls went top-down -> bottom-up
    # (queue -> bitmap) and bottom-up -> top-down (bitmap -> queue)
    def both_switches(ds):
        bu = [k for k, x in enumerate(ds) if x == 1]
        return bool(bu) and ds[0] != 1 and any(x != 1 for x in ds[bu[0]:])
    assert any(both_switches(ds) for ds in dirs), dirs
    g.close()


def test_static_entry_many_levels(d):
    """2^20 vertices: an R-MAT scale-19 core, a path of 3,000 vertices hanging
    off one core vertex, and the rest isolated. A BFS from the path's far end
    runs thousands of top-down levels before the core switches it bottom-up."""
    n = d.DOBFS_STATIC_MAX_VERTICES
    core = inputs.rmat(19)
    src, dst = inputs.rmat_pairs(core)
    hub = int(np.bincount(np.concatenate([src, dst]), minlength=core.n_vertices).argmax())
    plen = 3000
    path = np.arange(core.n_vertices, core.n_vertices + plen, dtype=np.int32)
    psrc = np.concatenate([[hub], path[:-1]]).astype(np.int32)
    pdst = path
    g = d.pairs_graph(n, np.concatenate([src, psrc]), np.concatenate([dst, pdst]), flags=0)
    off64, cols, _ = g.export()
    og = oracle.Csr(off64, cols)
    far_end = int(path[-1])
    dirs = _static_vs_run(d, g, og, [far_end, hub], parent_none=(0,))
    assert len(dirs[0]) > plen
    g.close()


def test_static_entry_rejects_oversize_and_bad_root(d):
    off = torch.zeros(2, dtype=torch.int32, device="cuda")
    cols = torch.zeros(1, dtype=torch.int32, device="cuda")
    lv = torch.empty(1, dtype=torch.int32, device="cuda")
    big = d.DOBFS_STATIC_MAX_VERTICES + 1
    with pytest.raises(d.DobfsError) as e:
        d.dobfs_run_static(off, cols, big, 0, lv)
    assert e.value.status == d.DOBFS_ERR_INVALID and "static working memory" in str(e.value)
    with pytest.raises(d.DobfsError) as e:
        d.dobfs_run_static(off, cols, 1, 1, lv)
    assert e.value.status == d.DOBFS_ERR_INVALID
    # an isolated single vertex: level 0 at the root
    d.dobfs_run_static(off, cols, 1, 0, lv)
    torch.cuda.synchronize()
    assert lv.item() == 0
