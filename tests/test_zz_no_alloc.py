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
