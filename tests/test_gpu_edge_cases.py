"""GPU edge cases through the C ABI: graphs without edges, a single vertex,
input made only of self-loops, vertex counts that are not multiples of 4 or
32 (ragged tails of the vectorised passes), empty batches, and R-MAT builds
with no pairs (one-shot and chunked). Results against the oracle."""
import time

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


def _run(d, g, root, **kw):
    n = g.n
    lv = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    pa = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    st = g.run(int(root), lv, pa, d.make_opts(**kw), want_stats=True)
    torch.cuda.synchronize()
    return lv.cpu().numpy(), pa.cpu().numpy(), st


def _isolated_expect(n, r):
    lv = np.full(n, -1, dtype=np.int32)
    pa = np.full(n, -1, dtype=np.int32)
    lv[r] = 0
    pa[r] = r
    return lv, pa


@pytest.mark.parametrize("n", [1, 5, 33, 1000])
@pytest.mark.parametrize("flags", [0, 0x2, 0x2 | 0x10])
def test_graph_without_edges(d, n, flags):
    empty = np.zeros(0, dtype=np.int32)
    loops = np.arange(n, dtype=np.int32)  # self-loops only: dropped, so no edges either
    for src, dst in ((empty, empty), (loops, loops)):
        g = d.pairs_graph(n, src, dst, flags=flags)
        assert g.info.n_entries == 0 and g.info.n_nonisolated == 0
        for r in sorted({0, n // 2, n - 1}):
            for mode in (0, 1, 2):
                lv, pa, st = _run(d, g, r, direction=mode)
                elv, epa = _isolated_expect(n, r)
                np.testing.assert_array_equal(lv, elv)
                np.testing.assert_array_equal(pa, epa)
                assert st.levels == 1 and st.reached == 1 and st.teps_edges == 0
        roots = np.array(sorted({0, n - 1, n // 3}), dtype=np.int32)
        out = torch.full((len(roots), n), 7, dtype=torch.int32, device="cuda")
        d.dobfs_run_batch(g.handle, torch.from_numpy(roots).cuda(), out)
        got = out.cpu().numpy()
        for i, r in enumerate(roots):
            np.testing.assert_array_equal(got[i], _isolated_expect(n, int(r))[0])
        g.close()


@pytest.mark.parametrize("n", [33, 1001, 4099])
@pytest.mark.parametrize("flags", [0, 0x2])
def test_ragged_vertex_counts(d, n, flags):
    rng = np.random.default_rng(n)
    m = 6 * n
    # a dense core and a sparse tail, plus isolated vertices at random places
    src = np.concatenate([rng.integers(0, n // 8 + 1, m // 2), rng.integers(0, n, m // 2)]).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    keep = rng.random(m) < 0.9
    src, dst = src[keep], dst[keep]
    og = oracle.csr_from_pairs(n, src, dst)
    g = d.pairs_graph(n, src, dst, flags=flags)
    deg = og.degrees()
    roots = inputs.sample_roots(0x5EED + n, n, min(70, int((deg > 0).sum())), deg > 0)
    ref_l, ref_p = oracle.bfs_many(og, roots)
    for i, r in enumerate(roots[:6]):
        for mode in (0, 1, 2):
            lv, pa, _ = _run(d, g, int(r), direction=mode)
            np.testing.assert_array_equal(lv, ref_l[i])
            rule, bad = oracle.check_bfs(og, int(r), lv, pa)
            assert rule == 0, (oracle.RULES[rule], bad)
        lv, pa, _ = _run(d, g, int(r), flags=d.DOBFS_RUN_CANONICAL_PARENT)
        np.testing.assert_array_equal(pa, ref_p[i])
    # batched rows (a full group and a partial one) and host outputs
    out = torch.full((len(roots), n), 7, dtype=torch.int32, device="cuda")
    d.dobfs_run_batch(g.handle, torch.from_numpy(np.ascontiguousarray(roots)).cuda(), out)
    np.testing.assert_array_equal(out.cpu().numpy(), ref_l)
    host = np.full((3, n), 7, dtype=np.int32)
    d.dobfs_run_batch(g.handle, np.ascontiguousarray(roots[:3]), host)
    np.testing.assert_array_equal(host, ref_l[:3])
    g.close()


def test_empty_batch(d):
    spec = inputs.rmat(10)
    g = d.rmat_graph(spec)
    out = torch.empty((0, g.n), dtype=torch.int32, device="cuda")
    d.dobfs_run_batch(g.handle, torch.empty(0, dtype=torch.int32, device="cuda"), out)
    g.close()


@pytest.mark.parametrize("flags", [0, 0x2, 0x2 | 0x40])
def test_rmat_without_pairs(d, flags):
    ta, tab, tabc = inputs.rmat(8).thresholds
    g = d.Graph(d.dobfs_graph_create_rmat(8, 0, ta, tab, tabc, 1, flags, None))
    assert g.info.n_entries == 0 and g.n == 256
    lv, pa, _ = _run(d, g, 17)
    elv, epa = _isolated_expect(256, 17)
    np.testing.assert_array_equal(lv, elv)
    np.testing.assert_array_equal(pa, epa)
    g.close()


def test_serve_on_graph_without_edges(d):
    n = 77
    g = d.pairs_graph(n, np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.int32), flags=0x2)
    for ss_max in (0, 2):
        srv = d.dobfs_serve_create(d.make_serve_opts(ss_max=ss_max))
        try:
            gid = d.dobfs_serve_add_graph(srv, g.handle)
            outs = [torch.full((n,), 7, dtype=torch.int32, device="cuda") for _ in range(3)]
            tickets = [d.dobfs_serve_submit(srv, gid, r, outs[i]) for i, r in enumerate((0, 40, 76))]
            for i, t in enumerate(tickets):
                t0 = time.time()
                while True:
                    r = d.dobfs_serve_poll(srv, t)
                    if r is not None:
                        break
                    assert time.time() - t0 < 60, "query did not finish"
                    time.sleep(0.0005)
                assert r.status == 0 and r.levels == 1
                np.testing.assert_array_equal(outs[i].cpu().numpy(), _isolated_expect(n, (0, 40, 76)[i])[0])
        finally:
            d.dobfs_serve_destroy(srv)
    g.close()
