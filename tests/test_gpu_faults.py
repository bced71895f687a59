"""Failure handling, injected on the host: device allocations that fail, and
bounded host waits that run out.

The library takes every device allocation through the allocator hook
(dobfs_set_allocator). A counting allocator that delegates to PyTorch and
refuses the k-th request stands in for an out-of-memory device: each entry
point must return DOBFS_ERR_OOM, free what it had allocated (no block left
outstanding), and leave the library usable. Nothing here faults the GPU.
"""
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
    yield dobfs
    dobfs.use_torch_allocator()


class FailingAllocator:
    """Delegates to PyTorch; refuses request number `fail_at` (0-based)."""

    def __init__(self, d, fail_at=None):
        self.d = d
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        dev = torch.cuda.current_device()

        @d.ALLOC_FN
        def _alloc(nbytes, stream, ctx):
            k = self.calls
            self.calls += 1
            if self.fail_at is not None and k == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
            self.live[p] = int(nbytes)
            return p

        @d.FREE_FN
        def _free(ptr, stream, ctx):
            self.live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

        self._keep = (_alloc, _free)

    def install(self):
        self.d._check(self.d.load().dobfs_set_allocator(self._keep[0], self._keep[1], None))
        return self


def _levels(d, g, r):
    lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
    g.run(int(r), lv)
    torch.cuda.synchronize()
    return lv.cpu().numpy()


def test_graph_build_fails_cleanly_at_every_allocation(d):
    spec = inputs.rmat(12)
    for flags in (0, d.DOBFS_GRAPH_REINDEX, d.DOBFS_GRAPH_REINDEX | d.DOBFS_GRAPH_CHUNKED):
        counter = FailingAllocator(d).install()
        g = d.rmat_graph(spec, flags=flags)
        total = counter.calls
        g.close()
        torch.cuda.synchronize()
        assert total > 5 and not counter.live
        for k in range(total):
            fa = FailingAllocator(d, fail_at=k).install()
            with pytest.raises(d.DobfsError) as e:
                d.rmat_graph(spec, flags=flags)
            assert e.value.status == d.DOBFS_ERR_OOM, (flags, k, e.value)
            torch.cuda.synchronize()
            assert not fa.live, "allocation %d refused: %d blocks left" % (k, len(fa.live))
    # the library is usable afterwards
    d.use_torch_allocator()
    og = oracle.csr_from_rmat(spec)
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    root = int(inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 1, og.degrees() > 0)[0])
    np.testing.assert_array_equal(_levels(d, g, root), oracle.bfs(og, root)[0])
    g.close()


def test_run_batch_and_serve_fail_cleanly(d):
    spec = inputs.rmat(12)
    og = oracle.csr_from_rmat(spec)
    d.use_torch_allocator()
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 8, og.degrees() > 0)
    ref, _ = oracle.bfs_many(og, roots, want_parent=False)
    # host outputs need a staging buffer (the graph's first host-output run)
    fa = FailingAllocator(d, fail_at=0).install()
    host = np.empty(og.n, dtype=np.int32)
    with pytest.raises(d.DobfsError) as e:
        g.run(int(roots[0]), host)
    assert e.value.status == d.DOBFS_ERR_OOM
    assert not fa.live
    # a graph's first batch allocates its lane group (kept for later batches):
    # refuse each of those allocations in turn, on a fresh graph each time
    rt = torch.from_numpy(np.ascontiguousarray(roots)).cuda()
    out = torch.empty((8, og.n), dtype=torch.int32, device="cuda")
    d.use_torch_allocator()
    g2 = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    counter = FailingAllocator(d).install()
    d.dobfs_run_batch(g2.handle, rt, out)
    torch.cuda.synchronize()
    total = counter.calls
    assert total >= 3 and len(counter.live) == total
    g2.close()
    assert not counter.live
    for k in range(total):
        d.use_torch_allocator()
        g2 = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
        fb = FailingAllocator(d, fail_at=k).install()
        with pytest.raises(d.DobfsError) as e:
            d.dobfs_run_batch(g2.handle, rt, out)
        assert e.value.status == d.DOBFS_ERR_OOM
        torch.cuda.synchronize()
        assert not fb.live, "allocation %d refused: %d blocks left" % (k, len(fb.live))
        # the graph is still usable once memory is back
        d.dobfs_run_batch(g2.handle, rt, out)
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        g2.close()
        assert not fb.live
    # a server allocates the graph's lane groups when the graph is added: refuse
    # each of those allocations in turn; the server then takes the graph and works
    counter = FailingAllocator(d).install()
    srv = d.dobfs_serve_create()
    d.dobfs_serve_add_graph(srv, g.handle)
    d.dobfs_serve_destroy(srv)
    total = counter.calls
    assert total >= 3 and not counter.live
    for k in range(total):
        fs = FailingAllocator(d, fail_at=k).install()
        srv = d.dobfs_serve_create()
        try:
            with pytest.raises(d.DobfsError) as e:
                d.dobfs_serve_add_graph(srv, g.handle)
            assert e.value.status == d.DOBFS_ERR_OOM
            torch.cuda.synchronize()
            assert not fs.live, "allocation %d refused: %d blocks left" % (k, len(fs.live))
            d.use_torch_allocator()
            gid = d.dobfs_serve_add_graph(srv, g.handle)
            out1 = torch.full((og.n,), 9, dtype=torch.int32, device="cuda")
            t = d.dobfs_serve_submit(srv, gid, int(roots[1]), out1)
            t0 = time.time()
            while d.dobfs_serve_poll(srv, t) is None:
                assert time.time() - t0 < 60, "query did not finish"
                time.sleep(0.001)
            np.testing.assert_array_equal(out1.cpu().numpy(), ref[1])
        finally:
            d.dobfs_serve_destroy(srv)
    # after the failures: the graph still answers, single and batched
    d.use_torch_allocator()
    np.testing.assert_array_equal(_levels(d, g, roots[2]), ref[2])
    out = torch.empty((8, og.n), dtype=torch.int32, device="cuda")
    d.dobfs_run_batch(g.handle, torch.from_numpy(np.ascontiguousarray(roots)).cuda(), out)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    g.close()


def test_graph_load_fails_cleanly_at_every_allocation(d, tmp_path):
    spec = inputs.rmat(12)
    og = oracle.csr_from_rmat(spec)
    d.use_torch_allocator()
    g = d.rmat_graph(spec, flags=d.DOBFS_GRAPH_REINDEX)
    path = str(tmp_path / "g.dobfs")
    g.save(path)
    g.close()
    counter = FailingAllocator(d).install()
    h = d.load_graph(path)
    total = counter.calls
    h.close()
    torch.cuda.synchronize()
    assert total > 5 and not counter.live
    for k in range(total):
        fa = FailingAllocator(d, fail_at=k).install()
        with pytest.raises(d.DobfsError) as e:
            d.load_graph(path)
        assert e.value.status == d.DOBFS_ERR_OOM, (k, e.value)
        torch.cuda.synchronize()
        assert not fa.live, "allocation %d refused: %d blocks left" % (k, len(fa.live))
    d.use_torch_allocator()
    h = d.load_graph(path)
    root = int(inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 1, og.degrees() > 0)[0])
    np.testing.assert_array_equal(_levels(d, h, root), oracle.bfs(og, root)[0])
    h.close()


def test_bounded_wait_runs_out_then_completes(d):
    """dobfs_graph_wait: a run and a batch queued behind a fixed-length
    spinning kernel (torch.cuda._sleep, about half a second) are still running
    at a 0 ms and a 20 ms limit (DOBFS_ERR_TIMEOUT; nothing is cancelled), and
    a wait without limit then returns once they are done, with the oracle's
    levels. No GPU wait is involved: the kernels only run late."""
    spec = inputs.rmat(14)
    og = oracle.csr_from_rmat(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 3, og.degrees() > 0)
    ref, _ = oracle.bfs_many(og, roots, want_parent=False)
    g = d.rmat_graph(spec)
    assert g.wait(0)  # nothing queued
    s = torch.cuda.Stream()
    lv = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    out = torch.full((2, g.n), 7, dtype=torch.int32, device="cuda")
    o = d.make_opts(stream=s)
    # warm-up: the run workspace, its CUDA graph and the batch's lane group
    # exist afterwards, so the calls below only queue work
    g.run(int(roots[0]), lv, None, o)
    d.dobfs_run_batch(g.handle, np.ascontiguousarray(roots[1:]), out, opts=o)
    assert g.wait(-1)
    for batch in (False, True):
        lv.fill_(7)
        out.fill_(7)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            torch.cuda._sleep(1_000_000_000)
        if batch:
            d.dobfs_run_batch(g.handle, np.ascontiguousarray(roots[1:]), out, opts=o)
        else:
            g.run(int(roots[0]), lv, None, o)
        assert not g.wait(0)
        assert not g.wait(20)
        assert "still running" in d.last_error()
        assert g.wait(-1)
        if batch:
            np.testing.assert_array_equal(out.cpu().numpy(), ref[1:])
        else:
            np.testing.assert_array_equal(lv.cpu().numpy(), ref[0])
    g.close()
    with pytest.raises(d.DobfsError) as e:
        d.dobfs_graph_wait(None, 0)
    assert e.value.status == d.DOBFS_ERR_INVALID


def test_grid_barrier_completes_and_times_out(d):
    """The grid barrier of the fused small-graph loop: many rounds over every
    resident block complete with every block's writes visible after each
    barrier; a barrier that waits for a block that was never launched runs
    out after its 2 s bound in every block, the launch ends, the flag says
    so, and the library (and context) stay usable."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for blocks, rounds in ((1, 10), (sms, 2000), (4 * sms, 500)):
        assert d.dobfs_debug_grid_barrier(blocks, rounds, 0) == (rounds, 0, False)
    t0 = time.perf_counter()
    passed, short, timed_out = d.dobfs_debug_grid_barrier(2 * sms, 3, 1)
    dt = time.perf_counter() - t0
    assert timed_out and passed == 0 and short == 0
    assert 1.5 < dt < 60, dt
    with pytest.raises(d.DobfsError) as e:
        d.dobfs_debug_grid_barrier(0, 1, 0)
    assert e.value.status == d.DOBFS_ERR_INVALID
    # a small graph (fused loop) after the timed-out launch: levels exact
    spec = inputs.rmat(12)
    og = oracle.csr_from_rmat(spec)
    g = d.rmat_graph(spec)
    r = int(inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 1, og.degrees() > 0)[0])
    lv = np.empty(og.n, dtype=np.int32)
    g.run(r, lv)
    np.testing.assert_array_equal(lv, oracle.bfs(og, r)[0])
    g.close()


def test_random_access_probe(d):
    """The scattered-access measurement aid runs and checks its arguments."""
    for width, write in ((4, False), (8, False), (16, False), (8, True)):
        ms, made = d.dobfs_debug_random_access(1 << 26, 1 << 20, width, write)
        assert ms > 0 and made >= 1 << 20
    for bad in (dict(array_bytes=3 << 20), dict(array_bytes=1 << 10), dict(width=12), dict(accesses=0)):
        kw = dict(array_bytes=1 << 26, accesses=1 << 20, width=8)
        kw.update(bad)
        with pytest.raises(d.DobfsError) as e:
            d.dobfs_debug_random_access(kw["array_bytes"], kw["accesses"], kw["width"])
        assert e.value.status == d.DOBFS_ERR_INVALID
