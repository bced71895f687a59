"""GPU tests of the query server (continuous batching over resident graphs).

Each query's level array must equal the oracle's for its root, whether the
query runs alone or in a mix of concurrent queries on several graphs of
different scales, with lanes joining traversals already in flight and more
queries than one lane group holds.
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
    return dobfs


@pytest.fixture(scope="module")
def graphs(d):
    out = []
    for scale, flags in ((11, 0), (13, 0x2), (15, 0x2)):
        spec = inputs.rmat(scale)
        og = oracle.csr_from_rmat(spec)
        roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 160, og.degrees() > 0)
        ref, _ = oracle.bfs_many(og, roots, want_parent=False)
        out.append((d.rmat_graph(spec, flags=flags), og, roots, ref))
    return out


def _wait(d, srv, ticket, timeout=60.0):
    t0 = time.time()
    while True:
        r = d.dobfs_serve_poll(srv, ticket)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "query did not finish"
        time.sleep(0.0005)


@pytest.mark.parametrize("ss_max,lane_words", [(0, 1), (2, 1), (0, 2), (2, 2)])
def test_alone_and_in_the_mix(d, graphs, ss_max, lane_words):
    """ss_max = 0: every query runs in a lane group; 2: lone queries take the
    single-source path and bursts the lane groups. Groups of 64 lanes
    (lane_words 1) or 128 (2); the mix holds more queries per graph than a
    group has lanes."""
    srv = d.dobfs_serve_create(d.make_serve_opts(max_groups_per_graph=2, ss_max=ss_max, lane_words=lane_words))
    try:
        gids = [d.dobfs_serve_add_graph(srv, g.handle) for g, _, _, _ in graphs]
        # alone: one query at a time
        alone = {}
        for gi, (g, og, roots, ref) in enumerate(graphs):
            for k in range(3):
                out = torch.full((og.n,), 9, dtype=torch.int32, device="cuda")
                r = _wait(d, srv, d.dobfs_serve_submit(srv, gids[gi], int(roots[k]), out))
                alone[(gi, k)] = out.cpu().numpy()
                np.testing.assert_array_equal(alone[(gi, k)], ref[k])
                assert r.status == 0 and r.levels == int(ref[k].max()) + 1
                assert r.submit_ns <= r.admit_ns <= r.done_ns and r.latency_ns == r.done_ns - r.submit_ns
        # the mix: every query of every graph submitted at once (more than a lane group holds
        # per graph, so queries may wait for lanes or a second group); host outputs for some
        outs, tickets = {}, {}
        n_mix = 160 if lane_words == 2 else 80
        for k in range(n_mix):
            for gi, (g, og, roots, ref) in enumerate(graphs):
                if k % 7 == 3:
                    out = np.full(og.n, 9, dtype=np.int32)
                else:
                    out = torch.full((og.n,), 9, dtype=torch.int32, device="cuda")
                outs[(gi, k)] = out
                tickets[(gi, k)] = d.dobfs_serve_submit(srv, gids[gi], int(roots[k]), out)
        for key, t in tickets.items():
            r = _wait(d, srv, t)
            assert r.status == 0
        for (gi, k), out in outs.items():
            got = out if isinstance(out, np.ndarray) else out.cpu().numpy()
            np.testing.assert_array_equal(got, graphs[gi][3][k])
            if (gi, k) in alone:
                np.testing.assert_array_equal(got, alone[(gi, k)])
        st = d.dobfs_serve_get_stats(srv)
        assert st.completed == 9 + 3 * n_mix and st.in_flight == 0
    finally:
        d.dobfs_serve_destroy(srv)


def test_lanes_join_in_flight(d, graphs):
    g, og, roots, ref = graphs[2]
    srv = d.dobfs_serve_create()
    try:
        gid = d.dobfs_serve_add_graph(srv, g.handle)
        outs, tickets = [], []
        for k in range(40):  # staggered arrivals: later queries join traversals already running
            out = torch.full((og.n,), 9, dtype=torch.int32, device="cuda")
            outs.append(out)
            tickets.append(d.dobfs_serve_submit(srv, gid, int(roots[k]), out))
            time.sleep(0.0003 * (k % 5))
        for t in tickets:
            _wait(d, srv, t)
        for k, out in enumerate(outs):
            np.testing.assert_array_equal(out.cpu().numpy(), ref[k])
    finally:
        d.dobfs_serve_destroy(srv)


def test_admission_by_memory(d, graphs):
    g, og, roots, ref = graphs[0]
    # a budget that holds the lane group and two host-output staging buffers at a time
    probe = d.dobfs_serve_create(d.make_serve_opts(max_device_bytes=1 << 40))
    gid = d.dobfs_serve_add_graph(probe, g.handle)
    group_bytes = d.dobfs_serve_get_stats(probe).reserved_bytes
    d.dobfs_serve_destroy(probe)
    srv = d.dobfs_serve_create(d.make_serve_opts(max_device_bytes=group_bytes + 2 * 4 * og.n + 16,
                                                 max_groups_per_graph=1))
    try:
        gid = d.dobfs_serve_add_graph(srv, g.handle)
        outs = [np.full(og.n, 9, dtype=np.int32) for _ in range(10)]
        tickets = [d.dobfs_serve_submit(srv, gid, int(roots[k]), outs[k]) for k in range(10)]
        for t in tickets:
            _wait(d, srv, t)
        for k in range(10):
            np.testing.assert_array_equal(outs[k], ref[k])
        assert d.dobfs_serve_get_stats(srv).reserved_bytes == group_bytes
    finally:
        d.dobfs_serve_destroy(srv)
    tiny = d.dobfs_serve_create(d.make_serve_opts(max_device_bytes=1024))
    try:
        with pytest.raises(d.DobfsError) as e:
            d.dobfs_serve_add_graph(tiny, g.handle)
        assert e.value.status == d.DOBFS_ERR_BUSY
    finally:
        d.dobfs_serve_destroy(tiny)


def test_serve_errors(d, graphs):
    g, og, roots, ref = graphs[0]
    srv = d.dobfs_serve_create()
    try:
        gid = d.dobfs_serve_add_graph(srv, g.handle)
        out = torch.empty(og.n, dtype=torch.int32, device="cuda")
        for args in ((gid + 5, 0, out, None), (gid, og.n, out, None), (gid, 0, out, out)):
            with pytest.raises(d.DobfsError) as e:
                d.dobfs_serve_submit(srv, *args)
            assert e.value.status == d.DOBFS_ERR_INVALID
        with pytest.raises(d.DobfsError):
            d.dobfs_serve_poll(srv, 123456)
    finally:
        d.dobfs_serve_destroy(srv)


@pytest.mark.parametrize("direction", [2, 3])  # every step bottom-up; a seeded coin per lane and step
def test_lanes_join_bottom_up_steps(d, graphs, direction):
    """Lanes that join a group between steps start top-down: when the step
    chosen for the running lanes is bottom-up, the server runs it as a step
    of both kinds (the new lanes pushed top-down, the others searched
    bottom-up). Queries join at any level here, one at a time, into groups
    whose steps are bottom-up or mixed; every result is bit-exact."""
    g, og, roots, ref = graphs[2]
    srv = d.dobfs_serve_create(d.make_serve_opts(direction=direction, join_window=1000, admit_div=0, gather_us=0,
                                                 ss_max=0, flush_delay=0))
    try:
        gid = d.dobfs_serve_add_graph(srv, g.handle)
        outs, tickets = [], []
        for k in range(48):
            out = torch.full((og.n,), 9, dtype=torch.int32, device="cuda")
            outs.append(out)
            tickets.append(d.dobfs_serve_submit(srv, gid, int(roots[k]), out))
            time.sleep(0.0002 * (k % 7))
        for t in tickets:
            _wait(d, srv, t)
        for k, out in enumerate(outs):
            np.testing.assert_array_equal(out.cpu().numpy(), ref[k])
        assert d.dobfs_serve_get_stats(srv).cohorts < 48  # some queries joined running groups
    finally:
        d.dobfs_serve_destroy(srv)
