"""Replica dispatcher on the GPU: two replicas of one graph (two device
copies on cuda:0, no kernel waits on another), one of them lost on its
first chunk (a host-side exception); the rows still equal the oracle's."""
import numpy as np
import pytest

import dobfs_inputs as inputs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_gpu_replicas_with_failover():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_04359_b300 import build, dobfs
    from paper_1503_04359_b300.replicas import ReplicaPool, gpu_replica
    build.build()
    dobfs.load()
    dobfs.use_torch_allocator()
    spec = inputs.rmat(14)
    og = oracle.csr_from_rmat(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 200, og.degrees() > 0)
    ref, _ = oracle.bfs_many(og, roots, want_parent=False)
    graphs = [dobfs.rmat_graph(spec) for _ in range(2)]
    healthy = gpu_replica(graphs[0])
    inner = gpu_replica(graphs[1])
    calls = [0]

    def flaky(r):
        calls[0] += 1
        if calls[0] == 1:
            raise RuntimeError("replica lost")
        return inner(r)

    pool = ReplicaPool([healthy, flaky], chunk=64)
    np.testing.assert_array_equal(pool.run(roots, og.n), ref)
    assert list(pool.stats.retired) == [1] and pool.stats.requeued == 1
    for g in graphs:
        g.close()
