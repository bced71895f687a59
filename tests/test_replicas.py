"""Replica dispatcher with failover (host side, CPU): roots split in chunks
over replicas; a replica that raises is retired and its chunk re-run by the
others. Replicas here are CPU callables (the oracle's BFS)."""
import threading
import time

import numpy as np
import pytest

import dobfs_inputs as inputs
import oracle
from paper_1503_04359_b300.replicas import ReplicaFailure, ReplicaPool


@pytest.fixture(scope="module")
def small():
    spec = inputs.rmat(9)
    og = oracle.csr_from_rmat(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 50, og.degrees() > 0)
    ref, _ = oracle.bfs_many(og, roots, want_parent=False)
    return og, roots, ref


def cpu_replica(og, fail_on_call=None, delay=0.0, log=None, name=None):
    calls = [0]

    def run(roots):
        calls[0] += 1
        if log is not None:
            log.append((name, len(roots)))
        if delay:
            time.sleep(delay)
        if fail_on_call is not None and calls[0] == fail_on_call:
            raise RuntimeError("replica %s lost" % name)
        return oracle.bfs_many(og, roots, want_parent=False)[0]

    return run


def test_all_healthy(small):
    og, roots, ref = small
    pool = ReplicaPool([cpu_replica(og, name=i) for i in range(3)], chunk=7)
    np.testing.assert_array_equal(pool.run(roots, og.n), ref)
    assert sum(pool.stats.chunks_done.values()) == 8 and not pool.stats.retired


def test_failover_reruns_the_lost_chunk(small):
    og, roots, ref = small
    log = []
    reps = [cpu_replica(og, fail_on_call=2, log=log, name="a", delay=0.01),
            cpu_replica(og, log=log, name="b", delay=0.01),
            cpu_replica(og, log=log, name="c", delay=0.01)]
    pool = ReplicaPool(reps, chunk=5)
    np.testing.assert_array_equal(pool.run(roots, og.n), ref)
    assert list(pool.stats.retired) == [0] and pool.stats.requeued == 1
    assert pool.stats.chunks_done[0] == 1
    assert sum(pool.stats.chunks_done.values()) == 10


def test_last_chunk_lost_while_others_idle(small):
    """The failing replica holds the last chunk: a replica already idle must
    wake up and take it back."""
    og, roots, ref = small
    gate = threading.Event()

    def slow_then_fail(r):
        gate.wait(5)
        raise RuntimeError("lost")

    fast = cpu_replica(og, name="fast")

    def fast_and_release(r):
        out = fast(r)
        gate.set()  # the failing replica gives up its chunk only after this one finished
        return out

    pool = ReplicaPool([slow_then_fail, fast_and_release], chunk=25)
    np.testing.assert_array_equal(pool.run(roots, og.n), ref)
    assert list(pool.stats.retired) == [0]


def test_every_replica_lost(small):
    og, roots, _ = small
    pool = ReplicaPool([cpu_replica(og, fail_on_call=1, name=i) for i in range(2)], chunk=10)
    with pytest.raises(ReplicaFailure) as e:
        pool.run(roots, og.n)
    assert set(e.value.errors) == {0, 1} and e.value.remaining > 0


def test_wrong_shape_retires(small):
    og, roots, ref = small
    pool = ReplicaPool([lambda r: np.zeros((1, 1), dtype=np.int32), cpu_replica(og, name="ok")], chunk=8)
    np.testing.assert_array_equal(pool.run(roots, og.n), ref)
    assert 0 in pool.stats.retired


def test_bad_arguments():
    with pytest.raises(ValueError):
        ReplicaPool([])
    with pytest.raises(ValueError):
        ReplicaPool([lambda r: r], chunk=0)
