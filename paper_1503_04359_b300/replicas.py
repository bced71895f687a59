"""Host dispatcher over graph replicas, with failover.

Batched and served BFS shard by root: every replica holds the whole graph
(one per GPU) and the roots are independent, so scale-out needs no
collective. ``ReplicaPool`` hands roots out in chunks from one queue to one
host thread per replica. A replica whose run raises is retired and the chunk
it held goes back to the queue, so the others finish the job (failover); the
job fails only if every replica has been retired with roots left.

A replica is any callable ``fn(roots: np.ndarray) -> np.ndarray`` returning
one level row per root; ``gpu_replica`` makes one from a device graph.
Failures are host-side events (an exception from the call); nothing here
waits on a GPU.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field
from typing import Callable

import numpy as np


class ReplicaFailure(RuntimeError):
    """Every replica was retired before all roots were done."""

    def __init__(self, errors: dict[int, BaseException], remaining: int):
        super().__init__("all %d replicas failed with %d roots left: %s" %
                         (len(errors), remaining, "; ".join("replica %d: %r" % kv for kv in sorted(errors.items()))))
        self.errors = errors
        self.remaining = remaining


@dataclass
class PoolStats:
    chunks_done: dict[int, int] = field(default_factory=dict)  # replica -> chunks completed
    retired: dict[int, str] = field(default_factory=dict)      # replica -> error text
    requeued: int = 0                                          # chunks handed back after a failure
    seconds: float = 0.0


class ReplicaPool:
    def __init__(self, replicas: list[Callable[[np.ndarray], np.ndarray]], chunk: int = 64):
        if not replicas:
            raise ValueError("ReplicaPool needs at least one replica")
        if chunk < 1:
            raise ValueError("chunk must be >= 1")
        self.replicas = list(replicas)
        self.chunk = chunk
        self.stats = PoolStats()

    def run(self, roots, n_vertices: int) -> np.ndarray:
        """Level rows [len(roots), n_vertices], row i for roots[i]."""
        roots = np.ascontiguousarray(roots, dtype=np.int32)
        out = np.empty((len(roots), n_vertices), dtype=np.int32)
        todo = collections.deque((lo, min(len(roots), lo + self.chunk)) for lo in range(0, len(roots), self.chunk))
        lock = threading.Lock()
        cv = threading.Condition(lock)
        state = {"pending": len(todo), "alive": len(self.replicas)}
        errors: dict[int, BaseException] = {}
        stats = PoolStats(chunks_done={i: 0 for i in range(len(self.replicas))})
        t0 = time.perf_counter()

        def worker(i: int) -> None:
            fn = self.replicas[i]
            while True:
                with cv:
                    while not todo and state["pending"] > 0 and state["alive"] > 0:
                        cv.wait()  # another replica holds the last chunks: wait in case one fails
                    if not todo:
                        return
                    lo, hi = todo.popleft()
                try:
                    rows = np.asarray(fn(roots[lo:hi]))
                    if rows.shape != (hi - lo, n_vertices):
                        raise ValueError("replica returned shape %s for %d roots" % (rows.shape, hi - lo))
                    out[lo:hi] = rows
                except BaseException as e:  # noqa: BLE001 - any failure retires the replica
                    with cv:
                        todo.appendleft((lo, hi))
                        stats.requeued += 1
                        errors[i] = e
                        stats.retired[i] = repr(e)
                        state["alive"] -= 1
                        cv.notify_all()
                    return
                with cv:
                    state["pending"] -= 1
                    stats.chunks_done[i] += 1
                    cv.notify_all()

        threads = [threading.Thread(target=worker, args=(i,), daemon=True) for i in range(len(self.replicas))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        stats.seconds = time.perf_counter() - t0
        self.stats = stats
        if todo:
            raise ReplicaFailure(errors, sum(hi - lo for lo, hi in todo))
        return out


def gpu_replica(graph, device: int = 0, opts=None) -> Callable[[np.ndarray], np.ndarray]:
    """A replica running dobfs_run_batch on `graph` (a dobfs.Graph on `device`)."""
    import torch

    from . import dobfs

    def run(roots: np.ndarray) -> np.ndarray:
        with torch.cuda.device(device):
            stream = torch.cuda.current_stream()
            out = torch.empty((len(roots), graph.n), dtype=torch.int32, device="cuda")
            r = torch.from_numpy(np.ascontiguousarray(roots, dtype=np.int32)).cuda()
            o = opts if opts is not None else dobfs.make_opts(stream=stream)
            dobfs.dobfs_run_batch(graph.handle, r, out, opts=o)
            return out.cpu().numpy()

    return run
